// FP32 CUDA-core kernels of libtnc: the permute-fused complex64 contraction
// GEMM, the FP64 final reduction and the FP64 slice sum.
//
// Pairwise contraction (Sec. 2.1.1) in the TTGT arrangement of Sec. 5.3.1
// (free modes of A first, contracted modes last; contracted modes of B first):
// the permutation is folded into the operand load. Each binary mode of an
// operand has an element stride; the address of A(m, k) is the sum of the
// strides of the set bits of m and k. As in the paper's recursion formula
// (Sec. 5.3.1, map[i+k] = map[i] + k*offset) only the tile-local low bits go
// through a table; the high bits of a tile origin contribute one offset.
#include "f32_device.cuh"
#include "kernels.h"

namespace tnc {

namespace {

using namespace f32dev;

__global__ void __launch_bounds__(NT, 2) k_gemm_f32(const __grid_constant__ GemmParams p) {
    extern __shared__ __align__(16) uint8_t gemm_dyn[];
    GemmSmem& sm = *reinterpret_cast<GemmSmem*>(gemm_dyn);
    gemm_tile(p, blockIdx.x, blockIdx.z, p.slice0, sm);
}

// Many independent contractions in one launch (nodes of one tree level): CTA
// b serves tile b - tile_off[i] of node i, tile_off[i] <= b < tile_off[i+1].
__global__ void __launch_bounds__(NT, 2) k_gemm_f32_group(const GemmParams* __restrict__ params,
                                                       const int64_t* __restrict__ tile_off, int n,
                                                       int64_t slice0) {
    extern __shared__ __align__(16) uint8_t gemm_dyn[];
    GemmSmem& sm = *reinterpret_cast<GemmSmem*>(gemm_dyn);
    const int64_t b = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tile_off[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    gemm_tile(params[lo], b - tile_off[lo], blockIdx.z, slice0, sm);
}

// FP64 partial sums of a contraction with R = M*N <= 64 outputs.
__global__ void __launch_bounds__(256) k_root_partials(const __grid_constant__ RootParams rp,
                                                       double2* __restrict__ partials) {
    __shared__ double2 red[256];
    __shared__ int64_t root_ta[5][256], root_tb[5][256];  // offsets of 8-bit groups of j (K <= 2^40)
    const int R = 1 << (rp.g.mb + rp.g.nb);
    const int z = blockIdx.y;
    root_chunk<0>(rp, blockIdx.x, z, rp.g.slice0, partials + ((int64_t)z * rp.chunks + blockIdx.x) * R, red, root_ta,
                  root_tb);
}

// out[r] += sum_i partials[i][perm(r)], i ascending (fixed order)
__global__ void k_accumulate_partials(const double2* __restrict__ partials, int count,
                                      const __grid_constant__ PermParams pp, double2* __restrict__ out) {
    const int64_t R = 1ll << pp.obits;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int64_t src = bits_offset(r, pp.ostride, pp.obits, 0);
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < count; ++i) {
        double2 v = partials[(int64_t)i * R + src];
        acc.x += v.x;
        acc.y += v.y;
    }
    out[r].x += acc.x;
    out[r].y += acc.y;
}

// out[r] += sum_z src_z[perm(r)] in FP64, z ascending
__global__ void k_slice_sum_f32(const __grid_constant__ SumParams p, int batch, double2* __restrict__ out) {
    const int64_t R = 1ll << p.obits;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int64_t off = bits_offset(r, p.ostride, p.obits, 0);
    double2 acc = make_double2(0.0, 0.0);
    for (int z = 0; z < batch; ++z) {
        const float2* src = p.src.ptr + z * p.src.batch_stride + slice_offset(p.src, p.slice0 + z);
        float2 v = src[off];
        acc.x += v.x;
        acc.y += v.y;
    }
    out[r].x += acc.x;
    out[r].y += acc.y;
}

}  // namespace

__global__ void __launch_bounds__(NT, 2) k_gemm_f32_group_multi(const GemmParams* __restrict__ params,
                                                             const int64_t* __restrict__ tile_off, int n,
                                                             const int* __restrict__ net,
                                                             const int64_t* __restrict__ rs0,
                                                             const int* __restrict__ rb);

// The FP32 GEMM kernels take GemmSmem (over 48 KB) as dynamic shared memory;
// the limit is raised once per process (a host-side setting, not a stream
// operation, so it is safe before or during graph capture).
cudaError_t gemm_smem_attr() {
    static cudaError_t done = [] {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GemmSmem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_gemm_f32_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GemmSmem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_gemm_f32_group_multi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(GemmSmem));
        return e;
    }();
    return done;
}

cudaError_t launch_gemm_f32(const GemmParams& p, int batch, cudaStream_t s) {
    int64_t M = 1ll << p.mb, N = 1ll << p.nb;
    int64_t tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    if (tiles > 0x7fffffffll || batch < 1 || batch > 65535) return cudaErrorInvalidConfiguration;
    cudaError_t e = gemm_smem_attr();
    if (e != cudaSuccess) return e;
    k_gemm_f32<<<dim3((unsigned)tiles, 1, batch), NT, sizeof(GemmSmem), s>>>(p);
    return cudaGetLastError();
}

// Grouped contractions of several networks: node i belongs to network
// net[i]; slice z of the launch maps to slice rs0[net] + z of that network and
// exists only for z < rb[net] (networks batch different numbers of slices).
__global__ void __launch_bounds__(NT, 2) k_gemm_f32_group_multi(const GemmParams* __restrict__ params,
                                                             const int64_t* __restrict__ tile_off, int n,
                                                             const int* __restrict__ net,
                                                             const int64_t* __restrict__ rs0,
                                                             const int* __restrict__ rb) {
    extern __shared__ __align__(16) uint8_t gemm_dyn[];
    GemmSmem& sm = *reinterpret_cast<GemmSmem*>(gemm_dyn);
    const int64_t b = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tile_off[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const int w = net[lo];
    if ((int)blockIdx.z >= rb[w]) return;
    gemm_tile(params[lo], b - tile_off[lo], blockIdx.z, rs0[w], sm);
}

// Root reductions of several networks in one launch: block x serves chunk
// x - blk_off[i] of network i; partial sums go to that network's buffer.
__global__ void __launch_bounds__(256) k_root_partials_multi(const RootParams* __restrict__ roots,
                                                             double2* const* __restrict__ partials,
                                                             const int64_t* __restrict__ blk_off, int n,
                                                             const int64_t* __restrict__ rs0,
                                                             const int* __restrict__ rb) {
    __shared__ double2 red[256];
    __shared__ int64_t root_ta[5][256], root_tb[5][256];
    const int64_t x = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (blk_off[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    const int z = blockIdx.z;
    if (z >= rb[lo]) return;
    const RootParams& rp = roots[lo];
    const int chunk = (int)(x - blk_off[lo]);
    const int R = 1 << (rp.g.mb + rp.g.nb);
    root_chunk<0>(rp, chunk, z, rs0[lo], partials[lo] + ((int64_t)z * rp.chunks + chunk) * R, red, root_ta, root_tb);
}

// out_i[r] += sum over network i's partial sums (slices in order, then chunks).
__global__ void k_accumulate_multi(const RootParams* __restrict__ roots, double2* const* __restrict__ partials,
                                   const PermParams* __restrict__ perms, double2* const* __restrict__ outs,
                                   const int* __restrict__ rb) {
    const int i = blockIdx.x;
    const PermParams& pp = perms[i];
    const int64_t R = 1ll << pp.obits;
    const int count = rb[i] * roots[i].chunks;
    for (int64_t r = threadIdx.x; r < R; r += blockDim.x) {
        const int64_t src = bits_offset(r, pp.ostride, pp.obits, 0);
        double2 acc = make_double2(0.0, 0.0);
        for (int c = 0; c < count; ++c) {
            double2 v = partials[i][(int64_t)c * R + src];
            acc.x += v.x;
            acc.y += v.y;
        }
        outs[i][r].x += acc.x;
        outs[i][r].y += acc.y;
    }
}

int64_t gemm_f32_tiles(int mb, int nb) {
    int64_t M = 1ll << mb, N = 1ll << nb;
    return ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
}

cudaError_t launch_gemm_f32_group(const GemmParams* d_params, const int64_t* d_tile_off, int n,
                                  int64_t total_tiles, int64_t slice0, int batch, cudaStream_t s) {
    if (n < 1 || total_tiles < 1 || total_tiles > 0x7fffffffll || batch < 1 || batch > 65535)
        return cudaErrorInvalidConfiguration;
    cudaError_t e = gemm_smem_attr();
    if (e != cudaSuccess) return e;
    k_gemm_f32_group<<<dim3((unsigned)total_tiles, 1, batch), NT, sizeof(GemmSmem), s>>>(d_params, d_tile_off, n,
                                                                                       slice0);
    return cudaGetLastError();
}

cudaError_t launch_gemm_f32_group_multi(const GemmParams* d_params, const int64_t* d_tile_off, int n,
                                        int64_t total_tiles, const int* d_net, const int64_t* d_rs0,
                                        const int* d_rb, int max_batch, cudaStream_t s) {
    if (n < 1 || total_tiles < 1 || total_tiles > 0x7fffffffll || max_batch < 1 || max_batch > 65535)
        return cudaErrorInvalidConfiguration;
    cudaError_t e = gemm_smem_attr();
    if (e != cudaSuccess) return e;
    k_gemm_f32_group_multi<<<dim3((unsigned)total_tiles, 1, max_batch), NT, sizeof(GemmSmem), s>>>(
        d_params, d_tile_off, n, d_net, d_rs0, d_rb);
    return cudaGetLastError();
}

cudaError_t launch_root_multi(const RootParams* d_roots, double2* const* d_partials, const int64_t* d_blk_off,
                              int n, int64_t total_blocks, const PermParams* d_perms, double2* const* d_outs,
                              const int64_t* d_rs0, const int* d_rb, int max_batch, cudaStream_t s) {
    if (n < 1 || total_blocks < 1 || total_blocks > 0x7fffffffll || max_batch < 1 || max_batch > 65535)
        return cudaErrorInvalidConfiguration;
    k_root_partials_multi<<<dim3((unsigned)total_blocks, 1, max_batch), 256, 0, s>>>(d_roots, d_partials, d_blk_off,
                                                                                   n, d_rs0, d_rb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_accumulate_multi<<<n, 256, 0, s>>>(d_roots, d_partials, d_perms, d_outs, d_rb);
    return cudaGetLastError();
}

cudaError_t launch_root_partials(const RootParams& p, int batch, double2* partials, cudaStream_t s) {
    if (p.g.mb + p.g.nb > 6 || batch < 1 || batch > 65535) return cudaErrorInvalidConfiguration;
    k_root_partials<<<dim3(p.chunks, batch), 256, 0, s>>>(p, partials);
    return cudaGetLastError();
}

cudaError_t launch_accumulate_partials(const double2* partials, int count, const PermParams& pp,
                                       double2* out, cudaStream_t s) {
    int64_t R = 1ll << pp.obits;
    k_accumulate_partials<<<(unsigned)((R + 255) / 256), 256, 0, s>>>(partials, count, pp, out);
    return cudaGetLastError();
}

cudaError_t launch_slice_sum_f32(const SumParams& p, int batch, double2* out, cudaStream_t s) {
    int64_t R = 1ll << p.obits;
    k_slice_sum_f32<<<(unsigned)((R + 255) / 256), 256, 0, s>>>(p, batch, out);
    return cudaGetLastError();
}

}  // namespace tnc
