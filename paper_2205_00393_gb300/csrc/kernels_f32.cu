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
#include "kernels.h"

namespace tnc {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
constexpr int LOG_BK = 4;

__device__ __forceinline__ int64_t slice_offset(const Operand& op, int64_t s) {
    int64_t off = 0;
    for (int j = 0; j < op.n_sl; ++j) off += ((s >> op.sl_bit[j]) & 1) * op.sl_stride[j];
    return off;
}

// sum of str[j] over the set bits j in [from, nbits) of x
__device__ __forceinline__ int64_t bits_offset(int64_t x, const int64_t* str, int nbits, int from) {
    int64_t off = 0;
    for (int j = from; j < nbits; ++j)
        if ((x >> j) & 1) off += str[j];
    return off;
}

__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

// C[m][n] = sum_k A(m,k) B(k,n), one 64x64 tile per CTA, 4x4 complex per thread.
__global__ void __launch_bounds__(NT) k_gemm_f32(const __grid_constant__ GemmParams p) {
    __shared__ float2 As[BK][BM + 1];
    __shared__ float2 Bs[BK][BN + 1];
    __shared__ int64_t rowA[BM], colB[BN], klA[BK], klB[BK];

    const int tid = threadIdx.x;
    const int64_t M = 1ll << p.mb, N = 1ll << p.nb, K = 1ll << p.kb;
    const int64_t tiles_n = (N + BN - 1) / BN;
    const int64_t tile = blockIdx.x;
    const int64_t m0 = (tile / tiles_n) * BM, n0 = (tile % tiles_n) * BN;
    const int z = blockIdx.z;
    const int64_t s = p.slice0 + z;
    const float2* __restrict__ A = p.A.ptr + z * p.A.batch_stride + slice_offset(p.A, s);
    const float2* __restrict__ B = p.B.ptr + z * p.B.batch_stride + slice_offset(p.B, s);

    if (tid < BM) rowA[tid] = (m0 + tid < M) ? bits_offset(m0 + tid, p.am, p.mb, 0) : 0;
    else if (tid < BM + BN) {
        int t = tid - BM;
        colB[t] = (n0 + t < N) ? bits_offset(n0 + t, p.bn, p.nb, 0) : 0;
    } else if (tid < BM + BN + BK) {
        int t = tid - BM - BN;
        klA[t] = bits_offset(t, p.ak, p.kb < LOG_BK ? p.kb : LOG_BK, 0);
    } else if (tid < BM + BN + 2 * BK) {
        int t = tid - BM - BN - BK;
        klB[t] = bits_offset(t, p.bk, p.kb < LOG_BK ? p.kb : LOG_BK, 0);
    }
    // load mapping: walk the operand's unit-stride mode with consecutive threads
    const bool a_kfast = p.kb > 0 && p.ak[0] == 1;
    const bool b_nfast = p.nb > 0 && p.bn[0] == 1;

    const int tx = tid & 15, ty = tid >> 4;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    __syncthreads();

    for (int64_t k0 = 0; k0 < K; k0 += BK) {
        const int64_t khA = bits_offset(k0, p.ak, p.kb, LOG_BK);
        const int64_t khB = bits_offset(k0, p.bk, p.kb, LOG_BK);
#pragma unroll
        for (int i = 0; i < (BM * BK) / NT; ++i) {
            int e = tid + i * NT;
            int kk, mm;
            if (a_kfast) { kk = e % BK; mm = e / BK; }
            else { mm = e % BM; kk = e / BM; }
            float2 v = make_float2(0.f, 0.f);
            if (m0 + mm < M && k0 + kk < K) v = A[rowA[mm] + khA + klA[kk]];
            As[kk][mm] = v;
        }
#pragma unroll
        for (int i = 0; i < (BN * BK) / NT; ++i) {
            int e = tid + i * NT;
            int kk, nn;
            if (b_nfast) { nn = e % BN; kk = e / BN; }
            else { kk = e % BK; nn = e / BK; }
            float2 v = make_float2(0.f, 0.f);
            if (n0 + nn < N && k0 + kk < K) v = B[colB[nn] + khB + klB[kk]];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cmac(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
    float2* C = p.C + z * p.c_batch_stride;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t n = n0 + tx + 16 * j;
            if (n < N) C[m * N + n] = acc[i][j];
        }
    }
}

// FP64 partial sums of a contraction with R = M*N <= 64 outputs.
__global__ void __launch_bounds__(256) k_root_partials(const __grid_constant__ RootParams rp,
                                                       double2* __restrict__ partials) {
    __shared__ double2 red[256];
    const GemmParams& p = rp.g;
    const int R = 1 << (p.mb + p.nb);
    const int lanes = 256 / R;
    const int r = threadIdx.x / lanes, lane = threadIdx.x % lanes;
    const int64_t m = r >> p.nb, n = r & ((1 << p.nb) - 1);
    const int z = blockIdx.y;
    const int64_t s = p.slice0 + z;
    const float2* A = p.A.ptr + z * p.A.batch_stride + slice_offset(p.A, s) + bits_offset(m, p.am, p.mb, 0);
    const float2* B = p.B.ptr + z * p.B.batch_stride + slice_offset(p.B, s) + bits_offset(n, p.bn, p.nb, 0);
    const int64_t K = 1ll << p.kb;
    const int64_t kc = K / rp.chunks;
    const int64_t k_lo = blockIdx.x * kc, k_hi = k_lo + kc;
    double re = 0.0, im = 0.0;
    for (int64_t k = k_lo + lane; k < k_hi; k += lanes) {
        float2 a = A[bits_offset(k, p.ak, p.kb, 0)];
        float2 b = B[bits_offset(k, p.bk, p.kb, 0)];
        re += (double)a.x * b.x - (double)a.y * b.y;
        im += (double)a.x * b.y + (double)a.y * b.x;
    }
    red[threadIdx.x] = make_double2(re, im);
    __syncthreads();
    for (int st = lanes / 2; st > 0; st >>= 1) {
        if (lane < st) {
            double2 o = red[threadIdx.x + st];
            red[threadIdx.x].x += o.x;
            red[threadIdx.x].y += o.y;
        }
        __syncthreads();
    }
    if (lane == 0) partials[((int64_t)z * rp.chunks + blockIdx.x) * R + r] = red[threadIdx.x];
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

cudaError_t launch_gemm_f32(const GemmParams& p, int batch, cudaStream_t s) {
    int64_t M = 1ll << p.mb, N = 1ll << p.nb;
    int64_t tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    if (tiles > 0x7fffffffll || batch < 1 || batch > 65535) return cudaErrorInvalidConfiguration;
    k_gemm_f32<<<dim3((unsigned)tiles, 1, batch), NT, 0, s>>>(p);
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
