// Kernels of the adjoint (reverse-mode) pass.
//
// For a pairwise contraction C = A (x) B of the tree, the environment of a
// child, E_A = dF/dA for F = sum_o g_o O_o (holomorphic), is the contraction
// of E_C with the sibling B over B's free indices, and likewise for B; the
// environment GEMMs themselves run on the gather-fused FP32 GEMM. The kernels
// here seed the root environment, fold per-slice environments into leaves
// (each slice fixes the leaf's sliced modes, Sec. 2.1.1) and into the
// environments of slice-invariant tensors, and apply the chain rule to gate
// parameters. Accumulation over slices is FP64.
#include "kernels.h"

namespace tnc {

namespace {

__device__ __forceinline__ int64_t bits_offset(int64_t x, const int64_t* str, int nbits) {
    int64_t off = 0;
    for (int j = 0; j < nbits; ++j)
        if ((x >> j) & 1) off += str[j];
    return off;
}

// E_z[root offset of r] = g[r] for every slice z of the batch (FP32).
__global__ void k_env_seed(const __grid_constant__ SeedParams p, int batch) {
    const int64_t R = 1ll << p.obits;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int64_t off = bits_offset(r, p.ostride, p.obits);
    const double2 g = p.grad[r];
    const float2 v = make_float2((float)g.x, (float)g.y);
    for (int z = 0; z < batch; ++z) p.E[z * p.batch_stride + off] = v;
}

// grad[e] += sum over slices z of the batch whose sliced bits match leaf
// element e of E_z[unsliced part of e]; one thread per leaf element, z in order.
__global__ void k_leaf_env_accum(const __grid_constant__ LeafEnvParams p, int batch) {
    const int64_t n = 1ll << p.L;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double ax = 0.0, ay = 0.0;
    for (int z = 0; z < batch; ++z) {
        const int64_t s = p.slice0 + z;
        bool ok = true;
        int64_t off = 0;
        for (int q = 0; q < p.L; ++q) {
            const int bit = (int)((e >> (p.L - 1 - q)) & 1);
            if (p.sl_bit[q] >= 0) {
                if ((int)((s >> p.sl_bit[q]) & 1) != bit) {
                    ok = false;
                    break;
                }
            } else if (bit) {
                off += p.env_stride[q];
            }
        }
        if (ok) {
            const float2 v = p.env[z * p.env_batch_stride + off];
            ax += v.x;
            ay += v.y;
        }
    }
    p.grad[e].x += ax;
    p.grad[e].y += ay;
}

// acc[i] += sum_z E[z * bs + i] in FP64, z in order.
__global__ void k_accum_batch_f64(const float2* __restrict__ E, int64_t n, int batch, int64_t bs,
                                  double2* __restrict__ acc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double ax = 0.0, ay = 0.0;
    for (int z = 0; z < batch; ++z) {
        const float2 v = E[z * bs + i];
        ax += v.x;
        ay += v.y;
    }
    acc[i].x += ax;
    acc[i].y += ay;
}

__global__ void k_f64_to_f32(const double2* __restrict__ src, int64_t n, float2* __restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

// out[q] = sum_e env[env_off[q] + e] * d[d_off[q] + e], e < size[q], in FP64.
__global__ void __launch_bounds__(256) k_param_grads(const int64_t* __restrict__ env_off,
                                                     const int64_t* __restrict__ d_off,
                                                     const int64_t* __restrict__ size,
                                                     const float2* __restrict__ env,
                                                     const float2* __restrict__ d, double2* __restrict__ out) {
    __shared__ double2 red[256];
    const int q = blockIdx.x;
    const int64_t n = size[q];
    double ax = 0.0, ay = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        const float2 a = env[env_off[q] + e], b = d[d_off[q] + e];
        ax += (double)a.x * b.x - (double)a.y * b.y;
        ay += (double)a.x * b.y + (double)a.y * b.x;
    }
    red[threadIdx.x] = make_double2(ax, ay);
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            red[threadIdx.x].x += red[threadIdx.x + st].x;
            red[threadIdx.x].y += red[threadIdx.x + st].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = red[0];
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

cudaError_t launch_env_seed(const SeedParams& p, int batch, cudaStream_t s) {
    k_env_seed<<<blocks_for(1ll << p.obits), 256, 0, s>>>(p, batch);
    return cudaGetLastError();
}

cudaError_t launch_leaf_env_accum(const LeafEnvParams& p, int batch, cudaStream_t s) {
    if (p.L > 31) return cudaErrorInvalidValue;
    k_leaf_env_accum<<<blocks_for(1ll << p.L), 256, 0, s>>>(p, batch);
    return cudaGetLastError();
}

cudaError_t launch_accum_batch_f64(const float2* E, int64_t n, int batch, int64_t bs, double2* acc,
                                   cudaStream_t s) {
    k_accum_batch_f64<<<blocks_for(n), 256, 0, s>>>(E, n, batch, bs, acc);
    return cudaGetLastError();
}

cudaError_t launch_f64_to_f32(const double2* src, int64_t n, float2* dst, cudaStream_t s) {
    k_f64_to_f32<<<blocks_for(n), 256, 0, s>>>(src, n, dst);
    return cudaGetLastError();
}

cudaError_t launch_param_grads(int n, const int64_t* env_off, const int64_t* d_off, const int64_t* size,
                               const float2* env, const float2* d, double2* out, cudaStream_t s) {
    if (n < 1) return cudaSuccess;
    k_param_grads<<<n, 256, 0, s>>>(env_off, d_off, size, env, d, out);
    return cudaGetLastError();
}

}  // namespace tnc
