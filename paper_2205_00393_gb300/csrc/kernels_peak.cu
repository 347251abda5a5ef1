// Peak-rate probes: the denominators of the roofline fractions that the
// benchmark reports, measured by this library's own kernels on the GPU at
// hand instead of taken from unit counts and nominal ratios.
//
//  kind 0: FP32 FMA on the CUDA cores. Every thread runs 8 independent FMA
//          chains; 2 flops per FMA.
//  kind 1: tcgen05.mma kind::tf32, M = 128, N = 256, K = 8 per instruction.
//  kind 2: tcgen05.mma kind::f16 with BF16 operands, M = 128, N = 256, K = 16.
//  kind 3: tcgen05.mma kind::f16 with FP16 operands, same shape.
// The MMA probes run one CTA per SM: one thread issues MMAs back to back on
// operands resident in shared memory (64-byte swizzled K-major tiles filled
// with nonzero values) into one TMEM accumulator, committing to an mbarrier
// every 64 instructions and waiting for that commit (bounded) before issuing
// further, so the tensor pipe is kept full without an unbounded queue.
#include <cuda.h>

#include "kernels.h"
#include "tnc.h"

namespace {

constexpr int kChains = 8;
constexpr int kMmaBatch = 64;
constexpr uint32_t kPeakSpin = 1u << 26;

__global__ void __launch_bounds__(256) k_peak_ffma(int64_t iters, float* sink) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 1.0f + 1e-3f * (float)(threadIdx.x + j);
    const float b = 0.99999994f, c = 1e-7f;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == -1.0f) sink[0] = s;  // never taken; keeps the chains alive
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// K-major, 64-byte swizzle, 8-row groups 512 bytes apart, descriptor version 1
__device__ __forceinline__ uint64_t desc64(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

template <int KIND>  // 1 tf32, 2 bf16, 3 fp16
__global__ void __launch_bounds__(128, 1) k_peak_mma(int64_t iters, int* err) {
    constexpr uint32_t fmt = KIND == 1 ? 2u : (KIND == 2 ? 1u : 0u);
    constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
    __shared__ __align__(1024) uint8_t tiles[(128 + 256) * 64];  // A: 128 rows, B: 256 rows, 64 bytes of K each
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_sh;
    const int warp = threadIdx.x >> 5;
    // nonzero operands: small values in both formats (bit patterns of ~0.5 .. 1)
    uint32_t* w = reinterpret_cast<uint32_t*>(tiles);
    for (int i = threadIdx.x; i < (128 + 256) * 16; i += 128)
        w[i] = KIND == 1 ? 0x3F000000u + ((uint32_t)i << 8) : (KIND == 2 ? 0x3F003F00u + (i & 0x7F) : 0x38003800u + (i & 0x3FF));
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_sh))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_sh;
    if (threadIdx.x == 0) {
        const uint64_t a = desc64(smem_u32(tiles)), b = desc64(smem_u32(tiles + 128 * 64));
        uint32_t phase = 0;
        bool ok = true;
        for (int64_t it = 0; it < iters && ok; it += kMmaBatch) {
            for (int j = 0; j < kMmaBatch; ++j) {
                const uint32_t acc = (it > 0 || j > 0) ? 1u : 0u;
                if constexpr (KIND == 1)
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                                 : "memory");
                else
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                                 : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar))
                         : "memory");
            uint32_t i = 0;
            while (i < kPeakSpin && !mbar_try(smem_u32(&bar), phase)) ++i;
            if (i == kPeakSpin) {
                atomicExch(err, 4);
                ok = false;
            }
            phase ^= 1u;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
    }
}

float* g_sink = nullptr;
int* g_err = nullptr;

}  // namespace

extern "C" tnc_status tnc_peak_probe(int kind, int64_t iters, double* flops_out, void* stream) {
    auto fail = [](tnc_status st, const std::string& m) {
        tnc::set_last_error(m);
        return st;
    };
    if (!flops_out) return fail(TNC_E_INVALID, "NULL output");
    if (kind < 0 || kind > 3 || iters < 1 || iters > (1ll << 30)) return fail(TNC_E_INVALID, "bad kind or iters");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(TNC_E_CUDA, "device query failed");
    if (!g_sink) {
        if (cudaMalloc(&g_sink, 256) != cudaSuccess) return fail(TNC_E_OOM, "probe buffer");
        g_err = reinterpret_cast<int*>(g_sink + 32);
        if (cudaMemset(g_sink, 0, 256) != cudaSuccess) return fail(TNC_E_CUDA, "probe buffer");
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (kind == 0) {
        const int blocks = sms * 8;  // 2048 threads per SM
        k_peak_ffma<<<blocks, 256, 0, s>>>(iters, g_sink);
        *flops_out = (double)blocks * 256 * (double)iters * 16 * kChains * 2;
    } else {
        iters = (iters + kMmaBatch - 1) / kMmaBatch * kMmaBatch;
        const int k = kind == 1 ? 8 : 16;
        if (kind == 1) k_peak_mma<1><<<sms, 128, 0, s>>>(iters, g_err);
        else if (kind == 2) k_peak_mma<2><<<sms, 128, 0, s>>>(iters, g_err);
        else k_peak_mma<3><<<sms, 128, 0, s>>>(iters, g_err);
        *flops_out = (double)sms * (double)iters * 2.0 * 128 * 256 * k;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TNC_E_CUDA, std::string("probe launch: ") + cudaGetErrorString(e));
    return TNC_OK;
}
