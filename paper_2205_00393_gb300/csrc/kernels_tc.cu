// Split-precision complex GEMM on the 5th-generation tensor cores (tcgen05).
//
// A pairwise contraction C[m,n] = sum_k A(m,k) B(k,n) (Sec. 2.1.1, in the
// TTGT arrangement of Sec. 5.3.1) runs in two kernels:
//
//  1. k_split_operand: the permute-fused operand load. It gathers the FP32
//     complex operand through its per-bit stride table (the permutation and
//     the slice fixing), stages a 32x64 tile in shared memory so that both the
//     gather and the writes are coalesced, and writes, for each of the three
//     real matrices of the 3M complex product (Re, Im, Re+Im), the split
//     parts as K-major planes:  BF16: x = x0 + x1 + x2 (three parts),
//     TF32: x = x0 + x1 (two parts).
//  2. k_cgemm_tc: a warp-specialised tcgen05 GEMM on 128x128 output tiles.
//     One warp issues TMA loads (128-byte swizzle, the three or two parts of
//     one real matrix per box) into a shared-memory ring guarded by mbarriers;
//     one thread issues tcgen05.mma (kind::f16 or kind::tf32, FP32
//     accumulation) for every part pair (i, j) with i + j <= 2 (BF16) or
//     i + j <= 1 (TF32) into one of three TMEM accumulators
//     T1 = Re A Re B, T2 = Im A Im B, T3 = (Re+Im)A (Re+Im)B; eight epilogue
//     warps move each K-chunk's T1..T3 into FP32 registers and finally write
//     C = (T1 - T2) + i (T3 - T1 - T2).
//
// Every mbarrier wait is bounded; a wait that gives up records an error code
// in the caller's error word, the CTA drains its own copies in flight, frees
// its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>

#include "kernels.h"

namespace tnc {

namespace {

constexpr int TM = 128, TN = 128;
constexpr int SMEM_PIPE = 192 * 1024;             // shared memory for the TMA ring
constexpr uint32_t kSpinLimit = 1u << 24;
constexpr int kErrTimeout = 4;

// KIND 0: three BF16 parts (6 pairs), kind::f16; 1: two TF32 parts (3 pairs),
// kind::tf32; 2: two BF16 parts (3 pairs), kind::f16; 3: two FP16 parts of
// the operand scaled by a power of two (3 pairs), kind::f16. ROWB: bytes of K
// per tile row and k-block, which is also the swizzle width (64 or 128).
template <int KIND, int ROWB> struct Cfg {
    static constexpr int PARTS = KIND == 0 ? 3 : 2;
    static constexpr int NPAIRS = KIND == 0 ? 6 : 3;
    static constexpr int ELEM = KIND == 1 ? 4 : 2;
    static constexpr int BK = ROWB / ELEM;                     // K elements per k-block
    static constexpr int PART_TILE = 128 * ROWB;               // bytes of one part tile
    static constexpr int STAGE_BYTES = 2 * PARTS * PART_TILE;  // A and B parts of one product
    static constexpr int STAGES = SMEM_PIPE / STAGE_BYTES;
    static constexpr int KSTEPS = ROWB / 32;                   // MMAs per k-block (32 bytes of K each)
};

// Split FP16x2 operand scale. With m = max |Re|, |Im| of the operand, the
// scale 2^e puts m * 2^e in [2^13, 2^14), so Re + Im (at most 2m) stays below
// the FP16 maximum; x = x0 + x1 carries 22 significant bits wherever x1 is a
// normal FP16 (|x| >= m 2^-16), and below that an absolute error under
// m 2^-38 (half the FP16 subnormal spacing after scaling). e is clamped to
// [-126, 126] so that 2^e and 2^-e are normal floats.
__host__ __device__ __forceinline__ int fp16_scale_exp(uint32_t amax_bits) {
    if (amax_bits == 0) return 0;
    const int e = 140 - (int)((amax_bits >> 23) & 0xFFu);
    return e < -126 ? -126 : (e > 126 ? 126 : e);
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
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

// Bounded wait; false if it gave up or another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          uint32_t limit = kSpinLimit) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 255) == 255 && *abort_flag) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            int c3, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major, ROWB-byte swizzle (layout type
// 2 = 128B, 4 = 64B), 8-row groups 8*ROWB bytes apart, descriptor version 1.
template <int ROWB>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)((8 * ROWB) >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;                    // version
    d |= (uint64_t)(ROWB == 128 ? 2 : 4) << 61;
    return d;
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (KIND != 1) {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Instruction descriptor: FP32 accumulator, A/B format (1 = BF16, 2 = TF32),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
// A/B format: kind::f16 0 = F16, 1 = BF16; kind::tf32 2 = TF32.
template <int KIND>
__host__ __device__ constexpr uint32_t ab_format() {
    return KIND == 1 ? 2u : (KIND == 3 ? 0u : 1u);
}

template <int KIND>
__host__ __device__ constexpr uint32_t instr_desc() {
    return (1u << 4) | (ab_format<KIND>() << 7) | (ab_format<KIND>() << 10) |
           ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// Part pairs, smallest magnitudes first.
__constant__ int kPairsBF16[6][2] = {{1, 1}, {0, 2}, {2, 0}, {0, 1}, {1, 0}, {0, 0}};
__constant__ int kPairs2[3][2] = {{0, 1}, {1, 0}, {0, 0}};

// K is processed in chunks of KC_ELEMS. Within a chunk the three real
// products run one after the other (product-major), each accumulating in its
// own TMEM columns; when a product's chunk is complete the epilogue warps move
// it into FP32 registers (Cr += T1 - T2, Ci += T3 - T1 - T2) while the tensor
// cores work on the next product. The tensor core's accumulation into TMEM
// does not round to nearest, so its error grows linearly with the number of
// accumulated MMAs; short chunks bound that growth and the register sums
// across chunks round to nearest.
constexpr int KC_ELEMS = 256;
constexpr int EPI_WARPS = 8;   // warps 0-7: epilogue (warp w: TMEM lanes 32*(w%4), columns 64*(w/4))
constexpr int EPI_LDW = 66;    // float2 per row of a warp's staged 32 x 64 output block (2 of padding)
static_assert(EPI_WARPS * 32 * EPI_LDW * 8 <= SMEM_PIPE, "staged epilogue fits the pipeline ring");
constexpr int PRODUCER_WARP = 8, MMA_WARP = 9, NTHREADS = 320;

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int KIND, int ROWB>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_cgemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ TcGemmParams p) {
    using C_ = Cfg<KIND, ROWB>;
    constexpr int PART_TILE_BYTES = C_::PART_TILE;
    constexpr int STAGE_A = C_::PARTS * PART_TILE_BYTES;
    constexpr int STAGE_BYTES = 2 * STAGE_A;
    const int GROUP_M = p.group_m < 1 ? 1 : p.group_m;
    extern __shared__ __align__(1024) uint8_t dsmem[];
    __shared__ __align__(8) uint64_t full_bar[C_::STAGES], empty_bar[C_::STAGES], tfull[3], tfree[3], drain_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~uintptr_t(1023));
    const int64_t N = 1ll << p.nb, K = 1ll << p.kb;
    // grouped rasterisation: consecutive CTAs cover GROUP_M row tiles x all column tiles
    const int64_t tiles_n = N / TN, tiles_m = (1ll << p.mb) / TM;
    const int64_t per_group = (int64_t)GROUP_M * tiles_n;
    const int64_t cta = blockIdx.x;
    const int64_t grp = cta / per_group, in_grp = cta % per_group;
    const int64_t gm = (tiles_m - grp * GROUP_M) < GROUP_M ? (tiles_m - grp * GROUP_M) : GROUP_M;
    const int m0 = (int)((grp * GROUP_M + in_grp % gm) * TM);
    const int n0 = (int)((in_grp / gm) * TN);
    const int z = blockIdx.z;
    const int za = p.a_shared ? 0 : z, zb = p.b_shared ? 0 : z;  // batch entry of each operand's planes
    const int nkb = (int)((K >> p.ksplit_bits) / C_::BK);  // k-blocks of this CTA's K split
    const int kb_off = (int)blockIdx.y * nkb;
    const int kpc = nkb < KC_ELEMS / C_::BK ? nkb : KC_ELEMS / C_::BK;  // k-blocks per chunk
    const int nchunks = nkb / kpc;
    const int n_it = nchunks * 3 * kpc;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C_::STAGES; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int t = 0; t < 3; ++t) {
            mbar_init(smem_u32(&tfull[t]), 1);
            mbar_init(smem_u32(&tfree[t]), EPI_WARPS);
        }
        mbar_init(smem_u32(&drain_bar), 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;
    volatile int* abort_flag = &abort_sh;
    const uint32_t spin = p.spin_limit ? p.spin_limit : kSpinLimit;

    if (warp == PRODUCER_WARP && lane == 0) {
        // ---------------- TMA producer: stages in (chunk, product, k-block) order
        int issued = 0;
        for (int it = 0; it < n_it && !p.test_stall; ++it) {
            const int s = it % C_::STAGES;
            const uint32_t ph = (uint32_t)(it / C_::STAGES) & 1u;
            if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, abort_flag, spin)) {
                abort_sh = 1;
                atomicExch(p.err, kErrTimeout);
                break;
            }
            const int c = it / (3 * kpc), r = it % (3 * kpc);
            const int t = r / kpc, kb = c * kpc + r % kpc;
            const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
            const uint32_t fb = smem_u32(&full_bar[s]);
            mbar_expect_tx(fb, STAGE_BYTES);
            tma_load_4d(sa, &tmA, (kb + kb_off) * C_::BK, m0, t * C_::PARTS, za, fb);
            tma_load_4d(sa + STAGE_A, &tmB, (kb + kb_off) * C_::BK, n0, t * C_::PARTS, zb, fb);
            issued = it + 1;
        }
        if (*abort_flag) {
            // drain: wait (bounded) for every load that may still be in flight
            int first = issued - C_::STAGES < 0 ? 0 : issued - C_::STAGES;
            for (int it = first; it < issued; ++it) {
                const int s = it % C_::STAGES;
                const uint32_t ph = (uint32_t)(it / C_::STAGES) & 1u;
                for (uint32_t i = 0; i < spin && !mbar_try(smem_u32(&full_bar[s]), ph); ++i) {
                }
            }
        }
    } else if (warp == MMA_WARP && lane == 0) {
        // ---------------- MMA issuer
        constexpr uint32_t idesc = instr_desc<KIND>();
        bool any = false;
        for (int it = 0; it < n_it && !*abort_flag; ++it) {
            const int s = it % C_::STAGES;
            const uint32_t ph = (uint32_t)(it / C_::STAGES) & 1u;
            const int c = it / (3 * kpc), r = it % (3 * kpc);
            const int t = r / kpc, kbi = r % kpc;
            if ((kbi == 0 && c > 0 && !mbar_wait(smem_u32(&tfree[t]), (uint32_t)(c - 1) & 1u, abort_flag, spin)) ||
                !mbar_wait(smem_u32(&full_bar[s]), ph, abort_flag, spin)) {
                abort_sh = 1;
                atomicExch(p.err, kErrTimeout);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
            const uint32_t sb = sa + STAGE_A;
            const uint32_t d = tmem + (uint32_t)(t * TN);
#pragma unroll
            for (int q = 0; q < C_::NPAIRS; ++q) {
                const int pa = KIND == 0 ? kPairsBF16[q][0] : kPairs2[q][0];
                const int pb = KIND == 0 ? kPairsBF16[q][1] : kPairs2[q][1];
#pragma unroll
                for (int j = 0; j < C_::KSTEPS; ++j) {  // MMAs of 32 bytes of K per swizzle row
                    const uint64_t ad = smem_desc<ROWB>(sa + pa * PART_TILE_BYTES + j * 32);
                    const uint64_t bd = smem_desc<ROWB>(sb + pb * PART_TILE_BYTES + j * 32);
                    mma<KIND>(d, ad, bd, idesc, (kbi > 0 || q > 0 || j > 0) ? 1u : 0u);
                }
            }
            any = true;
            mma_commit(smem_u32(&empty_bar[s]));
            if (kbi == kpc - 1) mma_commit(smem_u32(&tfull[t]));
        }
        if (*abort_flag && any) {
            mma_commit(smem_u32(&drain_bar));
            for (uint32_t i = 0; i < spin && !mbar_try(smem_u32(&drain_bar), 0); ++i) {
            }
        }
    } else if (warp < EPI_WARPS) {
        // ---------------- epilogue: chunk partials TMEM -> FP32 registers -> C
        const int g = warp & 3, h = warp >> 2;
        float cr[64], ci[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) {
            cr[j] = 0.f;
            ci[j] = 0.f;
        }
        bool ok = true;
        for (int c = 0; c < nchunks && ok; ++c) {
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                int w = 0;
                if (lane == 0) w = mbar_wait(smem_u32(&tfull[t]), (uint32_t)c & 1u, abort_flag, spin) ? 1 : 0;
                w = __shfl_sync(0xffffffffu, w, 0);
                if (!w) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * g) << 16) + (uint32_t)(t * TN + 64 * h + 32 * half), v);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = 32 * half + j;
                        if (t == 0) {
                            cr[col] += v[j];
                            ci[col] -= v[j];
                        } else if (t == 1) {
                            cr[col] -= v[j];
                            ci[col] -= v[j];
                        } else {
                            ci[col] += v[j];
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&tfree[t]));
            }
        }
        if (!ok) {
            if (lane == 0 && !abort_sh) {
                abort_sh = 1;
                atomicExch(p.err, kErrTimeout);
            }
        } else {
            if constexpr (KIND == 3) {  // undo the operand scales 2^eA 2^eB (exact)
                const float sa = pow2f(-fp16_scale_exp(p.amax_a[p.a_shared ? 0 : z])),
                            sb = pow2f(-fp16_scale_exp(p.amax_b[p.b_shared ? 0 : z]));
#pragma unroll
                for (int j = 0; j < 64; ++j) {
                    cr[j] = cr[j] * sa * sb;
                    ci[j] = ci[j] * sa * sb;
                }
            }
            // Stage the warp's 32 x 64 complex block in shared memory (every MMA that
            // read the pipeline ring has completed), then write whole 512-byte rows
            // with coalesced 16-byte stores.
            float2* stg = reinterpret_cast<float2*>(smem) + (size_t)warp * 32 * EPI_LDW;
#pragma unroll
            for (int j = 0; j < 64; j += 2)
                reinterpret_cast<float4*>(stg + lane * EPI_LDW + j)[0] = make_float4(cr[j], ci[j], cr[j + 1], ci[j + 1]);
            __syncwarp();
            const int64_t ld = p.ksplit_bits ? N : (p.c_ld ? p.c_ld : N);
            float2* cb = p.ksplit_bits
                             ? p.partial + ((int64_t)blockIdx.y * gridDim.z + z) * ((int64_t)N << p.mb)
                             : p.C + (int64_t)z * p.c_batch_stride;
            float2* cbase = cb + (int64_t)(m0 + 32 * g) * ld + n0 + 64 * h;
            if (p.accumulate) {
#pragma unroll 4
                for (int r = 0; r < 32; ++r) {
                    float4* dst = reinterpret_cast<float4*>(cbase + (int64_t)r * ld) + lane;
                    const float4 v = reinterpret_cast<const float4*>(stg + r * EPI_LDW)[lane];
                    const float4 o = *dst;
                    *dst = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
                }
            } else {
#pragma unroll 4
                for (int r = 0; r < 32; ++r)
                    reinterpret_cast<float4*>(cbase + (int64_t)r * ld)[lane] =
                        reinterpret_cast<const float4*>(stg + r * EPI_LDW)[lane];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    __syncthreads();
    if (warp == MMA_WARP) {
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
    }
}

// ------------------------------------------------------------ operand split

__device__ __forceinline__ int64_t slice_offset(const Operand& op, int64_t s) {
    int64_t off = 0;
    for (int j = 0; j < op.n_sl; ++j) off += ((s >> op.sl_bit[j]) & 1) * op.sl_stride[j];
    return off;
}

__device__ __forceinline__ int64_t bits_offset(int64_t x, const int64_t* str, int nbits, int from) {
    int64_t off = 0;
    for (int j = from; j < nbits; ++j)
        if ((x >> j) & 1) off += str[j];
    return off;
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

constexpr int SPLIT_TILE = 2048;  // elements per split tile: SR rows x SK k
// SK: 256 k when k is the operand's unit-stride mode (reads of 2 KB and plane
// writes of 512 B per row), else 64 (32 when K = 32) so that a gather whose
// unit stride lies along the rows stays coalesced too.
__host__ __device__ inline int split_tile_k(int kb, bool kfast) {
    const int K = 1 << (kb < 9 ? kb : 9);
    return kfast ? (K < 256 ? K : 256) : (K < 64 ? K : 64);
}
// shared-memory slot of tile element (rr, kk): one padding slot every 8 k keeps
// the write phase's 8-wide groups on distinct banks
constexpr int SPLIT_SMEM = 2368;  // >= SR * (SK + SK / 8 + 1) for every SK above

// planes: out[((z * (3*PARTS) + q) * R + r) * K + k], q = t * PARTS + part
template <int KIND>
__global__ void __launch_bounds__(256) k_split_operand(const __grid_constant__ SplitParams p) {
    using C_ = Cfg<KIND, 64>;
    __shared__ float2 tile[SPLIT_SMEM];
    __shared__ int64_t roff[64], koff[256];
    const int64_t R = 1ll << p.rb, K = 1ll << p.kb;
    const bool kfast = p.kb > 0 && p.ks[0] == 1;
    const int SK = split_tile_k(p.kb, kfast);
    const int SR = SPLIT_TILE / SK;
    const int LD = SK + SK / 8 + 1;
    const int64_t tiles_k = K / SK;
    const int64_t r0 = (blockIdx.x / tiles_k) * SR, k0 = (blockIdx.x % tiles_k) * SK;
    const int z = blockIdx.z;
    const float2* src = p.src.ptr + z * p.src.batch_stride + slice_offset(p.src, p.slice0 + z);
    const int tid = threadIdx.x;
    if (tid < SR) roff[tid] = bits_offset(r0 + tid, p.rs, p.rb, 0);
    if (tid < SK) koff[tid] = bits_offset(k0 + tid, p.ks, p.kb, 0);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SPLIT_TILE / 256; ++i) {
        int e = tid + i * 256;
        int rr, kk;
        if (kfast) { kk = e % SK; rr = e / SK; }
        else { rr = e % SR; kk = e / SR; }
        tile[rr * LD + kk + (kk >> 3)] = src[roff[rr] + koff[kk]];
    }
    __syncthreads();
    constexpr int Q = 3 * C_::PARTS;
    const int64_t plane = R * K;
    uint8_t* out = reinterpret_cast<uint8_t*>(p.dst) + (int64_t)z * Q * plane * C_::ELEM;
    // one thread per 8 consecutive k of one row (SR rows x SK/8 groups = 256):
    // every part of every real matrix leaves as one 16-byte (TF32: 32-byte) store
    const int gpr = SK / 8;
    const int rr = tid / gpr, g8 = tid % gpr;
    float v[3][8];
    const float sc = KIND == 3 ? pow2f(fp16_scale_exp(p.amax[z])) : 1.f;  // FP16x2 operand scale (exact)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float2 x = tile[rr * LD + 9 * g8 + j];  // element (rr, 8 g8 + j)
        if constexpr (KIND == 3) {
            x.x *= sc;
            x.y *= sc;
        }
        v[0][j] = x.x;
        v[1][j] = x.y;
        v[2][j] = x.x + x.y;
    }
    const int64_t idx = (r0 + rr) * K + k0 + 8 * g8;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
#pragma unroll
        for (int q = 0; q < C_::PARTS; ++q) {
            if constexpr (KIND == 1) {
                float hi[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    hi[j] = tf32_round(v[t][j]);
                    v[t][j] -= hi[j];
                }
                float4* dst = reinterpret_cast<float4*>(out + ((t * 2 + q) * plane + idx) * 4);
                dst[0] = make_float4(hi[0], hi[1], hi[2], hi[3]);
                dst[1] = make_float4(hi[4], hi[5], hi[6], hi[7]);
            } else {
                uint32_t w[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if constexpr (KIND == 3) {
                        const __half2 h = __floats2half2_rn(v[t][2 * j], v[t][2 * j + 1]);
                        v[t][2 * j] -= __low2float(h);
                        v[t][2 * j + 1] -= __high2float(h);
                        w[j] = *reinterpret_cast<const uint32_t*>(&h);
                    } else {
                        const __nv_bfloat162 h = __floats2bfloat162_rn(v[t][2 * j], v[t][2 * j + 1]);
                        v[t][2 * j] -= __low2float(h);
                        v[t][2 * j + 1] -= __high2float(h);
                        w[j] = *reinterpret_cast<const uint32_t*>(&h);
                    }
                }
                reinterpret_cast<uint4*>(out + ((t * C_::PARTS + q) * plane + idx) * 2)[0] =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
}

// Split FP16x2: max of |Re| and |Im| over the whole tensor behind an operand,
// per batch entry, as float bits (non-negative floats order like their bits).
// An operand covers every element of its tensor (free, contracted and sliced
// binary modes together), so the max is order-free and a linear scan; for a
// slice or a row panel of the tensor it is an upper bound, which is all the
// scale needs. One atomic per block; amax must be zeroed first.
constexpr int ABSMAX_BLOCKS = 152 * 4;

__global__ void __launch_bounds__(256) k_absmax(const float2* __restrict__ base, int64_t batch_stride, int64_t n,
                                                uint32_t* amax) {
    __shared__ uint32_t wmax[8];
    const int z = blockIdx.z;
    const float2* src = base + (int64_t)z * batch_stride;
    uint32_t m = 0;
    const int64_t step = (int64_t)gridDim.x * 256;
    int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    for (; i + 3 * step < n; i += 4 * step) {  // four loads in flight per thread
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = src[i + u * step];
#pragma unroll
        for (int u = 0; u < 4; ++u) m = max(m, max(__float_as_uint(fabsf(v[u].x)), __float_as_uint(fabsf(v[u].y))));
    }
    for (; i < n; i += step) {
        const float2 v = src[i];
        m = max(m, max(__float_as_uint(fabsf(v.x)), __float_as_uint(fabsf(v.y))));
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < 8 ? wmax[threadIdx.x] : 0u;
        m = __reduce_max_sync(0xffffffffu, m);
        if (threadIdx.x == 0) atomicMax(amax + z, m);
    }
}

// ------------------------------------------------------------ K-split reduction
// C[z][m][n] (+)= sum over splits, in order, of partial[split][z][m][n]: FP64
// sums rounded once, two complex elements per thread step.
__global__ void __launch_bounds__(256) k_ksplit_reduce(const float4* __restrict__ partial, int nsplit, int batch,
                                                       int64_t mn2, int nb, float2* C, int64_t c_batch_stride,
                                                       int64_t c_ld, int accumulate) {
    const int z = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < mn2; i += (int64_t)gridDim.x * 256) {
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        for (int sp = 0; sp < nsplit; ++sp) {
            const float4 v = partial[((int64_t)sp * batch + z) * mn2 + i];
            a0 += v.x;
            a1 += v.y;
            a2 += v.z;
            a3 += v.w;
        }
        const int64_t e = 2 * i;  // first of the two complex elements
        const int64_t m = e >> nb, n = e & ((1ll << nb) - 1);
        float4* dst = reinterpret_cast<float4*>(C + (int64_t)z * c_batch_stride + m * c_ld + n);
        float4 r = make_float4((float)a0, (float)a1, (float)a2, (float)a3);
        if (accumulate) {
            const float4 o = *dst;
            r = make_float4(o.x + r.x, o.y + r.y, o.z + r.z, o.w + r.w);
        }
        *dst = r;
    }
}

// ------------------------------------------------------------ host helpers

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
    static EncodeFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    }
    return fn;
}

// 4D map over planes [batch][3*PARTS][rows][K]; box = (BK, box_rows, PARTS, 1).
template <int KIND, int ROWB>
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t K, int batch, int box_rows = 128,
              int box_parts = Cfg<KIND, ROWB>::PARTS) {
    using C_ = Cfg<KIND, ROWB>;
    EncodeFn enc = encoder();
    if (!enc) return false;
    const int Q = 3 * C_::PARTS;
    cuuint64_t dims[4] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)Q, (cuuint64_t)batch};
    cuuint64_t strides[3] = {(cuuint64_t)(K * C_::ELEM), (cuuint64_t)(rows * K * C_::ELEM),
                             (cuuint64_t)(Q * rows * K * C_::ELEM)};
    cuuint32_t box[4] = {(cuuint32_t)C_::BK, (cuuint32_t)box_rows, (cuuint32_t)box_parts, 1u};  // BK * ELEM = ROWB bytes
    cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = KIND == 1   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : KIND == 3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                               : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = enc(map, dt, 4,
                     const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     ROWB == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int KIND, int ROWB>
cudaError_t launch_tc_impl(const TcGemmParams& p, const void* planesA, const void* planesB, int batch,
                           cudaStream_t s) {
    using C_ = Cfg<KIND, ROWB>;
    const int64_t M = 1ll << p.mb, N = 1ll << p.nb, K = 1ll << p.kb;
    if (K % C_::BK || N % TN) return cudaErrorInvalidValue;
    CUtensorMap ta, tb;
    if (!make_map<KIND, ROWB>(&ta, planesA, M, K, batch) || !make_map<KIND, ROWB>(&tb, planesB, N, K, batch))
        return cudaErrorInvalidValue;
    const int smem = C_::STAGES * C_::STAGE_BYTES + 1024;
    static_assert(C_::STAGES >= 2 && C_::STAGES * C_::STAGE_BYTES + 1024 <= 227 * 1024, "shared memory");
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_cgemm_tc<KIND, ROWB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int64_t tiles = (M / TM) * (N / TN);
    if ((K >> p.ksplit_bits) < C_::BK || (p.ksplit_bits && (!p.partial || p.accumulate))) return cudaErrorInvalidValue;
    k_cgemm_tc<KIND, ROWB><<<dim3((unsigned)tiles, 1u << p.ksplit_bits, batch), NTHREADS, smem, s>>>(ta, tb, p);
    return cudaGetLastError();
}

template <int KIND>
cudaError_t launch_tc_rows(const TcGemmParams& p, const void* pa, const void* pb, int batch, cudaStream_t s) {
    // 128-byte rows need K to span whole 128-byte k-blocks
    const int64_t K = 1ll << p.kb;
    if (p.row_bytes == 128 && K % Cfg<KIND, 128>::BK == 0) return launch_tc_impl<KIND, 128>(p, pa, pb, batch, s);
    return launch_tc_impl<KIND, 64>(p, pa, pb, batch, s);
}

}  // namespace

// tnc_mode -> kernel configuration: 1 TF32 (2 parts), 2 BF16 (3 parts), 3 BF16 (2 parts),
// 4 scaled FP16 (2 parts)
static int kind_of(int mode) { return mode == 1 ? 1 : (mode == 2 ? 0 : (mode == 4 ? 3 : 2)); }

int tc_plane_count(int mode) { return mode == 2 ? 9 : 6; }
int tc_elem_bytes(int mode) { return mode == 1 ? 4 : 2; }
int tc_min_kb(int) { return 5; }

cudaError_t launch_split(const SplitParams& p, int mode, int batch, cudaStream_t s) {
    const int64_t R = 1ll << p.rb, K = 1ll << p.kb;
    if (K < 32 || batch < 1 || batch > 65535) return cudaErrorInvalidConfiguration;
    const int64_t SK = split_tile_k(p.kb, p.kb > 0 && p.ks[0] == 1), SR = SPLIT_TILE / SK;
    if (R < SR) return cudaErrorInvalidConfiguration;
    const int64_t blocks = (R / SR) * (K / SK);
    const dim3 grid((unsigned)blocks, 1, batch);
    switch (kind_of(mode)) {
        case 0: k_split_operand<0><<<grid, 256, 0, s>>>(p); break;
        case 1: k_split_operand<1><<<grid, 256, 0, s>>>(p); break;
        case 3:
            if (!p.amax) return cudaErrorInvalidValue;  // launch_absmax ran before
            k_split_operand<3><<<grid, 256, 0, s>>>(p);
            break;
        default: k_split_operand<2><<<grid, 256, 0, s>>>(p); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_ksplit_reduce(const float2* partial, int ksplit_bits, int batch, int mb, int nb, float2* C,
                                 int64_t c_batch_stride, int64_t c_ld, int accumulate, cudaStream_t s) {
    if (!partial || !C || ksplit_bits < 1 || batch < 1 || batch > 65535 || nb < 1) return cudaErrorInvalidValue;
    const int64_t mn2 = (1ll << (mb + nb)) / 2;  // float4 steps of two complex elements
    const int64_t want = (mn2 + 255) / 256;
    const unsigned blocks = (unsigned)(want < 152 * 16 ? want : 152 * 16);
    k_ksplit_reduce<<<dim3(blocks, batch), 256, 0, s>>>(reinterpret_cast<const float4*>(partial), 1 << ksplit_bits,
                                                        batch, mn2, nb, C, c_batch_stride, c_ld, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_absmax(const Operand& src, int bits, int batch, uint32_t* amax, cudaStream_t s) {
    if (!amax || bits < 0 || bits > 40 || batch < 1 || batch > 65535) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(uint32_t) * (size_t)batch, s);
    if (e != cudaSuccess) return e;
    const int64_t n = 1ll << bits;
    const int64_t want = (n + 2047) / 2048;
    const unsigned blocks = (unsigned)(want < ABSMAX_BLOCKS ? (want < 1 ? 1 : want) : ABSMAX_BLOCKS);
    k_absmax<<<dim3(blocks, 1, batch), 256, 0, s>>>(src.ptr, src.batch_stride, n, amax);
    return cudaGetLastError();
}

cudaError_t launch_cgemm_tc(const TcGemmParams& p, int mode, const void* planesA, const void* planesB,
                            int batch, cudaStream_t s) {
    if (p.mb < 7 || p.nb < 7 || p.kb < tc_min_kb(mode) || batch < 1 || batch > 65535)
        return cudaErrorInvalidConfiguration;
    switch (kind_of(mode)) {
        case 0: return launch_tc_rows<0>(p, planesA, planesB, batch, s);
        case 1: return launch_tc_rows<1>(p, planesA, planesB, batch, s);
        case 3:
            if (!p.amax_a || !p.amax_b) return cudaErrorInvalidValue;
            return launch_tc_rows<3>(p, planesA, planesB, batch, s);
        default: return launch_tc_rows<2>(p, planesA, planesB, batch, s);
    }
}

}  // namespace tnc
