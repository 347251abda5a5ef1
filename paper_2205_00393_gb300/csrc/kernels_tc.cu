// Split-precision complex GEMM on the 5th-generation tensor cores (tcgen05).
//
// A pairwise contraction C[m,n] = sum_k A(m,k) B(k,n) (Sec. 2.1.1, in the
// TTGT arrangement of Sec. 5.3.1) runs in two kernels:
//
//  1. k_split_operand: the permute-fused operand load. It gathers the FP32
//     complex operand through its per-bit stride table (the permutation and
//     the slice fixing), stages a tile of whole 256-wide K chunks in shared
//     memory so that both the gather and the writes are coalesced, and
//     writes the real and the imaginary part as split parts in K-major
//     planes:  BF16: x = x0 + x1 + x2 (three parts); TF32 and BF16x2:
//     x = x0 + x1; FP16x2: the row's chunk is first scaled by a power of
//     two (below), then x = x0 + x1 in FP16.
//  2. k_cgemm_tc: a warp-specialised tcgen05 GEMM on 128x128 complex output
//     tiles. One warp issues TMA loads (one box per operand and stage: every
//     part of Re and Im) into a shared-memory ring guarded by mbarriers; one
//     thread issues tcgen05.mma (kind::f16 or kind::tf32, FP32 accumulation)
//     for every part pair (i, j) with i + j <= 2 (three parts) or i + j <= 1
//     (two parts), four real products each:
//         Cr += Ar Br,  Cr += (-Ai) Bi  (the MMA's negate-A bit),
//         Ci += Ar Bi,  Ci += Ai Br,
//     so the complex tile lives in 256 TMEM columns and two such buffers
//     alternate per 128-wide K chunk; eight epilogue warps move each chunk's
//     Cr, Ci into FP32 registers while the tensor cores fill the other
//     buffer, and finally write C.
//
// Split FP16x2 scaling: every row of A and every column of B is scaled by its
// own power of two per 256-wide K chunk (the largest |Re|, |Im| of that row
// chunk lands in [2^14, 2^15)). Within a chunk the scales of row m and
// column n multiply every product of C[m,n]'s chunk sum by the same 2^(eA+eB),
// so the epilogue undoes them exactly when it moves the chunk out of TMEM.
//
// Every mbarrier wait is bounded; a wait that gives up records an error code
// in the caller's error word, the CTA drains its own copies in flight, frees
// its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>

#include "f32_device.cuh"
#include "kernels.h"

namespace tnc {

namespace {

constexpr int TM = 128, TN = 128;                 // complex output tile
constexpr int SMEM_PIPE = 192 * 1024;             // shared memory for the TMA ring
constexpr uint32_t kSpinLimit = 1u << 24;
constexpr int kErrTimeout = 4;
constexpr int KC_ELEMS = 256;                     // K per FP16x2 scale chunk (whole chunks per CTA)
constexpr int KD_ELEMS = 128;                     // K per TMEM accumulation (drained into registers)

// KIND 0: three BF16 parts (6 pairs), kind::f16; 1: two TF32 parts (3 pairs),
// kind::tf32; 2: two BF16 parts (3 pairs), kind::f16; 3: two FP16 parts of
// the scaled operand (3 pairs), kind::f16. ROWB: bytes of K per tile row and
// k-block, which is also the swizzle width (32 or 64).
template <int KIND, int ROWB> struct Cfg {
    static constexpr int PARTS = KIND == 0 ? 3 : 2;
    static constexpr int NPAIRS = KIND == 0 ? 6 : 3;
    static constexpr int PLANES = 2 * PARTS;                   // Re parts, then Im parts
    static constexpr int ELEM = KIND == 1 ? 4 : 2;
    static constexpr int BK = ROWB / ELEM;                     // K elements per k-block
    static constexpr int PART_TILE = 128 * ROWB;               // bytes of one part tile (128 rows)
    static constexpr int OP_BYTES = PLANES * PART_TILE;        // one operand's share of a stage
    static constexpr int STAGE_BYTES = 2 * OP_BYTES;
    static constexpr int STAGES = SMEM_PIPE / STAGE_BYTES > 8 ? 8 : SMEM_PIPE / STAGE_BYTES;
    static constexpr int KSTEPS = ROWB / 32;                   // MMAs per k-block (32 bytes of K each)
};

// Split FP16x2 scale exponent of a row chunk whose largest |Re|, |Im| has the
// float bits amax_bits: 2^e puts that maximum in [2^14, 2^15), below the FP16
// maximum 65504. x0 = fp16(x) and x1 = fp16(x - x0) then carry 22 significant
// bits for every element within 2^16 of the chunk maximum (x1 is a normal
// FP16 there); smaller elements keep an absolute error below 2^-39 of it.
// e is clamped to [-126, 126] so that 2^e and 2^-e are normal floats.
__host__ __device__ __forceinline__ int fp16_scale_exp(uint32_t amax_bits) {
    if (amax_bits == 0) return 0;
    const int e = 141 - (int)((amax_bits >> 23) & 0xFFu);
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

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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
// 4 = 64B, 6 = 32B), 8-row groups 8*ROWB bytes apart, descriptor version 1.
template <int ROWB>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)((8 * ROWB) >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;                    // version
    d |= (uint64_t)(ROWB == 64 ? 4 : 6) << 61;
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

// 16 consecutive 32-bit TMEM columns of this warp's 32 lanes (one per lane)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Instruction descriptor: FP32 accumulator (bit 4), A/B format at bits 7 and
// 10 (kind::f16: 0 = F16, 1 = BF16; kind::tf32: 2 = TF32), negate A at bit
// 13, both operands K-major, N >> 3 at bit 17, M >> 4 at bit 24.
template <int KIND>
__host__ __device__ constexpr uint32_t ab_format() {
    return KIND == 1 ? 2u : (KIND == 3 ? 0u : 1u);
}

template <int KIND>
__host__ __device__ constexpr uint32_t instr_desc(bool negate_a) {
    return (1u << 4) | (ab_format<KIND>() << 7) | (ab_format<KIND>() << 10) | (negate_a ? (1u << 13) : 0u) |
           ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// Part pairs, smallest magnitudes first.
__constant__ int kPairsBF16[6][2] = {{1, 1}, {0, 2}, {2, 0}, {0, 1}, {1, 0}, {0, 0}};
__constant__ int kPairs2[3][2] = {{0, 1}, {1, 0}, {0, 0}};

// K is processed in chunks of KD_ELEMS. Each chunk accumulates in one of two
// TMEM buffers of 256 columns (Cr in the first 128, Ci in the last 128); when
// a chunk is complete the epilogue warps move it into FP32 registers while
// the tensor cores work on the next chunk in the other buffer. The tensor
// core's accumulation into TMEM does not round to nearest, so its error grows
// linearly with the number of accumulated MMAs: with four real products per
// complex product, every accumulator element takes 2 x (part pairs) MMAs per
// 16 (TF32: 8) of K, so short chunks bound that growth, and the register sums
// across chunks round to nearest. One FP16x2 scale chunk (KC_ELEMS of K)
// spans two accumulation chunks.
constexpr int EPI_WARPS = 8;   // warps 0-7: epilogue (warp w: TMEM lanes 32*(w%4), columns 64*(w/4))
constexpr int EPI_LDW = 66;    // float2 per row of a warp's staged 32 x 64 output block (2 of padding)
static_assert(EPI_WARPS * 32 * EPI_LDW * 8 <= SMEM_PIPE, "staged epilogue fits the pipeline ring");
constexpr int PRODUCER_WARP = 8, MMA_WARP = 9, NTHREADS = 320;

// Shared-memory state of one CTA's tensor-core pipeline.
struct TcShared {
    uint64_t full_bar[8], empty_bar[8], tfull[2], tfree[2], drain_bar;
    uint32_t tmem_base;
    int abort;
    float colscale[EPI_WARPS][64];  // split FP16x2: per-warp column factors of a chunk
};

// k-blocks and TMEM chunks a CTA's tensor-core roles have processed so far:
// the barrier phases of the pipeline continue from one output tile to the
// next when a CTA computes several (the persistent executor).
struct TcPipe {
    uint32_t it = 0, ch = 0;
};

// thread 0, before the CTA-wide barrier that precedes the first tile
__device__ __forceinline__ void tc_init(TcShared& sh) {
    for (int s = 0; s < 8; ++s) {
        mbar_init(smem_u32(&sh.full_bar[s]), 1);
        mbar_init(smem_u32(&sh.empty_bar[s]), 1);
    }
    for (int t = 0; t < 2; ++t) {
        mbar_init(smem_u32(&sh.tfull[t]), 1);
        mbar_init(smem_u32(&sh.tfree[t]), EPI_WARPS);
    }
    mbar_init(smem_u32(&sh.drain_bar), 1);
    sh.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One 128x128 complex output tile of the contraction p: tile index `cta` in
// grouped rasterisation order, K split ky, batch entry z of nbatch. Run by all
// NTHREADS threads (warps 0-7 epilogue, warp 8 TMA producer, warp 9 MMA
// issuer); smem is the TMA ring (also the epilogue's staging area), tmem the
// CTA's 512 TMEM columns. On a bounded wait that gives up, sh.abort and
// *p.err are set and the roles stop (MMAs and loads in flight drained).
template <int KIND, int ROWB, bool GLOBAL_MAPS = false>
__device__ __forceinline__ void tc_tile(const CUtensorMap* tmA, const CUtensorMap* tmB, const TcGemmParams& p,
                                        int64_t cta, int ky, int z, int nbatch, uint8_t* smem, TcShared& sh,
                                        uint32_t tmem, TcPipe& pipe) {
    using C_ = Cfg<KIND, ROWB>;
    constexpr int PT = C_::PART_TILE;
    const int GROUP_M = p.group_m < 1 ? 1 : p.group_m;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t M = 1ll << p.mb, N = 1ll << p.nb, K = 1ll << p.kb;
    // grouped rasterisation: consecutive tiles cover GROUP_M row tiles x all column tiles
    const int64_t tiles_n = N / TN, tiles_m = M / TM;
    const int64_t per_group = (int64_t)GROUP_M * tiles_n;
    const int64_t grp = cta / per_group, in_grp = cta % per_group;
    const int64_t gm = (tiles_m - grp * GROUP_M) < GROUP_M ? (tiles_m - grp * GROUP_M) : GROUP_M;
    const int m0 = (int)((grp * GROUP_M + in_grp % gm) * TM);
    const int n0 = (int)((in_grp / gm) * TN);
    const int za = p.a_shared ? 0 : z, zb = p.b_shared ? 0 : z;  // batch entry of each operand's planes
    const int nkb = (int)((K >> p.ksplit_bits) / C_::BK);         // k-blocks of this K split
    const int kb_off = ky * nkb;
    const int kpc = nkb < KD_ELEMS / C_::BK ? nkb : KD_ELEMS / C_::BK;  // k-blocks per chunk
    const int nchunks = nkb / kpc;
    volatile int* abort_flag = &sh.abort;
    const uint32_t spin = p.spin_limit ? p.spin_limit : kSpinLimit;

    if (warp == PRODUCER_WARP && lane == 0) {
        // ---------------- TMA producer: one stage per k-block, every plane of A and of B
        asm volatile("fence.proxy.async.global;" ::: "memory");  // planes written by generic stores
        if constexpr (GLOBAL_MAPS) {  // tensor maps in global memory: acquire them for the tensormap proxy
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmA) : "memory");
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmB) : "memory");
        }
        int issued = 0;
        for (int it = 0; it < nkb && !p.test_stall; ++it) {
            const uint32_t g = pipe.it + it;
            const int s = g % C_::STAGES;
            const uint32_t ph = (g / C_::STAGES) & 1u;
            if (!mbar_wait(smem_u32(&sh.empty_bar[s]), ph ^ 1u, abort_flag, spin)) {
                sh.abort = 1;
                atomicExch(p.err, kErrTimeout);
                break;
            }
            const uint32_t sa = smem_u32(smem + s * C_::STAGE_BYTES);
            const uint32_t fb = smem_u32(&sh.full_bar[s]);
            mbar_expect_tx(fb, C_::STAGE_BYTES);
            tma_load_4d(sa, tmA, (it + kb_off) * C_::BK, m0, 0, za, fb);
            tma_load_4d(sa + C_::OP_BYTES, tmB, (it + kb_off) * C_::BK, n0, 0, zb, fb);
            issued = it + 1;
        }
        if (*abort_flag) {
            // drain: wait (bounded) for every load that may still be in flight
            int first = issued - C_::STAGES < 0 ? 0 : issued - C_::STAGES;
            for (int it = first; it < issued; ++it) {
                const uint32_t g = pipe.it + it;
                const int s = g % C_::STAGES;
                const uint32_t ph = (g / C_::STAGES) & 1u;
                for (uint32_t i = 0; i < spin && !mbar_try(smem_u32(&sh.full_bar[s]), ph); ++i) {
                }
            }
        }
    } else if (warp == MMA_WARP && lane == 0) {
        // ---------------- MMA issuer
        constexpr uint32_t idesc = instr_desc<KIND>(false), idesc_neg = instr_desc<KIND>(true);
        bool any = false;
        for (int it = 0; it < nkb && !*abort_flag; ++it) {
            const uint32_t g = pipe.it + it;
            const int s = g % C_::STAGES;
            const uint32_t ph = (g / C_::STAGES) & 1u;
            const int kbi = it % kpc;
            const uint32_t cgl = pipe.ch + it / kpc;  // chunk over all tiles of this CTA
            const int buf = cgl & 1;
            if ((kbi == 0 && cgl >= 2 &&
                 !mbar_wait(smem_u32(&sh.tfree[buf]), ((cgl - 2) >> 1) & 1u, abort_flag, spin)) ||
                !mbar_wait(smem_u32(&sh.full_bar[s]), ph, abort_flag, spin)) {
                sh.abort = 1;
                atomicExch(p.err, kErrTimeout);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = smem_u32(smem + s * C_::STAGE_BYTES);
            const uint32_t sb = sa + C_::OP_BYTES;
            const uint32_t dr = tmem + (uint32_t)(buf * 2 * TN), di = dr + TN;
#pragma unroll
            for (int q = 0; q < C_::NPAIRS; ++q) {
                const int pa = KIND == 0 ? kPairsBF16[q][0] : kPairs2[q][0];
                const int pb = KIND == 0 ? kPairsBF16[q][1] : kPairs2[q][1];
#pragma unroll
                for (int j = 0; j < C_::KSTEPS; ++j) {  // MMAs of 32 bytes of K per swizzle row
                    const uint64_t ar = smem_desc<ROWB>(sa + pa * PT + j * 32);
                    const uint64_t ai = smem_desc<ROWB>(sa + (C_::PARTS + pa) * PT + j * 32);
                    const uint64_t br = smem_desc<ROWB>(sb + pb * PT + j * 32);
                    const uint64_t bi = smem_desc<ROWB>(sb + (C_::PARTS + pb) * PT + j * 32);
                    const uint32_t acc = (kbi > 0 || q > 0 || j > 0) ? 1u : 0u;
                    mma<KIND>(dr, ar, br, idesc, acc);
                    mma<KIND>(dr, ai, bi, idesc_neg, 1u);
                    mma<KIND>(di, ar, bi, idesc, acc);
                    mma<KIND>(di, ai, br, idesc, 1u);
                }
            }
            any = true;
            mma_commit(smem_u32(&sh.empty_bar[s]));
            if (kbi == kpc - 1) mma_commit(smem_u32(&sh.tfull[buf]));
        }
        if (*abort_flag && any) {
            mma_commit(smem_u32(&sh.drain_bar));
            for (uint32_t i = 0; i < spin && !mbar_try(smem_u32(&sh.drain_bar), 0); ++i) {
            }
        }
    } else if (warp < EPI_WARPS) {
        // ---------------- epilogue: chunk sums TMEM -> FP32 registers -> C
        const int g = warp & 3, h = warp >> 2;
        float cr[64], ci[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) {
            cr[j] = 0.f;
            ci[j] = 0.f;
        }
        // split FP16x2: per-chunk scale exponents of this lane's row and of the warp's 64 columns;
        // the columns' factors 2^-e go through a warp-private table in shared memory
        const int64_t sk = K < KC_ELEMS ? K : KC_ELEMS;  // K per scale chunk
        const int64_t nch = K / sk;                       // scale chunks over the whole K of the planes
        const int8_t* ea_row = nullptr;
        const int8_t* eb_col = nullptr;
        if constexpr (KIND == 3) {
            ea_row = p.sexp_a + (int64_t)za * nch * M + m0 + 32 * g + lane;
            eb_col = p.sexp_b + (int64_t)zb * nch * N + n0 + 64 * h;
        }
        float* colf = sh.colscale[warp];
        bool ok = true;
        for (int c = 0; c < nchunks && ok; ++c) {
            const uint32_t cgl = pipe.ch + c;
            const int buf = cgl & 1;
            int w = 0;
            if (lane == 0) w = mbar_wait(smem_u32(&sh.tfull[buf]), (cgl >> 1) & 1u, abort_flag, spin) ? 1 : 0;
            w = __shfl_sync(0xffffffffu, w, 0);
            if (!w) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // scale chunk of this TMEM chunk (chunk index over the planes' K x its K / scale chunk's K)
            const int64_t cg = ((int64_t)ky * nchunks + c) * (kpc * C_::BK) / sk;
            float sa = 1.f;
            if constexpr (KIND == 3) {
                sa = pow2f(-(int)ea_row[cg * M]);
                const char2 e2 = reinterpret_cast<const char2*>(eb_col + cg * N)[lane];
                colf[2 * lane] = pow2f(-(int)e2.x);
                colf[2 * lane + 1] = pow2f(-(int)e2.y);
                __syncwarp();
            }
            const uint32_t tbase = tmem + ((uint32_t)(32 * g) << 16) + (uint32_t)(buf * 2 * TN + 64 * h);
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {                // 16 columns at a time
#pragma unroll
                for (int part = 0; part < 2; ++part) {      // 0: Cr columns, 1: Ci columns
                    float v[16];
                    tmem_ld16(tbase + (uint32_t)(part * TN + 16 * q4), v);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        float x = v[j];
                        if constexpr (KIND == 3) x = x * sa * colf[16 * q4 + j];
                        if (part == 0) cr[16 * q4 + j] += x;
                        else ci[16 * q4 + j] += x;
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&sh.tfree[buf]));
        }
        if (!ok) {
            if (lane == 0 && !sh.abort) {
                sh.abort = 1;
                atomicExch(p.err, kErrTimeout);
            }
        } else {
            // Stage the warp's 32 x 64 complex block in shared memory (every MMA that
            // read the pipeline ring has completed), then write whole 512-byte rows
            // with coalesced 16-byte stores.
            float2* stg = reinterpret_cast<float2*>(smem) + (size_t)warp * 32 * EPI_LDW;
#pragma unroll
            for (int j = 0; j < 64; j += 2)
                reinterpret_cast<float4*>(stg + lane * EPI_LDW + j)[0] = make_float4(cr[j], ci[j], cr[j + 1], ci[j + 1]);
            __syncwarp();
            const int64_t ld = p.ksplit_bits ? N : (p.c_ld ? p.c_ld : N);
            float2* cb = p.ksplit_bits ? p.partial + ((int64_t)ky * nbatch + z) * (N << p.mb)
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
    pipe.it += nkb;
    pipe.ch += nchunks;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
}

template <int KIND, int ROWB>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_cgemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ TcGemmParams p) {
    extern __shared__ __align__(1024) uint8_t dsmem[];
    __shared__ TcShared sh;
    const int warp = threadIdx.x >> 5;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~uintptr_t(1023));
    if (threadIdx.x == 0) tc_init(sh);
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sh.tmem_base;
    TcPipe pipe;
    tc_tile<KIND, ROWB>(&tmA, &tmB, p, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.z, smem, sh, tmem, pipe);
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

// A split tile covers SR rows x SK k with SK = min(K, 256): whole K chunks,
// so each row's FP16x2 scale is decided inside one CTA. SR * SK is 2048 when
// k is the operand's unit-stride mode (reads of 2 KB runs along k), else 4096
// (16 rows of 256 k: runs of 128 bytes along the rows).
__host__ __device__ inline int split_tile_k(int kb) { return 1 << (kb < 8 ? kb : 8); }
__host__ __device__ inline int split_tile_rows(int kb, bool kfast) { return (kfast ? 2048 : 4096) / split_tile_k(kb); }
// shared-memory slots per tile row: one padding slot every 8 k keeps the
// write phase's 8-wide groups on distinct banks
__host__ __device__ inline int split_ld(int sk) { return sk + sk / 8 + 1; }
// largest split tile in bytes: SR * SK = 4096 elements, one padding slot per
// 8 k and one per row (SR <= 128 rows, which K >= 32 ensures)
constexpr int kSplitTileBytesMax = (4096 + 4096 / 8 + 128) * 8;

template <int BAR>
__device__ __forceinline__ void tc_bar() {
    if constexpr (BAR == 0) __syncthreads();
    else asm volatile("bar.sync 1, 256;" ::: "memory");
}

// planes: out[((z * PLANES + q) * R + r) * K + k], q = t * PARTS + part (t = 0 Re, 1 Im);
// FP16x2 scale exponents: sexp[(z * (K / SK) + chunk) * R + r]. Split tiles
// (blocks) block0 .. block0 + count - 1 of batch entry z (slice id slice0 +
// z), run by threads 0-255; BAR as in the FP32 routines (0: whole CTA, 1:
// named barrier over 256 threads). Each block is gathered (phase 1) into
// registers, staged in a shared-memory tile (phase 2) and converted into the
// part planes (phase 3). With count > 1 the blocks are software-pipelined:
// block i + 1's gather loads are in flight while block i is converted, so
// tile[] and the offset tables roff[], koff[] are double-buffered (tile[j]:
// split_tile_floats() float2 each; roff[j]: 128, koff[j]: 256 entries).
__host__ __device__ inline int split_tile_floats(int kb, bool kfast) {
    return split_tile_rows(kb, kfast) * split_ld(split_tile_k(kb));
}

struct SplitGeom {
    int64_t R, K, tiles_k;
    int SK, SR, LD, n;
    bool kfast;
};

__device__ __forceinline__ SplitGeom split_geom(const SplitParams& p) {
    SplitGeom g;
    g.R = 1ll << p.rb;
    g.K = 1ll << p.kb;
    g.kfast = p.kb > 0 && p.ks[0] == 1;
    g.SK = split_tile_k(p.kb);
    g.SR = split_tile_rows(p.kb, g.kfast);
    g.LD = split_ld(g.SK);
    g.tiles_k = g.K / g.SK;
    g.n = g.SR * g.SK;  // 2048 (k fastest) or 4096 elements
    return g;
}

// phase 0: the block's row and k offsets through the per-bit stride tables
__device__ __forceinline__ void split_offsets(const SplitParams& p, const SplitGeom& g, int64_t block, int64_t* roff,
                                              int64_t* koff) {
    const int64_t r0 = (block / g.tiles_k) * g.SR, k0 = (block % g.tiles_k) * g.SK;
    const int tid = threadIdx.x;
    if (tid < g.SR) roff[tid] = bits_offset(r0 + tid, p.rs, p.rb, 0);
    if (tid < g.SK) koff[tid] = bits_offset(k0 + tid, p.ks, p.kb, 0);
}

// phase 1: this thread's n / 256 elements of the block, all loads in flight
// (pairs adjacent along the unit-stride mode as one 16-byte load when p.vec2)
__device__ __forceinline__ void split_gather(const SplitParams& p, const SplitGeom& g, const float2* src,
                                             const int64_t* roff, const int64_t* koff, float4 (&v)[8]) {
    const int tid = threadIdx.x;
    if (p.vec2) {
        if (g.kfast) {  // 1024 pairs (rr, kk..kk+1)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int pi = tid + 256 * i, kk = 2 * (pi % (g.SK / 2)), rr = pi / (g.SK / 2);
                v[i] = *reinterpret_cast<const float4*>(src + roff[rr] + koff[kk]);
            }
        } else {  // 2048 pairs (rr..rr+1, kk)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int pi = tid + 256 * i, rr = 2 * (pi % (g.SR / 2)), kk = pi / (g.SR / 2);
                v[i] = *reinterpret_cast<const float4*>(src + roff[rr] + koff[kk]);
            }
        }
    } else {  // element e = tid + 256 i; two per float4
        const int ne = g.n / 256;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if (i >= ne) break;
            const int e = tid + 256 * i;
            const int rr = g.kfast ? e / g.SK : e % g.SR, kk = g.kfast ? e % g.SK : e / g.SR;
            const float2 x = src[roff[rr] + koff[kk]];
            if (i & 1) { v[i >> 1].z = x.x; v[i >> 1].w = x.y; }
            else { v[i >> 1].x = x.x; v[i >> 1].y = x.y; }
        }
    }
}

// phase 2: the gathered elements into the staging tile (row rr, k kk at
// rr * LD + kk + kk / 8)
__device__ __forceinline__ void split_stage(const SplitParams& p, const SplitGeom& g, const float4 (&v)[8],
                                            float2* tile) {
    const int tid = threadIdx.x, LD = g.LD;
    if (p.vec2) {
        if (g.kfast) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int pi = tid + 256 * i, kk = 2 * (pi % (g.SK / 2)), rr = pi / (g.SK / 2);
                float2* d = tile + rr * LD + kk + (kk >> 3);
                d[0] = make_float2(v[i].x, v[i].y);
                d[1] = make_float2(v[i].z, v[i].w);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int pi = tid + 256 * i, rr = 2 * (pi % (g.SR / 2)), kk = pi / (g.SR / 2);
                float2* d = tile + rr * LD + kk + (kk >> 3);
                d[0] = make_float2(v[i].x, v[i].y);
                d[LD] = make_float2(v[i].z, v[i].w);
            }
        }
    } else {
        const int ne = g.n / 256;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if (i >= ne) break;
            const int e = tid + 256 * i;
            const int rr = g.kfast ? e / g.SK : e % g.SR, kk = g.kfast ? e % g.SK : e / g.SR;
            tile[rr * LD + kk + (kk >> 3)] = (i & 1) ? make_float2(v[i >> 1].z, v[i >> 1].w)
                                                     : make_float2(v[i >> 1].x, v[i >> 1].y);
        }
    }
}

__device__ __forceinline__ void cp_async8(float2* dst, const float2* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// phases 1 and 2 as asynchronous copies: every element of the block goes from
// global memory straight into its staging-tile slot (8-byte cp.async, no
// registers held), one commit group per block
__device__ __forceinline__ void split_gather_async(const SplitParams& p, const SplitGeom& g, const float2* src,
                                                   const int64_t* roff, const int64_t* koff, float2* tile) {
    const int tid = threadIdx.x, LD = g.LD;
    const int ne = g.n / 256;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        if (i >= ne) break;
        // the element mapping of the pair loads: adjacent lanes take adjacent
        // pairs along the unit-stride mode (coalesced sectors)
        int rr, kk;
        if (p.vec2) {
            const int pi = tid + 256 * (i >> 1);
            if (g.kfast) {
                kk = 2 * (pi % (g.SK / 2)) + (i & 1);
                rr = pi / (g.SK / 2);
            } else {
                rr = 2 * (pi % (g.SR / 2)) + (i & 1);
                kk = pi / (g.SR / 2);
            }
        } else {
            const int e = tid + 256 * i;
            rr = g.kfast ? e / g.SK : e % g.SR;
            kk = g.kfast ? e % g.SK : e / g.SR;
        }
        cp_async8(tile + rr * LD + kk + (kk >> 3), src + roff[rr] + koff[kk]);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// phase 3: the staged tile of block `block` into the part planes (and, in
// FP16x2, the row chunks' scale exponents)
template <int KIND>
__device__ __forceinline__ void split_convert(const SplitParams& p, const SplitGeom& g, int64_t block, int z,
                                              const float2* tile) {
    using C_ = Cfg<KIND, 64>;
    const int64_t R = g.R, K = g.K, tiles_k = g.tiles_k;
    const int SK = g.SK, LD = g.LD, n = g.n;
    const int64_t r0 = (block / tiles_k) * g.SR, k0 = (block % tiles_k) * SK;
    const int tid = threadIdx.x;
    constexpr int Q = C_::PLANES;
    const int64_t plane = R * K;
    uint8_t* out = reinterpret_cast<uint8_t*>(p.dst) + (int64_t)z * Q * plane * C_::ELEM;
    // one thread per 8 consecutive k of one row: every part of Re and Im leaves
    // as one 16-byte (TF32: 32-byte) store; the groups of a row are adjacent lanes
    const int gpr = SK / 8;
    for (int gi = tid; gi < n / 8; gi += 256) {
        const int rr = gi / gpr, g8 = gi % gpr;
        float v[2][8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float2 x = tile[rr * LD + 9 * g8 + j];  // element (rr, 8 g8 + j)
            v[0][j] = x.x;
            v[1][j] = x.y;
        }
        if constexpr (KIND == 3) {
            // the row chunk's largest |Re|, |Im| (non-negative floats order like their bits)
            uint32_t m = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                m = max(m, max(__float_as_uint(fabsf(v[0][j])), __float_as_uint(fabsf(v[1][j]))));
            for (int off = gpr >> 1; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
            const int e = fp16_scale_exp(m);
            if (g8 == 0) p.sexp[((int64_t)z * tiles_k + k0 / SK) * R + r0 + rr] = (int8_t)e;
            const float sc = pow2f(e);  // exact
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                v[0][j] *= sc;
                v[1][j] *= sc;
            }
        }
        const int64_t idx = (r0 + rr) * K + k0 + 8 * g8;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
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
                            const __half2 hh = __floats2half2_rn(v[t][2 * j], v[t][2 * j + 1]);
                            v[t][2 * j] -= __low2float(hh);
                            v[t][2 * j + 1] -= __high2float(hh);
                            w[j] = *reinterpret_cast<const uint32_t*>(&hh);
                        } else {
                            const __nv_bfloat162 hh = __floats2bfloat162_rn(v[t][2 * j], v[t][2 * j + 1]);
                            v[t][2 * j] -= __low2float(hh);
                            v[t][2 * j + 1] -= __high2float(hh);
                            w[j] = *reinterpret_cast<const uint32_t*>(&hh);
                        }
                    }
                    reinterpret_cast<uint4*>(out + ((t * C_::PARTS + q) * plane + idx) * 2)[0] =
                        make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
        }
    }
}

// One block through registers (the standalone split kernel: many CTAs per
// SM keep the memory system busy).
template <int KIND, int BAR>
__device__ __forceinline__ void split_one_block(const SplitParams& p, int64_t block, int z, int64_t slice0,
                                                float2* tile, int64_t* roff, int64_t* koff) {
    const SplitGeom g = split_geom(p);
    const float2* src = p.src.ptr + z * p.src.batch_stride + slice_offset(p.src, slice0 + z);
    float4 v[8];
    split_offsets(p, g, block, roff, koff);
    tc_bar<BAR>();
    split_gather(p, g, src, roff, koff, v);
    split_stage(p, g, v, tile);
    tc_bar<BAR>();
    split_convert<KIND>(p, g, block, z, tile);
    tc_bar<BAR>();  // the tile may be refilled after this
}

// count consecutive blocks, software-pipelined (one CTA per SM runs them):
// the asynchronous copies of blocks i + 1 .. i + D - 1 are in flight while
// block i is converted, through a ring of D staging tiles and offset tables.
// Every block slot commits one copy group (empty past the last block), so
// "all but the newest D - 2 groups complete" means block i has landed.
constexpr int kSplitRing = 4;

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Slot q of the ring: its staging tile at tile0 + q * tile_stride (float2)
// and its offset tables at off0 + 384 q (128 row offsets, then 256 k offsets).
template <int KIND, int BAR, int D>
__device__ __forceinline__ void split_blocks(const SplitParams& p, int64_t block0, int count, int z, int64_t slice0,
                                             float2* tile0, int tile_stride, int64_t* off0) {
    static_assert(D >= 2, "at least one block ahead");
    auto tile = [&](int q) { return tile0 + q * tile_stride; };
    auto roff = [&](int q) { return off0 + 384 * q; };
    auto koff = [&](int q) { return off0 + 384 * q + 128; };
    const SplitGeom g = split_geom(p);
    const float2* src = p.src.ptr + z * p.src.batch_stride + slice_offset(p.src, slice0 + z);
    for (int q = 0; q < D - 1 && q < count; ++q) split_offsets(p, g, block0 + q, roff(q), koff(q));
    tc_bar<BAR>();
    for (int q = 0; q < D - 1; ++q) {
        if (q < count) split_gather_async(p, g, src, roff(q), koff(q), tile(q));
        else asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int i = 0; i < count; ++i) {
        const int j = i % D, jn = (i + D - 1) % D;
        // slot jn held block i - 1: its copies were read before the last barrier
        if (i + D - 1 < count) split_offsets(p, g, block0 + i + D - 1, roff(jn), koff(jn));
        cp_async_wait<D - 2>();
        tc_bar<BAR>();  // tile j and block i + D - 1's offsets complete
        if (i + D - 1 < count) split_gather_async(p, g, src, roff(jn), koff(jn), tile(jn));
        else asm volatile("cp.async.commit_group;" ::: "memory");
        split_convert<KIND>(p, g, block0 + i, z, tile(j));
    }
    cp_async_wait<0>();
    tc_bar<BAR>();  // the tiles may be refilled after this
}

template <int KIND>
__global__ void __launch_bounds__(256) k_split_operand(const __grid_constant__ SplitParams p) {
    extern __shared__ float2 tile[];
    __shared__ int64_t roff[128], koff[256];
    split_one_block<KIND, 0>(p, blockIdx.x, blockIdx.z, p.slice0, tile, roff, koff);
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

// 4D map over planes [batch][PLANES][rows][K]; box = (BK, 128 rows, PLANES, 1).
template <int KIND, int ROWB>
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t K, int batch) {
    using C_ = Cfg<KIND, ROWB>;
    EncodeFn enc = encoder();
    if (!enc) return false;
    constexpr int Q = C_::PLANES;
    cuuint64_t dims[4] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)Q, (cuuint64_t)batch};
    cuuint64_t strides[3] = {(cuuint64_t)(K * C_::ELEM), (cuuint64_t)(rows * K * C_::ELEM),
                             (cuuint64_t)(Q * rows * K * C_::ELEM)};
    cuuint32_t box[4] = {(cuuint32_t)C_::BK, 128u, (cuuint32_t)Q, 1u};  // BK * ELEM = ROWB bytes
    cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = KIND == 1   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : KIND == 3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                               : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = enc(map, dt, 4, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     ROWB == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int KIND, int ROWB>
cudaError_t launch_tc_impl(const TcGemmParams& p, const void* planesA, const void* planesB, int batch,
                           cudaStream_t s) {
    using C_ = Cfg<KIND, ROWB>;
    const int64_t M = 1ll << p.mb, N = 1ll << p.nb, K = 1ll << p.kb;
    if (K % C_::BK || N % TN || M % TM) return cudaErrorInvalidValue;
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
    const int64_t kcta = K >> p.ksplit_bits;  // K of one CTA: whole k-blocks, whole chunks
    if (kcta < C_::BK || (kcta > KC_ELEMS && kcta % KC_ELEMS) || (p.ksplit_bits && (!p.partial || p.accumulate)))
        return cudaErrorInvalidValue;
    k_cgemm_tc<KIND, ROWB><<<dim3((unsigned)tiles, 1u << p.ksplit_bits, batch), NTHREADS, smem, s>>>(ta, tb, p);
    return cudaGetLastError();
}

template <int KIND>
cudaError_t launch_tc_rows(const TcGemmParams& p, const void* pa, const void* pb, int batch, cudaStream_t s) {
    if (p.row_bytes == 32) return launch_tc_impl<KIND, 32>(p, pa, pb, batch, s);
    return launch_tc_impl<KIND, 64>(p, pa, pb, batch, s);
}

// ------------------------------------------------------------ persistent executor

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// One CTA per SM. Thread 0 takes the next task in list order and waits
// (bounded by p.wait_ns of the global timer) until the counters it names reach
// zero, while the other threads stage the task's parameters; then the CTA runs
// it. Split writers hand their planes to the TMA's async proxy; after the
// CTA's barrier, thread 0 fences and decrements the task's counters. A wait
// that runs out, a tensor-core wait that gives up, or an error another CTA has
// recorded stops every CTA at its next task.
template <int KIND, int NT_>
__global__ void __launch_bounds__(NT_, KIND >= 0 ? 1 : 2) k_persist(const __grid_constant__ PersistParams P) {
    extern __shared__ __align__(1024) uint8_t dsmem[];
    __shared__ TcShared sh;
    __shared__ int task_sh;
    const int tid = threadIdx.x, warp = tid >> 5;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~uintptr_t(1023));
    // scratch of the task types, all at the start of the dynamic shared memory:
    // the split's kSplitRing staging tiles, then as many pairs of offset tables
    constexpr int kSplitTileSlot = 40 * 1024;
    constexpr int D = kSplitRing;
    using CK = Cfg<(KIND < 0 ? 0 : KIND), 64>;  // the dynamic shared memory of the tensor-core variants
    static_assert(kSplitTileBytesMax <= kSplitTileSlot &&
                      D * kSplitTileSlot + D * (128 + 256) * 8 <= CK::STAGES * CK::STAGE_BYTES,
                  "split scratch fits the ring");
    float2* const split_tile0 = reinterpret_cast<float2*>(smem);
    int64_t* const split_off0 = reinterpret_cast<int64_t*>(smem + D * kSplitTileSlot);
    double2* root_red = reinterpret_cast<double2*>(smem);
    int64_t(*root_ta)[256] = reinterpret_cast<int64_t(*)[256]>(smem + 4096);
    int64_t(*root_tb)[256] = reinterpret_cast<int64_t(*)[256]>(smem + 4096 + 5 * 256 * 8);
    constexpr bool TC = KIND >= 0;
    if (tid == 0) {
        if constexpr (TC) tc_init(sh);
        else sh.abort = 0;
    }
    if constexpr (TC) {
        if (warp == MMA_WARP) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&sh.tmem_base)),
                         "r"(512u)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if constexpr (TC) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = TC ? sh.tmem_base : 0u;
    const uint64_t wait_ns = P.wait_ns ? P.wait_ns : 10000000000ull;
    TcPipe pipe;
    uint64_t t_wait0 = 0, t_run0 = 0;  // thread 0, for the optional profile
    // The current task's descriptor, and the parameter entry of an FP32 tile or
    // a final-contraction chunk, staged in shared memory while thread 0 waits
    // for the task's inputs: the loads leave the critical path of a dependency.
    __shared__ PersistTask task_sm;
    __shared__ int go_sh;  // 0 once thread 0's wait gave up
    __shared__ __align__(16) uint64_t prm_sm[(sizeof(RootParams) + 7) / 8];
    static_assert(sizeof(GemmParams) <= sizeof(prm_sm) && sizeof(GemmParams) % 8 == 0 &&
                      sizeof(RootParams) % 8 == 0 && (sizeof(RootParams) + 7) / 8 <= NT_,
                  "one 8-byte word of a parameter entry per thread");
    for (;;) {
        if (tid == 0) {
            const int next = atomicAdd(P.ticket, 1);
            task_sh = next;
            if (next < P.ntasks) task_sm = P.tasks[next];
        }
        __syncthreads();
        if (task_sh >= P.ntasks) break;
        const PersistTask tk = task_sm;
        // (not the FP32 variant's tiles: at two CTAs per SM their registers
        // are tighter, and the staged entry cost more spills than it saved)
        if ((TC && tk.type == PT_GEMM) || tk.type == PT_ROOT) {
            const uint64_t* src = tk.type == PT_GEMM ? reinterpret_cast<const uint64_t*>(P.gemm + tk.idx)
                                                     : reinterpret_cast<const uint64_t*>(P.root + tk.idx);
            const int words = (tk.type == PT_GEMM ? (int)sizeof(GemmParams) : (int)sizeof(RootParams)) / 8;
            if (tid < words) prm_sm[tid] = src[tid];
        }
        if (tid == 0) {
            int go = 1;
            const uint64_t t0 = global_ns();
            t_wait0 = t0;
            for (int w = 0; w < 3 && go; ++w) {
                const int c = tk.wait[w];
                if (c < 0) continue;
                // a few polls before backing off with sleeps
                for (int spin = 0; ld_acquire(P.counters + c) > 0; ++spin) {
                    if (*(volatile int*)P.err) {
                        go = 0;
                        break;
                    }
                    if (global_ns() - t0 > wait_ns) {
                        atomicExch(P.err, kErrTimeout);
                        go = 0;
                        break;
                    }
                    if (spin >= 8) __nanosleep(256);
                }
            }
            t_run0 = global_ns();
            go_sh = go;
        }
        // thread 0's acquire of the inputs' counters, then this barrier, orders
        // every thread's reads of them after the producers' writes
        __syncthreads();
        if (!go_sh) break;
        const int64_t slice0 = P.rs0 ? P.rs0[tk.net] : P.slice0;
        switch (tk.type) {
            case PT_GEMM:
                if (tid < 256)
                    f32dev::gemm_tile<1>(TC ? *reinterpret_cast<const GemmParams*>(prm_sm) : P.gemm[tk.idx], tk.item,
                                         tk.z, slice0, *reinterpret_cast<f32dev::GemmSmem*>(smem));
                break;
            case PT_SPLIT:
                if constexpr (TC) {
                    if (tid < 256) {
                        split_blocks<KIND, 1, D>(P.split[tk.idx], tk.item, tk.count, tk.z, slice0, split_tile0,
                                                 kSplitTileSlot / (int)sizeof(float2), split_off0);
                        asm volatile("fence.proxy.async.global;" ::: "memory");
                    }
                }
                break;
            case PT_TC:
                if constexpr (TC) {
                    const TcNode& nd = P.tc[tk.idx];
                    const int64_t tiles = (1ll << (nd.p.mb - 7)) << (nd.p.nb - 7);
                    tc_tile<KIND, 64, true>(&nd.map_a, &nd.map_b, nd.p, tk.item % tiles, (int)(tk.item / tiles),
                                            tk.z, nd.nbatch, smem, sh, tmem, pipe);
                }
                break;
            case PT_KRED: {
                const KredParams& kp = P.kred[tk.idx];
                const int64_t i0 = tk.item * 16384, i1 = i0 + 16384 < kp.mn2 ? i0 + 16384 : kp.mn2;
                for (int64_t i = i0 + tid; i < i1; i += NT_) {
                    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
                    for (int sp = 0; sp < kp.nsplit; ++sp) {
                        const float4 v = reinterpret_cast<const float4*>(kp.partial)[((int64_t)sp * kp.batch + tk.z) * kp.mn2 + i];
                        a0 += v.x;
                        a1 += v.y;
                        a2 += v.z;
                        a3 += v.w;
                    }
                    const int64_t e = 2 * i, m = e >> kp.nb, n = e & ((1ll << kp.nb) - 1);
                    float4* dst = reinterpret_cast<float4*>(kp.C + (int64_t)tk.z * kp.c_batch_stride + m * kp.c_ld + n);
                    float4 r = make_float4((float)a0, (float)a1, (float)a2, (float)a3);
                    if (kp.accumulate) {
                        const float4 o = *dst;
                        r = make_float4(o.x + r.x, o.y + r.y, o.z + r.z, o.w + r.w);
                    }
                    *dst = r;
                }
            } break;
            case PT_ROOT:  // count: the AccParams entry whose partials this chunk fills
                if (tid < 256) {
                    const RootParams& rp = *reinterpret_cast<const RootParams*>(prm_sm);
                    const int R = 1 << (rp.g.mb + rp.g.nb);
                    double2* part = const_cast<double2*>(P.acc[tk.count].partials);
                    f32dev::root_chunk<1>(rp, (int)tk.item, tk.z, slice0,
                                          part + ((int64_t)tk.z * rp.chunks + tk.item) * R, root_red, root_ta,
                                          root_tb);
                }
                break;
            case PT_ACC: {
                const AccParams& ap = P.acc[tk.idx];
                double2* const dst = P.out0 ? P.out0 : ap.out;
                const int64_t R = 1ll << ap.pp.obits;
                for (int64_t r = tid; r < R; r += NT_) {
                    const int64_t src = f32dev::bits_offset(r, ap.pp.ostride, ap.pp.obits, 0);
                    double2 acc = make_double2(0.0, 0.0);
                    for (int i = 0; i < ap.count; ++i) {
                        const double2 v = ap.partials[(int64_t)i * R + src];
                        acc.x += v.x;
                        acc.y += v.y;
                    }
                    dst[r].x += acc.x;
                    dst[r].y += acc.y;
                }
            } break;
            case PT_SUM: {
                const SumTaskParams& sp = P.sum[tk.idx];
                double2* const dst = P.out0 ? P.out0 : sp.out;
                const int64_t R = 1ll << sp.sp.obits;
                for (int64_t r = tid; r < R; r += NT_) {
                    const int64_t off = f32dev::bits_offset(r, sp.sp.ostride, sp.sp.obits, 0);
                    double2 acc = make_double2(0.0, 0.0);
                    for (int z = 0; z < sp.batch; ++z) {
                        const float2* src = sp.sp.src.ptr + z * sp.sp.src.batch_stride +
                                            f32dev::slice_offset(sp.sp.src, slice0 + z);
                        const float2 v = src[off];
                        acc.x += v.x;
                        acc.y += v.y;
                    }
                    dst[r].x += acc.x;
                    dst[r].y += acc.y;
                }
            } break;
            default:
                break;
        }
        // this task's generic shared-memory stores (split tiles, GEMM operands,
        // staged outputs) before the next task's TMA writes to the same bytes
        if constexpr (TC) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            // the barrier, then thread 0's fence: every thread's writes of the
            // task are visible before its counters count down
            __threadfence();
            if (sh.abort) atomicExch(P.err, kErrTimeout);
            atomicSub(P.counters + tk.signal, 1);
            if (tk.signal2 >= 0) atomicSub(P.counters + tk.signal2, 1);
            if (P.prof && tk.type >= 0 && tk.type < 8) {
                const uint64_t t1 = global_ns();
                atomicAdd(P.prof + 3 * tk.type, (unsigned long long)(t1 - t_run0));
                atomicAdd(P.prof + 3 * tk.type + 1, 1ull);
                atomicAdd(P.prof + 3 * tk.type + 2, (unsigned long long)(t_run0 - t_wait0));
            }
        }
        if (sh.abort) break;
    }
    if constexpr (TC) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (warp == MMA_WARP) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
        }
    }
}

template <int KIND, int NT_>
cudaError_t launch_persist_impl(const PersistParams& p, size_t smem, cudaStream_t s) {
    static size_t set_for = 0;
    if (smem > set_for) {
        cudaError_t e = cudaFuncSetAttribute(k_persist<KIND, NT_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set_for = smem;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    k_persist<KIND, NT_><<<KIND >= 0 ? sms : 2 * sms, NT_, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

// tnc_mode -> kernel configuration: 1 TF32 (2 parts), 2 BF16 (3 parts), 3 BF16 (2 parts),
// 4 scaled FP16 (2 parts)
static int kind_of(int mode) { return mode == 1 ? 1 : (mode == 2 ? 0 : (mode == 4 ? 3 : 2)); }

int tc_plane_count(int mode) { return mode == 2 ? 6 : 4; }
int tc_elem_bytes(int mode) { return mode == 1 ? 4 : 2; }
int tc_min_kb(int) { return 5; }
int tc_scale_chunks(int kb) { return 1 << (kb > 8 ? kb - 8 : 0); }

// Whether the split may load pairs of elements adjacent along the operand's
// unit-stride mode (bit 0 of k, else bit 0 of the rows) as one 16-byte load:
// the unit stride sits there, every other stride is even, and the base is
// 16-byte aligned, so every pair starts on a 16-byte boundary.
static bool split_pairs(const SplitParams& p) {
    const bool kfast = p.kb > 0 && p.ks[0] == 1;
    if (!kfast && !(p.rb > 0 && p.rs[0] == 1)) return false;
    if (reinterpret_cast<uintptr_t>(p.src.ptr) % 16 || p.src.batch_stride % 2) return false;
    for (int j = 0; j < p.src.n_sl; ++j)
        if (p.src.sl_stride[j] % 2) return false;
    for (int j = kfast ? 1 : 0; j < p.kb; ++j)
        if (p.ks[j] % 2) return false;
    for (int j = kfast ? 0 : 1; j < p.rb; ++j)
        if (p.rs[j] % 2) return false;
    return true;
}

cudaError_t launch_split(const SplitParams& p_in, int mode, int batch, cudaStream_t s) {
    SplitParams p = p_in;
    p.vec2 = split_pairs(p) ? 1 : 0;
    const int64_t R = 1ll << p.rb, K = 1ll << p.kb;
    if (K < 32 || batch < 1 || batch > 65535 || p.rb < 7) return cudaErrorInvalidConfiguration;
    const bool kfast = p.kb > 0 && p.ks[0] == 1;
    const int64_t SK = split_tile_k(p.kb), SR = split_tile_rows(p.kb, kfast);
    if (R < SR || SR > 128) return cudaErrorInvalidConfiguration;
    const int64_t blocks = (R / SR) * (K / SK);
    const dim3 grid((unsigned)blocks, 1, batch);
    const size_t smem = (size_t)SR * split_ld((int)SK) * sizeof(float2);
    switch (kind_of(mode)) {
        case 0: k_split_operand<0><<<grid, 256, smem, s>>>(p); break;
        case 1: k_split_operand<1><<<grid, 256, smem, s>>>(p); break;
        case 3:
            if (!p.sexp) return cudaErrorInvalidValue;
            k_split_operand<3><<<grid, 256, smem, s>>>(p);
            break;
        default: k_split_operand<2><<<grid, 256, smem, s>>>(p); break;
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

cudaError_t launch_persist(const PersistParams& p, int mode, cudaStream_t s) {
    if (!p.tasks || p.ntasks < 0 || !p.counters || !p.ticket || !p.err) return cudaErrorInvalidValue;
    if (mode == 0) {
        const size_t smem = (sizeof(f32dev::GemmSmem) > 28 * 1024 ? sizeof(f32dev::GemmSmem) : 28 * 1024) + 1024;
        return launch_persist_impl<-1, 256>(p, smem, s);
    }
    switch (kind_of(mode)) {
        case 0: return launch_persist_impl<0, NTHREADS>(p, Cfg<0, 64>::STAGES * Cfg<0, 64>::STAGE_BYTES + 1024, s);
        case 1: return launch_persist_impl<1, NTHREADS>(p, Cfg<1, 64>::STAGES * Cfg<1, 64>::STAGE_BYTES + 1024, s);
        case 3: return launch_persist_impl<3, NTHREADS>(p, Cfg<3, 64>::STAGES * Cfg<3, 64>::STAGE_BYTES + 1024, s);
        default: return launch_persist_impl<2, NTHREADS>(p, Cfg<2, 64>::STAGES * Cfg<2, 64>::STAGE_BYTES + 1024, s);
    }
}

bool tc_make_node(TcNode* node, const TcGemmParams& p, int mode, const void* planesA, const void* planesB,
                  int batch) {
    const int64_t M = 1ll << p.mb, N = 1ll << p.nb, K = 1ll << p.kb;
    if (p.mb < 7 || p.nb < 7 || p.kb < tc_min_kb(mode) || (K >> p.ksplit_bits) < 32) return false;
    if ((K >> p.ksplit_bits) > KC_ELEMS && (K >> p.ksplit_bits) % KC_ELEMS) return false;
    node->p = p;
    node->nbatch = batch;
    switch (kind_of(mode)) {
        case 0: return make_map<0, 64>(&node->map_a, planesA, M, K, batch) && make_map<0, 64>(&node->map_b, planesB, N, K, batch);
        case 1: return make_map<1, 64>(&node->map_a, planesA, M, K, batch) && make_map<1, 64>(&node->map_b, planesB, N, K, batch);
        case 3: return make_map<3, 64>(&node->map_a, planesA, M, K, batch) && make_map<3, 64>(&node->map_b, planesB, N, K, batch);
        default: return make_map<2, 64>(&node->map_a, planesA, M, K, batch) && make_map<2, 64>(&node->map_b, planesB, N, K, batch);
    }
}

int64_t tc_node_tiles(const TcGemmParams& p) { return ((1ll << (p.mb - 7)) << (p.nb - 7)) << p.ksplit_bits; }

int64_t tc_split_prepare(SplitParams& p) {
    p.vec2 = split_pairs(p) ? 1 : 0;
    const bool kfast = p.kb > 0 && p.ks[0] == 1;
    const int64_t SK = split_tile_k(p.kb), SR = split_tile_rows(p.kb, kfast);
    if (p.kb < 5 || SR > 128 || (1ll << p.rb) < SR) return 0;  // the tile and offset tables would not fit
    return ((1ll << p.rb) / SR) * ((1ll << p.kb) / SK);
}

cudaError_t launch_cgemm_tc(const TcGemmParams& p, int mode, const void* planesA, const void* planesB,
                            int batch, cudaStream_t s) {
    if (p.mb < 7 || p.nb < 7 || p.kb < tc_min_kb(mode) || batch < 1 || batch > 65535)
        return cudaErrorInvalidConfiguration;
    switch (kind_of(mode)) {
        case 0: return launch_tc_rows<0>(p, planesA, planesB, batch, s);
        case 1: return launch_tc_rows<1>(p, planesA, planesB, batch, s);
        case 3:
            if (!p.sexp_a || !p.sexp_b) return cudaErrorInvalidValue;
            return launch_tc_rows<3>(p, planesA, planesB, batch, s);
        default: return launch_tc_rows<2>(p, planesA, planesB, batch, s);
    }
}

}  // namespace tnc
