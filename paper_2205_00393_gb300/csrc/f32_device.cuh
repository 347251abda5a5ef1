// Device code shared by the FP32 CUDA-core kernels and the persistent
// executor: the permute-fused complex64 contraction tile and the FP64 final
// reduction. BAR selects the barrier among the threads that run a routine:
// 0 = the whole CTA (__syncthreads), 1 = named barrier 1 over threads 0-255 of
// a larger CTA (the persistent executor's other warps do not take part).
#pragma once

#include "kernels.h"

namespace tnc {
namespace f32dev {

template <int BAR>
__device__ __forceinline__ void bar_sync() {
    if constexpr (BAR == 0) __syncthreads();
    else asm volatile("bar.sync 1, 256;" ::: "memory");
}

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
// Shared-memory stages are double buffered: the gather of tile t+1 goes to
// registers while tile t is multiplied, then to the other stage (one barrier
// per tile). Accumulation is two-level: each group of GROUP_TILES k-tiles is
// summed in a fresh partial that is then added to the result with TwoSum
// (Knuth's error-free addition), whose rounding errors are collected in a
// per-thread compensation kept in shared memory and added once at the end.
// The FP32 rounding error thus grows like the 64-term partial sums alone
// instead of also with the K / 64 additions of partials, and the register
// budget (128 per thread) still keeps two CTAs per SM.
constexpr int PAD = 2;           // keeps 16-byte alignment of fragment rows
constexpr int GROUP_TILES = 4;   // 64 k-terms per partial sum


// B columns are stored interleaved: column n goes to half (n >> 1) & 1 at
// position (n >> 2) * 2 + (n & 1), so the two 16-byte halves of the four
// columns a thread owns are contiguous across the warp (one 256-byte span per
// load instead of a 512-byte stride).
constexpr int BH = BN / 2 + PAD;
struct GemmSmem {
    float2 As[2][BK][BM + PAD];
    float2 Bs[2][BK][2][BH];
    int64_t rowA[BM], colB[BN], klA[BK], klB[BK];
    float2 comp[16][NT];  // TwoSum compensation of each thread's 4 x 4 outputs
};

// a += b with the rounding error of the addition added to c (TwoSum: the
// error term is exact whatever the magnitudes of a and b)
__device__ __forceinline__ void two_sum_into(float& a, float b, float& c) {
    const float s = a + b;
    const float bv = s - a;
    const float e = (a - (s - bv)) + (b - bv);
    a = s;
    c += e;
}

// Operand pointer of gemm_tile. Alone in a launch (BAR 0) the operands were
// written by earlier launches and may be read through the read-only path;
// inside the persistent executor (BAR 1) other CTAs of the same launch wrote
// them, so the loads stay on the coherent path.
template <int BAR> struct OperandPtr { using type = const float2* __restrict__; };
template <> struct OperandPtr<1> { using type = const float2*; };

// One 64x64 output tile `tile` of slice z (slice id slice0 + z) of the
// contraction described by p.
template <int BAR = 0>
__device__ __forceinline__ void gemm_tile(const GemmParams& p, int64_t tile, int z, int64_t slice0,
                                          GemmSmem& sm) {
    auto& As = sm.As;
    auto& Bs = sm.Bs;
    auto& rowA = sm.rowA;
    auto& colB = sm.colB;
    auto& klA = sm.klA;
    auto& klB = sm.klB;
    const int tid = threadIdx.x;
    const int64_t M = 1ll << p.mb, N = 1ll << p.nb, K = 1ll << p.kb;
    const int64_t tiles_n = (N + BN - 1) / BN;
    const int64_t m0 = (tile / tiles_n) * BM, n0 = (tile % tiles_n) * BN;
    const int64_t s = slice0 + z;
    const typename OperandPtr<BAR>::type A = p.A.ptr + z * p.A.batch_stride + slice_offset(p.A, s);
    const typename OperandPtr<BAR>::type B = p.B.ptr + z * p.B.batch_stride + slice_offset(p.B, s);

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
    int la_k[4], la_m[4], lb_k[4], lb_n[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int e = tid + i * NT;
        if (a_kfast) { la_k[i] = e % BK; la_m[i] = e / BK; }
        else { la_m[i] = e % BM; la_k[i] = e / BM; }
        if (b_nfast) { lb_n[i] = e % BN; lb_k[i] = e / BN; }
        else { lb_k[i] = e % BK; lb_n[i] = e / BK; }
    }
    bar_sync<BAR>();

    float2 ra[4], rb[4];
    auto gather = [&](int64_t k0) {
        const int64_t khA = bits_offset(k0, p.ak, p.kb, LOG_BK);
        const int64_t khB = bits_offset(k0, p.bk, p.kb, LOG_BK);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ra[i] = make_float2(0.f, 0.f);
            if (m0 + la_m[i] < M && k0 + la_k[i] < K) ra[i] = A[rowA[la_m[i]] + khA + klA[la_k[i]]];
            rb[i] = make_float2(0.f, 0.f);
            if (n0 + lb_n[i] < N && k0 + lb_k[i] < K) rb[i] = B[colB[lb_n[i]] + khB + klB[lb_k[i]]];
        }
    };
    auto stage_store = [&](int st) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            As[st][la_k[i]][la_m[i]] = ra[i];
            Bs[st][lb_k[i]][(lb_n[i] >> 1) & 1][(lb_n[i] >> 2) * 2 + (lb_n[i] & 1)] = rb[i];
        }
    };

    const int tx = tid & 15, ty = tid >> 4;
    float2 acc[4][4], part[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc[i][j] = make_float2(0.f, 0.f);
            part[i][j] = make_float2(0.f, 0.f);
            sm.comp[4 * i + j][tid] = make_float2(0.f, 0.f);  // this thread's own slots
        }

    const int64_t ntiles = (K + BK - 1) / BK;
    // K is a power of two: below BK, the one k-tile has K nonzero rows and the
    // zero-padded rest is skipped
    const int kmax = K < BK ? (int)K : BK;
    gather(0);
    stage_store(0);
    bar_sync<BAR>();
    for (int64_t t = 0; t < ntiles; ++t) {
        const int st = (int)(t & 1);
        if (t + 1 < ntiles) gather((t + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            if (kk >= kmax) break;
            float4 a01 = *reinterpret_cast<const float4*>(&As[st][kk][4 * ty]);
            float4 a23 = *reinterpret_cast<const float4*>(&As[st][kk][4 * ty + 2]);
            float4 b01 = *reinterpret_cast<const float4*>(&Bs[st][kk][0][2 * tx]);
            float4 b23 = *reinterpret_cast<const float4*>(&Bs[st][kk][1][2 * tx]);
            float2 a[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w),
                           make_float2(a23.x, a23.y), make_float2(a23.z, a23.w)};
            float2 b[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w),
                           make_float2(b23.x, b23.y), make_float2(b23.z, b23.w)};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cmac(part[i][j], a[i], b[j]);
        }
        if ((t + 1) % GROUP_TILES == 0 || t + 1 == ntiles) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float2 c = sm.comp[4 * i + j][tid];
                    two_sum_into(acc[i][j].x, part[i][j].x, c.x);
                    two_sum_into(acc[i][j].y, part[i][j].y, c.y);
                    sm.comp[4 * i + j][tid] = c;
                    part[i][j] = make_float2(0.f, 0.f);
                }
        }
        if (t + 1 < ntiles) stage_store(st ^ 1);
        bar_sync<BAR>();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 c = sm.comp[4 * i + j][tid];
            acc[i][j].x += c.x;
            acc[i][j].y += c.y;
        }
    float2* C = p.C + z * p.c_batch_stride;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t m = m0 + 4 * ty + i;
        if (m >= M) continue;
        if (n0 + 4 * tx + 3 < N) {
            float4* dst = reinterpret_cast<float4*>(C + m * N + n0 + 4 * tx);
            dst[0] = make_float4(acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y);
            dst[1] = make_float4(acc[i][2].x, acc[i][2].y, acc[i][3].x, acc[i][3].y);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int64_t n = n0 + 4 * tx + j;
                if (n < N) C[m * N + n] = acc[i][j];
            }
        }
    }
}

// Sum over this thread's k in [k_lo, k_hi) (k = k_lo + lane, + lanes, ...) of
// A[k] B[k] for the final contraction. When the block's K range holds whole
// rows of lanes, k = lanes * j + lane: the low bits are the lane (one offset
// per thread) and the offsets of j's bits come from shared-memory tables ta,
// tb, one per 8-bit group (K <= 2^40); products are summed in FP32 over runs
// of 16 j and the runs in FP64. Called by every thread of the block.
template <int BAR = 0>
__device__ void root_dot(const GemmParams& p, const float2* A, const float2* B, int64_t k_lo, int64_t k_hi,
                         int lane, int lanes, int64_t (*root_ta)[256], int64_t (*root_tb)[256], double& re,
                         double& im) {
    const int64_t kc = k_hi - k_lo;
    int lb = 0;
    while ((1 << lb) < lanes) ++lb;
    if (kc >= lanes) {
        // k = lanes * j + lane: the low lb bits are the lane (one offset per
        // thread); the offsets of j's bits come from shared-memory tables, one
        // per 8-bit group. Products are summed in FP32 over runs of 16 j and
        // the runs in FP64.
        const int jb = p.kb - lb, ng = (jb + 7) / 8;
        for (int idx = threadIdx.x; idx < ng * 256; idx += 256) {
            const int g = idx >> 8, e = idx & 255;
            int64_t oa = 0, ob = 0;
            for (int t = 0; t < 8; ++t) {
                const int bit = lb + 8 * g + t;
                if (bit < p.kb && ((e >> t) & 1)) {
                    oa += p.ak[bit];
                    ob += p.bk[bit];
                }
            }
            root_ta[g][e] = oa;
            root_tb[g][e] = ob;
        }
        bar_sync<BAR>();
        const float2* Al = A + bits_offset(lane, p.ak, lb, 0);
        const float2* Bl = B + bits_offset(lane, p.bk, lb, 0);
        const int64_t j_lo = k_lo >> lb, j_hi = k_hi >> lb;
        for (int64_t j0 = j_lo; j0 < j_hi; j0 += 16) {
            const int64_t je = j0 + 16 < j_hi ? j0 + 16 : j_hi;
            float sr = 0.f, si = 0.f;
            for (int64_t j = j0; j < je; ++j) {
                int64_t oa = 0, ob = 0;
                for (int g = 0; g < ng; ++g) {
                    const int e = (int)((j >> (8 * g)) & 255);
                    oa += root_ta[g][e];
                    ob += root_tb[g][e];
                }
                const float2 a = Al[oa], b = Bl[ob];
                sr = fmaf(a.x, b.x, sr);
                sr = fmaf(-a.y, b.y, sr);
                si = fmaf(a.x, b.y, si);
                si = fmaf(a.y, b.x, si);
            }
            re += sr;
            im += si;
        }
    } else {
        for (int64_t k = k_lo + lane; k < k_hi; k += lanes) {
            float2 a = A[bits_offset(k, p.ak, p.kb, 0)];
            float2 b = B[bits_offset(k, p.bk, p.kb, 0)];
            re += (double)a.x * b.x - (double)a.y * b.y;
            im += (double)a.x * b.y + (double)a.y * b.x;
        }
    }
}


// FP64 partial sums of chunk `chunk` of a final contraction with R = M*N <= 64
// outputs, slice z (slice id slice0 + z), written to out[r] (r < R). Run by
// threads 0-255; red, ta, tb are shared-memory scratch.
template <int BAR = 0>
__device__ __forceinline__ void root_chunk(const RootParams& rp, int chunk, int z, int64_t slice0, double2* out,
                                           double2* red, int64_t (*ta)[256], int64_t (*tb)[256]) {
    const GemmParams& p = rp.g;
    const int R = 1 << (p.mb + p.nb);
    const int lanes = 256 / R;
    const int r = threadIdx.x / lanes, lane = threadIdx.x % lanes;
    const int64_t m = r >> p.nb, n = r & ((1 << p.nb) - 1);
    const int64_t s = slice0 + z;
    const float2* A = p.A.ptr + z * p.A.batch_stride + slice_offset(p.A, s) + bits_offset(m, p.am, p.mb, 0);
    const float2* B = p.B.ptr + z * p.B.batch_stride + slice_offset(p.B, s) + bits_offset(n, p.bn, p.nb, 0);
    const int64_t K = 1ll << p.kb;
    const int64_t kc = K / rp.chunks;
    const int64_t k_lo = chunk * kc, k_hi = k_lo + kc;
    double re = 0.0, im = 0.0;
    root_dot<BAR>(p, A, B, k_lo, k_hi, lane, lanes, ta, tb, re, im);
    red[threadIdx.x] = make_double2(re, im);
    bar_sync<BAR>();
    for (int st = lanes / 2; st > 0; st >>= 1) {
        if (lane < st) {
            double2 o = red[threadIdx.x + st];
            red[threadIdx.x].x += o.x;
            red[threadIdx.x].y += o.y;
        }
        bar_sync<BAR>();
    }
    if (lane == 0) out[r] = red[threadIdx.x];
}

}  // namespace f32dev
}  // namespace tnc
