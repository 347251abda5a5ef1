// Fused multi-step stem kernel: the GPU form of the paper's secondary slicing
// (Sec. 5.2, Fig. 8-9). A stem tensor that absorbs small branch tensors in n
// consecutive narrow contractions is read from HBM once and written once:
// the modes that live through all n steps (the paper slices exactly these,
// picking them by lifetime) index independent sub-tensors, one per CTA; each
// CTA keeps its sub-tensor in shared memory across the n absorptions. Every
// contraction is the same complex product as on the FP32 path (products and
// sums in FP32), so a fused group gives what its n separate launches give up
// to the order of the additions within one output element.
#include "kernels.h"

namespace tnc {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ int64_t slice_offset(const Operand& op, int64_t s) {
    int64_t off = 0;
    for (int j = 0; j < op.n_sl; ++j) off += ((s >> op.sl_bit[j]) & 1) * op.sl_stride[j];
    return off;
}

template <typename T>
__device__ __forceinline__ T bits_dec(uint32_t x, const T* str, int nbits) {
    T off = 0;
    for (int b = 0; b < nbits; ++b)
        if ((x >> b) & 1u) off += str[b];
    return off;
}

__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

// x with a zero bit inserted at each of the first nk positions of ins (ascending)
__device__ __forceinline__ uint32_t deposit(uint32_t x, const int* ins, int nk) {
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (t < nk) x = ((x >> ins[t]) << (ins[t] + 1)) | (x & ((1u << ins[t]) - 1u));
    return x;
}

// In-place step with K = N = 2^NK: every thread takes two rows per iteration
// (two independent FMA chains), loads their K elements, and writes the K
// results back to the same positions.
template <int NK>
__device__ __forceinline__ void inplace_step(float2* cur, const float2* bd, const int* ins, const int* kx, int rows,
                                             int tid) {
    constexpr int K = 1 << NK;
    // rows r0 + tid and r0 + NT + tid: consecutive lanes take consecutive rows
    for (int r0 = 0; r0 < rows; r0 += 2 * NT) {
        const bool two = r0 + NT + tid < rows;
        if (r0 + tid >= rows) break;
        uint32_t base[2];
        float2 x[2][K];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            base[h] = deposit((uint32_t)(r0 + h * NT + tid), ins, NK);
#pragma unroll
            for (int k = 0; k < K; ++k) x[h][k] = (h == 0 || two) ? cur[base[h] + kx[k]] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int n = 0; n < K; ++n) {
            float2 acc[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float2 b = bd[k * K + n];
                cmac(acc[0], x[0][k], b);
                cmac(acc[1], x[1][k], b);
            }
            cur[base[0] + kx[n]] = acc[0];
            if (two) cur[base[1] + kx[n]] = acc[1];
        }
    }
}

// One CTA per outer assignment (blockIdx.x) and slice of the batch (blockIdx.z).
// Shared memory: one or two buffers of 2^cap_log2 complex elements (X_{i-1},
// X_i) and the dense [K][N] copies of every step's branch.
__global__ void __launch_bounds__(NT, 4) k_stem_fused(const StemParams* __restrict__ P, int cap_log2,
                                                   int64_t slice0) {
    extern __shared__ float2 stem_smem[];
    const StemParams& p = *P;
    float2* cur = stem_smem;
    float2* nxt = stem_smem + (1 << cap_log2);
    float2* bsm = stem_smem + ((p.two_buffers ? 2 : 1) << cap_log2);
    const int z = blockIdx.z, tid = threadIdx.x;
    const int64_t s = slice0 + z;
    const uint32_t u = blockIdx.x;
    // dense [k][n] copies of the branches of this slice
    for (int i = 0; i < p.nsteps; ++i) {
        const StemStep& st = p.steps[i];
        const int N = 1 << st.nn, KN = 1 << (st.nk + st.nn);
        const float2* bp = st.br.ptr + z * st.br.batch_stride + slice_offset(st.br, s);
        for (int e = tid; e < KN; e += NT)
            bsm[st.b_off + e] = bp[bits_dec((uint32_t)(e >> st.nn), st.kstr_b, st.nk) +
                                   bits_dec((uint32_t)(e & (N - 1)), st.nstr_b, st.nn)];
    }
    // the sub-tensor X_0 of T_0 at this outer assignment
    int64_t ib = 0, ob = 0;
    for (int b = 0; b < p.nu; ++b)
        if ((u >> b) & 1u) {
            ib += p.ustr_in[b];
            ob += p.ustr_out[b];
        }
    const float2* src = p.in.ptr + z * p.in.batch_stride + slice_offset(p.in, s) + ib;
    {
        // element e = tid + NT * j: the low 8 bits are this thread's, decoded
        // once; every element goes straight to shared memory as an 8-byte
        // asynchronous copy, all of them in flight before the wait
        const int n_in = p.n_in, lo_bits = n_in < 8 ? n_in : 8;
        const int64_t lo = bits_dec((uint32_t)tid, p.istr, lo_bits);
        const int cnt = (1 << n_in) > NT ? (1 << n_in) / NT : 1;
        if (tid < (1 << n_in))
            for (int j = 0; j < cnt; ++j) {
                const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(cur + tid + NT * j));
                const float2* g = src + lo + bits_dec((uint32_t)j, p.istr + 8, n_in - lo_bits);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(g) : "memory");
            }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    for (int i = 0; i < p.nsteps; ++i) {
        const StemStep& st = p.steps[i];
        const int nk = st.nk, K = 1 << nk, N = 1 << st.nn, rows = 1 << st.nr;
        int kx[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) kx[k] = k < K ? bits_dec((uint32_t)k, st.kstr_x, nk) : 0;
        const float2* bd = bsm + st.b_off;
        if (st.inplace && (nk == 1 || nk == 2) && rows >= 2) {
            int ins[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) ins[t] = t < nk ? st.ins[t] : 0;
            if (nk == 1) inplace_step<1>(cur, bd, ins, kx, rows, tid);
            else inplace_step<2>(cur, bd, ins, kx, rows, tid);
            __syncthreads();
        } else if (st.inplace) {
            // rows r: the bits of X outside the contracted positions; a zero
            // is inserted at each contracted position, ascending
            int ins[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) ins[t] = t < nk ? st.ins[t] : 0;
            for (int r = tid; r < rows; r += NT) {
                uint32_t base = (uint32_t)r;
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (t < nk) base = ((base >> ins[t]) << (ins[t] + 1)) | (base & ((1u << ins[t]) - 1u));
                float2 xk[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) xk[k] = k < K ? cur[base + kx[k]] : make_float2(0.f, 0.f);
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                    if (n >= K) break;
                    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        if (k < K) cmac(acc, xk[k], bd[k * K + n]);
                    cur[base + kx[n]] = acc;
                }
            }
            __syncthreads();
        } else {
            int rstr[kStemMaxInner];
#pragma unroll
            for (int b = 0; b < kStemMaxInner; ++b) rstr[b] = b < st.nr ? st.rstr[b] : 0;
            for (int r = tid; r < rows; r += NT) {
                int xo = 0;
#pragma unroll
                for (int b = 0; b < kStemMaxInner; ++b)
                    if ((r >> b) & 1) xo += rstr[b];
                float2 xk[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) xk[k] = k < K ? cur[xo + kx[k]] : make_float2(0.f, 0.f);
                for (int n = 0; n < N; ++n) {
                    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        if (k < K) cmac(acc, xk[k], bd[k * N + n]);
                    nxt[r * N + n] = acc;
                }
            }
            __syncthreads();
            float2* t = cur;
            cur = nxt;
            nxt = t;
        }
    }
    float2* dst = p.out + z * p.out_batch_stride + ob;
    {
        const int n_out = p.n_out, lo_bits = n_out < 8 ? n_out : 8;
        const int64_t lo = bits_dec((uint32_t)tid, p.ostr, lo_bits);
        const int cnt = (1 << n_out) > NT ? (1 << n_out) / NT : 1;
        if (tid < (1 << n_out))
            for (int j = 0; j < cnt; ++j)
                dst[lo + bits_dec((uint32_t)j, p.ostr + 8, n_out - lo_bits)] = cur[tid + NT * j];
    }
}

}  // namespace

cudaError_t launch_stem_fused(const StemParams* d_params, const StemParams& hp, int cap_log2, int64_t slice0,
                              int batch, cudaStream_t s) {
    if (!d_params || cap_log2 < 1 || cap_log2 > kStemMaxInner || hp.nu < 0 || hp.nu > 30 || hp.nsteps < 1 ||
        hp.nsteps > kStemMaxSteps || hp.n_in > cap_log2 || hp.n_out > cap_log2 || batch < 1 || batch > 65535)
        return cudaErrorInvalidValue;
    // every step reads exactly the sub-tensor the previous one wrote, and an
    // in-place step's positions lie inside it, ascending
    int bits = hp.n_in;
    bool two = false;
    for (int i = 0; i < hp.nsteps; ++i) {
        const StemStep& st = hp.steps[i];
        if (st.nk < 0 || st.nk > 4 || st.nn < 0 || st.nn > 4 || st.nr < 0 || st.nr + st.nk != bits ||
            st.nr + st.nn > cap_log2 || st.b_off < 0 || st.b_off + (1 << (st.nk + st.nn)) > hp.b_total)
            return cudaErrorInvalidValue;
        if (st.inplace) {
            if (st.nk != st.nn) return cudaErrorInvalidValue;
            for (int t = 0; t < st.nk; ++t)
                if (st.ins[t] < 0 || st.ins[t] >= bits || (t > 0 && st.ins[t] <= st.ins[t - 1]))
                    return cudaErrorInvalidValue;
        } else {
            two = true;
        }
        bits = st.nr + st.nn;
    }
    if (bits != hp.n_out || (two && !hp.two_buffers)) return cudaErrorInvalidValue;
    const size_t smem = ((size_t)((hp.two_buffers ? 2u : 1u) << cap_log2) + (size_t)hp.b_total) * sizeof(float2);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    static int set_for = 0;
    if ((int)smem > set_for) {
        cudaError_t e = cudaFuncSetAttribute(k_stem_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set_for = (int)smem;
    }
    k_stem_fused<<<dim3(1u << hp.nu, 1, batch), NT, smem, s>>>(d_params, cap_log2, slice0);
    return cudaGetLastError();
}

}  // namespace tnc
