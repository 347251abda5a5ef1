// Internal interface between the host executors (host_*.cpp) and the CUDA
// kernels. Not part of the public C ABI.
//
// Tensors are complex64 arrays whose dimensions are all 2 internally: an index
// of dimension 2^d is split into d binary modes (most significant first), so a
// row-major tensor over indices is a row-major tensor over binary modes and
// every permutation is a permutation of address bits. A pairwise contraction
// (Sec. 2.1.1, TTGT form of Sec. 5.3.1: A's free modes first, contracted
// modes last; B's contracted modes first) is then
//     C[m, n] = sum_k A(m, k) B(k, n),   M = 2^mb, N = 2^nb, K = 2^kb,
// with A(m, k) = A_base[sum_j bit_j(m) am[j] + sum_j bit_j(k) ak[j]] (and
// likewise for B): the permutation is a per-bit stride table applied during
// the operand load, never a separate pass. The output is row-major [m][n].
#pragma once

#include <cstdint>
#include <string>
#include <cuda.h>
#include <cuda_runtime.h>

namespace tnc {

constexpr int kMaxBits = 40;      // binary modes per operand side
constexpr int kMaxSliceBits = 16; // sliced modes of one leaf

// One operand of a launch covering `batch` consecutive slices s = slice0 + z.
// Element address for slice z: ptr + z * batch_stride + slice_offset(s) + ...
// where slice_offset(s) = sum_j ((s >> sl_bit[j]) & 1) * sl_stride[j] fixes the
// sliced modes of a leaf (Sec. 2.1.1: a sliced index takes one value per task).
struct Operand {
    const float2* ptr;
    int64_t batch_stride;
    int n_sl;
    int sl_bit[kMaxSliceBits];
    int64_t sl_stride[kMaxSliceBits];
};

struct GemmParams {
    Operand A, B;
    float2* C;
    int64_t c_batch_stride;
    int mb, nb, kb;
    int64_t am[kMaxBits], ak[kMaxBits], bk[kMaxBits], bn[kMaxBits];
    int64_t slice0;
};

// Final contraction whose output has R = 2^(mb+nb) <= 64 elements: FP64
// partial sums over chunks of K (Sec. 2.1.1: results of all subtasks are
// accumulated; the reduction runs in FP64 in a fixed order).
struct RootParams {
    GemmParams g;
    int chunks;       // K is split into `chunks` equal parts (power of two)
};

// Accumulate an FP32 tensor of R = 2^obits elements per slice into the FP64
// result: out[r] += sum_z src_z[ sum_j bit_j(r) ostride[j] ] (r in result order).
struct SumParams {
    Operand src;
    int obits;
    int64_t ostride[kMaxBits];
    int64_t slice0;
};

// Result-order permutation for accumulating FP64 partials laid out in the
// root's own order.
struct PermParams {
    int obits;
    int64_t ostride[kMaxBits];
};

// Operand split for the tensor-core path: the logical matrix X[R][K]
// (R = M for A, N for B) with X(r, k) = src[r strides + k strides] is
// written as K-major planes [batch][2 * parts][R][K] (the parts of Re, then
// the parts of Im).
struct SplitParams {
    Operand src;
    int rb, kb;
    int64_t rs[kMaxBits], ks[kMaxBits];
    int64_t slice0;
    void* dst;
    int8_t* sexp;          // split FP16x2: scale exponents [batch][K / min(K, 256)][R] (written here)
    int vec2;              // set by launch_split: pairs along the unit-stride mode load as 16 bytes
};

struct TcGemmParams {
    int mb, nb, kb;
    float2* C;
    int64_t c_batch_stride;
    int64_t c_ld;    // elements between consecutive output rows (0 = 2^nb)
    int* err;        // device error word (4 = a bounded wait gave up)
    int row_bytes;   // 32 or 64: bytes of K per tile row and stage (swizzle width)
    int group_m;     // tile rasterisation: row tiles per group (1 = row-major)
    uint32_t spin_limit;  // polls before a bounded wait gives up
    int test_stall;       // tests only: the producer issues no loads, so waits run out
    const int8_t* sexp_a;    // split FP16x2: the operands' scale exponents (SplitParams::sexp), else null
    const int8_t* sexp_b;
    int ksplit_bits;         // > 0: K is split over 2^ksplit_bits CTAs (grid y); each writes its FP32
    float2* partial;         //   partial tile to partial[(split * batch + z) * M * N + m * N + n]
    int accumulate;          // 1 (no K split): add the result into C instead of overwriting it
    int a_shared, b_shared;  // 1: the operand is the same for every batch entry; its planes and scale
                             //   exponents exist once (batch entry 0)
};

int tc_plane_count(int mode);
int tc_elem_bytes(int mode);
int tc_min_kb(int mode);
// split FP16x2: K chunks of 256 (one if K <= 256) that carry their own scale
int tc_scale_chunks(int kb);
cudaError_t launch_split(const SplitParams& p, int mode, int batch, cudaStream_t s);
cudaError_t launch_cgemm_tc(const TcGemmParams& p, int mode, const void* planesA, const void* planesB,
                            int batch, cudaStream_t s);
// C[z][m][n] (+)= sum over s < 2^ksplit_bits, in order, of partial[s][z][m][n] (an FP64 sum
// rounded once); C rows c_ld apart, batch entries c_batch_stride apart.
cudaError_t launch_ksplit_reduce(const float2* partial, int ksplit_bits, int batch, int mb, int nb, float2* C,
                                 int64_t c_batch_stride, int64_t c_ld, int accumulate, cudaStream_t s);

// Adjoint pass. Root environment seed: E_z[sum_j bit_j(r) ostride[j]] = grad[r].
struct SeedParams {
    const double2* grad;
    int obits;
    int64_t ostride[kMaxBits];
    float2* E;
    int64_t batch_stride;
};

// Fold per-slice environments of one leaf into its FP64 gradient: leaf mode
// q (most significant first) is either sliced (sl_bit[q] >= 0: the slice id
// bit fixing it) or found at env_stride[q] in the environment.
struct LeafEnvParams {
    const float2* env;
    int64_t env_batch_stride;
    int L;
    int sl_bit[kMaxBits];
    int64_t env_stride[kMaxBits];
    int64_t slice0;
    double2* grad;
};

cudaError_t launch_env_seed(const SeedParams& p, int batch, cudaStream_t s);
cudaError_t launch_leaf_env_accum(const LeafEnvParams& p, int batch, cudaStream_t s);
cudaError_t launch_accum_batch_f64(const float2* E, int64_t n, int batch, int64_t bs, double2* acc,
                                   cudaStream_t s);
cudaError_t launch_f64_to_f32(const double2* src, int64_t n, float2* dst, cudaStream_t s);
cudaError_t launch_param_grads(int n, const int64_t* env_off, const int64_t* d_off, const int64_t* size,
                               const float2* env, const float2* d, double2* out, cudaStream_t s);

// Fused stem group (secondary slicing, Sec. 5.2): n consecutive stem steps
// T_i = contract(T_{i-1}, B_i), each contracting nk <= 4 binary modes of the
// stem with a small branch tensor B_i and adding its nn <= 4 other modes. The
// stem modes that survive all n steps are the outer modes U: one CTA per
// assignment of U (and per slice of the batch) gathers the sub-tensor X_0 of
// T_0 over the remaining (inner) modes into shared memory, runs the n
// absorptions there and writes X_n into T_n. A step with nk == nn runs in
// place: new mode b takes the bit position of contracted mode b, so
// X_i[.. n ..] = sum_k X_{i-1}[.. k ..] B_i[k, n] over the same positions.
// Other steps lay X_i out as [kept modes of X_{i-1} | new modes] in a second
// buffer. n = 1 is the streaming kernel of a single narrow contraction.
constexpr int kStemMaxSteps = 32;
constexpr int kStemMaxInner = 14;  // inner binary modes of any X_i

struct StemStep {
    int nr, nk, nn;                 // kept, contracted, new binary modes
    int inplace;                    // nk == nn: new bit b takes the place of contracted bit b in X
    int rstr[kStemMaxInner];        // general step: X_{i-1} stride of kept bit b (least significant first)
    int kstr_x[4];                  // X_{i-1} stride of contracted bit b
    int ins[4];                     // in place: the contracted bits' positions in X, ascending
    int kstr_b[4], nstr_b[4];       // branch strides of contracted and new bits
    int b_off;                      // offset of the step's dense [K][N] branch copy in shared memory
    Operand br;                     // the branch tensor (sliced leaf or intermediate)
};

struct StemParams {
    Operand in;                     // T_0
    int n_in;                       // inner bits of X_0
    int64_t istr[kStemMaxInner];    // T_0 stride of X_0 bit b
    int nu;                         // outer bits
    int64_t ustr_in[kMaxBits], ustr_out[kMaxBits];  // strides of outer bit b in T_0 and T_n
    int n_out;                      // inner bits of X_n
    int64_t ostr[kStemMaxInner];    // T_n stride of X_n bit b
    float2* out;                    // T_n
    int64_t out_batch_stride;
    int nsteps, b_total;            // steps; complex elements of all dense branch copies
    int two_buffers;                // 1 if some step is not in place
    StemStep steps[kStemMaxSteps];
};

// Launch fused stem groups: params is a device array of n groups; group g
// runs 2^nu[g] CTAs per slice (their maximum is max_outer_log2) with
// 2 * 2^cap_log2 + b_total complex elements of shared memory.
cudaError_t launch_stem_fused(const StemParams* d_params, const StemParams& host_params, int cap_log2,
                              int64_t slice0, int batch, cudaStream_t s);

// ------------------------------------------------- persistent executor
//
// One launch runs a whole slice batch (or many-network round): one CTA per
// SM pulls tasks from a device work list in list order. A task runs when the
// counters it waits on have reached zero; when it is done it decrements its
// own counter. The list is topologically ordered (a task only waits on tasks
// earlier in the list, which CTAs that are running have already taken), so
// the waits always end; they are bounded all the same and report
// TNC_E_TIMEOUT in the error word.
enum PersistTaskType {
    PT_GEMM = 0,   // one 64x64 FP32 tile (idx: GemmParams, item: tile)
    PT_SPLIT = 1,  // count split blocks from item on (idx: SplitParams)
    PT_TC = 2,     // one 128x128 tensor-core tile (idx: TcNode, item: tile + tiles * K split)
    PT_KRED = 3,   // K-split reduction of 16384 complex pairs from item * 16384 (idx: KredParams)
    PT_ROOT = 4,   // one chunk of a final contraction (idx: RootParams, item: chunk)
    PT_ACC = 5,    // ordered FP64 sum of a final contraction's chunk sums into the result (idx: AccParams)
    PT_SUM = 6,    // FP64 slice sum of a root tensor with more than 64 outputs (idx: SumTaskParams)
    PT_STALL = 7   // tests only: waits on a counter nothing signals
};

struct PersistTask {
    int type;
    int idx;        // parameter entry of the task's type
    int64_t item;   // tile, chunk or first block
    int z;          // batch entry
    int net;        // network (slice0 = rs0[net] when the launch has a table)
    int count;      // PT_SPLIT: blocks
    int wait[3];    // counters to wait for (-1: none)
    int signal;     // counter to decrement when done
    int signal2;    // a second one (-1: none): the task's tree level
};

// One tensor-core contraction of a work list: the launch parameters and the
// tensor maps of its planes (TMA reads them from global memory).
struct TcNode {
    CUtensorMap map_a, map_b;
    TcGemmParams p;
    int nbatch;     // batch entries (the K-split partials are [split][z][m][n])
};

struct KredParams {
    const float2* partial;
    int nsplit, batch, nb;
    int64_t mn2;            // float4 steps of two complex elements per batch entry
    float2* C;
    int64_t c_batch_stride, c_ld;
    int accumulate;
};

struct AccParams {
    const double2* partials;  // [count][R] in the root's order
    int count;
    PermParams pp;
    double2* out;
};

struct SumTaskParams {
    SumParams sp;
    int batch;
    double2* out;
};

struct PersistParams {
    const PersistTask* tasks;
    int ntasks;
    int* counters;
    int* ticket;
    int* err;
    const GemmParams* gemm;
    const SplitParams* split;
    const TcNode* tc;
    const KredParams* kred;
    const RootParams* root;
    const AccParams* acc;
    const SumTaskParams* sum;
    const int64_t* rs0;     // per network first slice of the batch (null: slice0)
    int64_t slice0;
    uint64_t wait_ns;       // bound of one dependency wait (0: 10 s)
    uint32_t spin_limit;    // bound of one tensor-core pipeline wait (0: default)
    // result of a single-network work list, given at launch (null: the
    // AccParams / SumTaskParams outputs recorded in the list)
    double2* out0;
    // optional profile (null: off): per task type t, prof[3t] global-timer ns
    // from the end of its dependency waits to the end of the task, summed over
    // CTAs, prof[3t + 1] tasks, prof[3t + 2] ns spent in its dependency waits
    unsigned long long* prof;
};
constexpr int kPersistProfWords = 3 * 8;

// Launch the persistent executor for mode (FP32 or a split mode) over p's
// work list; ticket and counters must hold 0 and the initial counts.
cudaError_t launch_persist(const PersistParams& p, int mode, cudaStream_t s);
// Fill a work-list tensor-core node (planes from launch_split layouts).
bool tc_make_node(TcNode* node, const TcGemmParams& p, int mode, const void* planesA, const void* planesB, int batch);
// Output tiles (x K splits) of a tensor-core contraction.
int64_t tc_node_tiles(const TcGemmParams& p);
// Split blocks of one batch entry; the split's pair-load flag is set.
int64_t tc_split_prepare(SplitParams& p);

// Message returned by tnc_last_error() on this thread.
void set_last_error(const std::string& msg);

cudaError_t launch_gemm_f32(const GemmParams& p, int batch, cudaStream_t s);
// 64x64 output tiles of one FP32 contraction of 2^mb x 2^nb outputs.
int64_t gemm_f32_tiles(int mb, int nb);
// Independent FP32 contractions in one launch; params and tile_off (n + 1
// prefix offsets of their tile counts) are device arrays.
cudaError_t launch_gemm_f32_group(const GemmParams* d_params, const int64_t* d_tile_off, int n,
                                  int64_t total_tiles, int64_t slice0, int batch, cudaStream_t s);
cudaError_t launch_root_partials(const RootParams& p, int batch, double2* partials, cudaStream_t s);
// Several networks per launch: node i of a grouped launch belongs to network
// net[i]; rs0[w] / rb[w] are network w's first slice and batch of the round.
cudaError_t launch_gemm_f32_group_multi(const GemmParams* d_params, const int64_t* d_tile_off, int n,
                                        int64_t total_tiles, const int* d_net, const int64_t* d_rs0,
                                        const int* d_rb, int max_batch, cudaStream_t s);
// Final reductions of n networks (FP64 partials, then ordered sums into outs).
cudaError_t launch_root_multi(const RootParams* d_roots, double2* const* d_partials, const int64_t* d_blk_off,
                              int n, int64_t total_blocks, const PermParams* d_perms, double2* const* d_outs,
                              const int64_t* d_rs0, const int* d_rb, int max_batch, cudaStream_t s);
cudaError_t launch_accumulate_partials(const double2* partials, int count, const PermParams& pp,
                                       double2* out, cudaStream_t s);
cudaError_t launch_slice_sum_f32(const SumParams& p, int batch, double2* out, cudaStream_t s);

}  // namespace tnc
