/*
 * tnc.h - C ABI of libtnc: sliced tensor-network contraction on GB300 (sm_103a).
 *
 * The library computes amplitudes of a tensor network (Sec. 2.1.1 of Liu et
 * al., "Lifetime-based Optimization for Simulating Quantum Circuits on a New
 * Sunway Supercomputer"): tensors are vertices, indices are edges, every index
 * joins at most two tensors, an index joining one tensor only is open and
 * survives into the result. A contraction tree fixes the order of pairwise
 * contractions; slicing fixes a set S of closed indices of dimension 2, giving
 * 2^|S| independent sub-contractions whose results are summed (Sec. 2.1.1,
 * Fig. 2). The host-side planner implements the paper's lifetime-based slice
 * finder (Algorithm 1) and simulated-annealing refiner (Algorithms 2-4).
 *
 * Conventions shared by every entry point:
 *  - Every call returns a tnc_status and never throws. On failure a message is
 *    available from tnc_last_error() (thread-local, valid until the next call
 *    on the same thread).
 *  - Complex numbers are interleaved (re, im). Host tensor data is complex64
 *    (2 floats per element), row-major over the tensor's index list: the last
 *    listed index varies fastest.
 *  - Index ids are integers in [0, n_indices); dimensions are powers of two.
 *  - The library copies every host input it is given; the caller keeps
 *    ownership of its buffers. Device buffers passed in (outputs, workspace)
 *    are owned by the caller and must stay valid until the stream work that
 *    uses them completes.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). All device
 *    work of a call is enqueued on it; calls return before it completes.
 *  - A network object is not thread-safe; use one per thread.
 */
#ifndef TNC_H
#define TNC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tnc_net* tnc_net_t;

typedef enum {
    TNC_OK = 0,
    TNC_E_INVALID = 1, /* malformed input: message says which argument   */
    TNC_E_OOM = 2,     /* device or host allocation failed               */
    TNC_E_CUDA = 3,    /* a CUDA runtime call failed                     */
    TNC_E_TIMEOUT = 4, /* a bounded device-side wait gave up             */
    TNC_E_STATE = 5    /* call out of order (e.g. contract before path)  */
} tnc_status;

/* Arithmetic used by the pairwise contractions. The slice sum and the final
 * amplitude reduction are always accumulated in FP64. In the split modes each
 * complex product takes four real products (Ar Br, Ai Bi, Ar Bi, Ai Br) on the
 * tcgen05 tensor cores, each over the listed part pairs, with FP32
 * accumulation. */
typedef enum {
    TNC_FP32 = 0,        /* complex64 on FP32 CUDA cores (4 real FMAs per complex MAC)     */
    TNC_SPLIT_TF32 = 1,  /* x = hi + lo in TF32, 3 part pairs, kind::tf32                  */
    TNC_SPLIT_BF16 = 2,  /* x = x0 + x1 + x2 in BF16, 6 part pairs, kind::f16              */
    TNC_SPLIT_BF16X2 = 3, /* x = x0 + x1 in BF16, 3 part pairs (cheaper, lower accuracy)   */
    TNC_SPLIT_FP16X2 = 4  /* 2^e x = x0 + x1 in FP16, 3 part pairs, kind::f16; e per row of A,
                             per column of B and per 256-wide chunk of K puts that chunk's
                             max |Re|, |Im| in [2^14, 2^15); undone exactly per chunk      */
} tnc_mode;

/* Build a network (Sec. 2.1.1: G = (V, E, w)).
 *  n_tensors       number of tensors (leaves), >= 1
 *  ranks[i]        number of indices of tensor i (0 allowed: a scalar)
 *  index_ids[i]    ranks[i] index ids of tensor i, in row-major order of its data
 *  n_indices       number of index ids; index_dims[e] = w(e), a power of two
 *  data_c64[i]     host pointer to 2 * prod(dims) floats of tensor i (copied)
 *  open_ids        the n_open indices that belong to exactly one tensor, in the
 *                  order of the result tensor (first = most significant)
 *  out             receives the handle; free it with tnc_destroy
 * Errors: TNC_E_INVALID if an index joins more than two tensors, repeats within
 * a tensor, has a non-power-of-two dimension, if an index on one tensor only is
 * not listed in open_ids (or vice versa), or if a tensor exceeds 2^31 elements.
 * No device memory is touched until the first contraction. */
tnc_status tnc_create_network(int n_tensors, const int* ranks,
                              const int64_t* const* index_ids, int64_t n_indices,
                              const int64_t* index_dims, const float* const* data_c64,
                              int n_open, const int64_t* open_ids, tnc_net_t* out);

/* Replace the data of leaf `tensor` (same shape) from host memory; used for
 * gate-parameter updates. The host copy is updated at once; the device copy on
 * the next contraction. */
tnc_status tnc_set_tensor_data(tnc_net_t net, int tensor, const float* data_c64);

/* Leaf variants: batches of correlated amplitudes (Sec. 1 and Sec. 6.2, the
 * "1M correlated samples" workload), e.g. B closed bitstrings of one circuit.
 * The n leaves leaf_ids[i] (the projection vectors of the closed qubits) take
 * n_variants data copies each: data_c64[i] points to n_variants x (the leaf's
 * elements) interleaved complex64 values in host memory, copy v first-index
 * major, copied at once. Copy v of every listed leaf forms variant v; the
 * other leaves are common to all variants. Variant v's slice s has slice id
 * v * 2^|S| + s, so tnc_contract over [v 2^|S| + lo, v 2^|S| + hi) contracts
 * variant v, and every subtree without a variant leaf (and without a sliced
 * index) is slice-invariant: computed once and shared by all variants. Up to
 * 2^24 variants; |S| plus ceil(log2 n_variants) must stay within 62 bits and
 * a leaf's sliced modes plus variant bits within 16. n = 0 removes the
 * variants. The adjoint pass (tnc_contract_backward) takes no variants
 * (TNC_E_STATE). Errors: TNC_E_INVALID for a bad leaf, repeated leaf, NULL
 * data or count. */
tnc_status tnc_set_leaf_variants(tnc_net_t net, int n, const int* leaf_ids, int64_t n_variants,
                                 const float* const* data_c64);

/* Contract variants [v_lo, v_hi) (of tnc_set_leaf_variants), each over its
 * slices [lo, hi) of [0, 2^|S|), into out_c128 (device): (v_hi - v_lo) blocks
 * of 2^(open qubits) complex128 values, variant v_lo first, each overwritten.
 * The slice-invariant tensors are computed by the first variant and reused
 * by the others (unless "cache_invariants" is on and they are still valid
 * from an earlier call, every call computes them once; the option itself is
 * left as it was). Errors: TNC_E_STATE without variants; TNC_E_INVALID for a range out
 * of bounds; the errors of tnc_contract. */
tnc_status tnc_contract_variants(tnc_net_t net, int64_t v_lo, int64_t v_hi, int64_t lo, int64_t hi, int mode,
                                 double* out_c128, void* stream);

/* Bytes of all leaves packed back to back in leaf order (complex64). */
tnc_status tnc_leaf_bytes(tnc_net_t net, size_t* bytes);

/* Copy all leaves, packed as tnc_leaf_bytes describes, from host memory
 * (pinned memory lets the copy overlap) to the device copy, enqueued on
 * `stream`. The host buffer must stay valid until the copy completes. */
tnc_status tnc_upload_leaves(tnc_net_t net, const float* packed_c64, void* stream);

/* Greedy contraction path in SSA form (leaves 0..n-1, step i creates n+i):
 * rank-1/rank-2 tensors are first absorbed into their largest-rank neighbour
 * (the simplification of Sec. 2.1.2), then the connected pair minimising
 * size(out) - size(a) - size(b) is contracted (ties: smaller ids), then
 * disconnected remainders are joined in ascending id order.
 * pairs_out receives 2 * (n_tensors - 1) ints; pair entries are (smaller, larger). */
tnc_status tnc_greedy_path(tnc_net_t net, int* pairs_out);

/* Set the contraction tree B (Sec. 2.1.1, Fig. 1) as an SSA path of
 * n_steps = n_tensors - 1 pairs. Errors: TNC_E_INVALID if the pairs do not
 * form a binary tree over all leaves or an intermediate exceeds 2^120 elements.
 * Clears any slicing set. A contraction additionally requires every
 * intermediate to keep at most 2^36 elements once the sliced indices are
 * fixed (TNC_E_INVALID from tnc_contract otherwise). */
tnc_status tnc_set_path(tnc_net_t net, int n_steps, const int* pairs);

/* Lifetime-based in-place slicing (Sec. 4): Algorithm 1 (slice finder on the
 * stem) then Algorithm 2 (simulated-annealing refiner, with Algorithms 3/4),
 * minimising the Eq. 3 cost under the constraint that every tree tensor keeps
 * at most 2^target_log2 elements. T0, Tf, alpha: starting temperature, final
 * temperature and cooling factor (defaults 1.0, 1e-4, 0.9 if <= 0).
 * Writes up to `cap` sliced index ids to out_ids in insertion order and their
 * number to *n_out. Errors: TNC_E_INVALID if the target is infeasible (a tree
 * tensor has more than target_log2 bits of open indices) or cap is too small;
 * TNC_E_STATE before tnc_set_path. Does not change the network's slicing set. */
tnc_status tnc_find_slices(tnc_net_t net, int target_log2, uint64_t seed,
                           double T0, double Tf, double alpha,
                           int64_t* out_ids, int* n_out, int cap);

/* Set the slicing set S (Sec. 2.1.1): n <= 120 closed indices of dimension 2.
 * Slice s in [0, 2^n) assigns bit j of s to the j-th smallest id of S. Slice
 * ids are int64, so only slices [0, 2^min(n, 62)) are addressable; with n > 62
 * the indices beyond the 62nd smallest take value 0 in every addressable
 * slice (a fixed subset of slices is still a well-defined partial sum).
 * Errors: TNC_E_INVALID for an open index, a dimension other than 2, a
 * repeated id or n > 120; TNC_E_STATE before tnc_set_path. */
tnc_status tnc_set_slices(tnc_net_t net, int n, const int64_t* ids);

/* Device workspace needed to contract `max_batch` slices at once with the
 * current path and slicing set (max_batch >= 1). */
tnc_status tnc_workspace_bytes(tnc_net_t net, int64_t max_batch, size_t* bytes);

/* Give the library caller-owned device workspace (e.g. from PyTorch's
 * allocator). Contractions then batch as many slices as fit. If none is set,
 * the library allocates (and owns) the workspace for batch 1 itself. */
tnc_status tnc_set_workspace(tnc_net_t net, void* dev_ptr, size_t bytes);

/* Sum over slices s in [slice_lo, slice_hi) of the sliced contraction
 * (Sec. 2.1.1; the per-slice results are accumulated, the paper's final
 * allReduce becomes an on-device FP64 reduction in a fixed order).
 *  out_c128  device pointer, 2 * 2^(sum of log2 dims of open indices) doubles,
 *            overwritten with the result in open_ids order.
 * With leaf variants (tnc_set_leaf_variants) the slice ids run over
 * [0, 2^(|S| + ceil(log2 n_variants))): variant v's slices start at v 2^|S|.
 * Errors: TNC_E_STATE before tnc_set_path; TNC_E_INVALID if the range is not
 * within [0, 2^min(|S| + variant bits, 62)] or mode is unknown; TNC_E_CUDA /
 * TNC_E_OOM from the device. */
tnc_status tnc_contract(tnc_net_t net, int64_t slice_lo, int64_t slice_hi, int mode,
                        double* out_c128, void* stream);

/* Reverse-mode (adjoint) pass. For F = sum_o g_o O_o, with O the sum over
 * slices [slice_lo, slice_hi) of the sliced contraction and g = grad_out_c128
 * (device, complex128, in open_ids order), writes the holomorphic
 * environments dF/dL of every leaf L into grad_leaves_c64 (device,
 * complex64, all leaves packed back to back as tnc_leaf_bytes describes,
 * overwritten; leaves with leaf_mask[i] == 0 are left at zero, leaf_mask may
 * be NULL = all). For a pairwise contraction C = A (x) B (Sec. 2.1.1) the
 * environment of A is E_C contracted with B over B's free indices, and
 * likewise for B; environments of slice-invariant subtrees are summed over
 * the slices in FP64 and propagated once. The forward contractions use
 * `mode`; the environment contractions run in FP32 on CUDA cores, leaf
 * gradients accumulate in FP64. budget_bytes bounds the workspace (0 = 32
 * GiB); as many slices as fit are processed per pass, every intermediate of a
 * pass is kept for the reverse walk. Errors: TNC_E_OOM if one slice does not
 * fit the budget; as tnc_contract otherwise. PyTorch's complex gradient
 * convention (grad = dL/dRe + i dL/dIm) maps to g = conj(grad), and a real
 * parameter theta then gets dL/dtheta = Re(sum dF/dL * dL/dtheta). */
tnc_status tnc_contract_backward(tnc_net_t net, int64_t slice_lo, int64_t slice_hi, int mode,
                                 const double* grad_out_c128, float* grad_leaves_c64,
                                 const unsigned char* leaf_mask, size_t budget_bytes, void* stream);

/* Chain rule to gate parameters: out_c128[q] = sum_e env[leaf q][e] * dleaf_q[e]
 * in FP64, for n_params parameters whose leaf tensors are leaf_ids[q] (host
 * array). dleaf_c64 (device) holds the derivative tensors dL/dparam, one per
 * parameter, packed in order (each the size of its leaf); env_packed_c64 is
 * the packed output of tnc_contract_backward; out_c128 is device memory. */
tnc_status tnc_param_grads(tnc_net_t net, int n_params, const int* leaf_ids, const float* dleaf_c64,
                           const float* env_packed_c64, double* out_c128, void* stream);

/* Wait for `stream` and report device-side failures of the last
 * contraction: TNC_E_TIMEOUT if a bounded wait inside a tensor-core kernel
 * gave up (the kernel then drained its copies, freed its tensor memory and
 * returned; the result is invalid but the context stays usable). */
tnc_status tnc_check_device(tnc_net_t net, void* stream);

/* Contract n networks together (many circuits of uneven size): network i over
 * slices [slice_lo[i], slice_hi[i]) into outs_c128[i] (device, overwritten),
 * with the same result as n tnc_contract calls. The level groups of all
 * networks share launches (level L of every network in one grouped launch)
 * and the final reductions of all networks share two launches per round of
 * slice batches; tensor-core nodes keep their own launches. With use_graph
 * != 0 and a non-default stream, the launch sequence is captured once into a
 * CUDA graph and replayed by later calls with identical arguments (networks,
 * ranges, outputs, workspaces, plans and options; leaf data may change between
 * calls). When every network has the "persistent" option on and the
 * persistent executor can run each of them, every round of slice batches is
 * instead ONE launch of the work-list kernel holding all networks' tasks,
 * ordered by tree level (level L of every network before level L + 1 of any);
 * each network's tasks wait only on its own tasks ("persist_deps"). A dependency wait that runs out
 * is then reported through the first network's tnc_check_device.
 * Every network needs at most 64 outputs and at least two tensors. A network
 * may appear once. Destroying a network drops the cached sequences using it. */
tnc_status tnc_contract_many(int n, const tnc_net_t* nets, const int64_t* slice_lo, const int64_t* slice_hi,
                             int mode, double* const* outs_c128, int use_graph, void* stream);

/* JSON statistics of the current plan: Eq. 1 cost, Eq. 3 cost, Eq. 2
 * overhead, sliced ids, per-node (M, N, K) and kernel choice, workspace,
 * "stem_groups": [first node index, steps, outer bits, largest inner bits,
 * per slice, log2 elements of its input stem, log2 elements of its output]
 * of every fused stem group for the current options, and
 * "tc_cuts": per split mode, [node index, A row-panel bits, B row-panel bits,
 * K-panel bits, K-split bits] of every tensor-core-eligible contraction for
 * the last batch size ("tc_cut_batch"); "persistent" and "persist_deps" (the
 * options); "last_persist_deps": 1 if the last persistent tnc_contract ran
 * with per-entry dependencies; "last_workspace": [bytes of the reusing
 * layout, bytes without reuse (0 if not considered)] for the last
 * tnc_contract batch; "level_cost": per mode, [per-level launches,
 * estimated seconds] of that batch with the slice-invariant levels, the
 * input of the automatic executor choice; "timed_persist_tc_cmacs": the
 * complex multiply-accumulates that timed persistent launches (since
 * tnc_set_timing) ran on the tensor cores. */
tnc_status tnc_stats(tnc_net_t net, char* json, size_t cap);

/* The workspace plan of one batch of `batch` slices (1..1024) in `mode`, for
 * inspection: the first-fit simulation that tnc_contract sizes and places
 * its workspace with, tree level by level (slice-invariant levels first,
 * then per-slice ones, then the final contraction), with reuse = 1 as for
 * the per-level executor and the level chain, 0 without reuse (per-entry
 * dependencies). JSON: {"peak": bytes, "events": [[op (0 allocation,
 * 1 release), kind (0 tensor, 1 / 2 split planes of operand A / B, 3 final
 * contraction scratch), id (tensor id; for planes and scratch the
 * contraction's output tensor id), byte offset, bytes, level], ...]} in
 * simulation order. Host logic, no GPU. Errors: TNC_E_INVALID for a bad
 * argument or a too small json capacity; TNC_E_STATE before tnc_set_path. */
tnc_status tnc_arena_json(tnc_net_t net, int64_t batch, int mode, int reuse, char* json, size_t cap);

/* The persistent executor's work list for one batch of `batch` slices
 * (1..1024) in `mode`, slice-invariant contractions included, for
 * inspection: the tasks in launch order and the initial counter values. With
 * deps = 1 the list is built as for an arena without memory reuse
 * (per-entry dependencies), with 0 as for the reusing arena (level chain);
 * see the "persist_deps" option. JSON: {"chain": 0|1, "counters": [initial
 * value per counter], "tasks": [[type, parameter index, item, batch entry,
 * wait counter 0, 1, 2 (-1: none), counter signalled, second counter
 * signalled (-1: none), tree level, network (0)], ...]} with the task types of the
 * executor (0 FP32 tile, 1 split blocks, 2 tensor-core tile, 3 K-split
 * reduction, 4 final-contraction chunk, 5 ordered sum of the chunks, 6 slice
 * sum of a root tensor). A task may start once every counter it waits on is
 * zero; each task decrements the counters it signals once. Nothing runs and
 * no device memory is touched: the addresses in the list refer to a stand-in
 * workspace. Host logic; FP32 mode needs no GPU, the split modes need the
 * CUDA driver to encode the tensor maps of their contractions.
 * Errors: TNC_E_INVALID for a bad argument or a too small json capacity;
 * TNC_E_STATE before tnc_set_path, with fused stem groups in use, or when a
 * contraction cannot run in the executor (row or K panels). */
tnc_status tnc_worklist_json(tnc_net_t net, int64_t batch, int mode, int deps, char* json, size_t cap);

/* The merged work list of n networks (one batch of `batch` slices each) as
 * one persistent launch of tnc_contract_many runs it: every network's list
 * built as by tnc_worklist_json, its parameter indices and counters offset
 * past the earlier networks', then all tasks ordered by tree level (level L
 * of every network before level L + 1 of any). Same JSON, with an 11th entry
 * per task: the network's position in nets. Errors as tnc_worklist_json,
 * and TNC_E_INVALID for n < 1 or a network given twice. */
tnc_status tnc_worklist_many_json(int n, const tnc_net_t* nets, int64_t batch, int mode, int deps, char* json,
                                  size_t cap);

/* Tuning options of the tensor-core GEMM (no effect on results):
 *  "tc_row_bytes"  32 or 64 (default 64): bytes of K per tile row and
 *                  pipeline stage, also the shared-memory swizzle width
 *  "tc_group_m"    1..64 (default 1): output row tiles per rasterisation
 *                  group (consecutive CTAs sweep all column tiles of a group)
 *  "backward_keep_every" 0 (default) or 1..64: the adjoint pass keeps the
 *                  per-slice intermediates of every k-th dependency level (and
 *                  the root's inputs) and recomputes the others from them in
 *                  the reverse walk; 0 picks the smallest k whose workspace
 *                  fits the budget
 *  "tc_plane_cap_log2" 16..40 (default 32): split-precision operand planes of
 *                  one contraction are limited to 2^value bytes per operand;
 *                  larger operands are processed in panels: of K when K is
 *                  the largest dimension (each panel's launch adds into the
 *                  output), else of whole 128-row tiles (results unchanged up
 *                  to the order of the K sum; workspace smaller)
 *  "cache_invariants" 0 (default) or 1: keep the slice-invariant tensors that
 *                  feed per-slice contractions in the workspace between calls
 *                  and skip their recomputation while the plan, leaf data,
 *                  mode, batch, workspace and tuning are unchanged (the
 *                  workspace must not be used for anything else meanwhile)
 *  "stem_cap_log2" 0 or 2..13 (default 13): fused stem groups (Sec. 5.2,
 *                  secondary slicing). Consecutive narrow stem steps (a
 *                  stem of more than 2^value elements absorbing branches of
 *                  at most 16 contracted and 16 new elements) run as one
 *                  launch when every tensor of the sub-path, without the stem
 *                  modes that live through all of its steps, fits 2^value
 *                  elements: one CTA per assignment of those long-lived modes
 *                  keeps its sub-tensor in shared memory across the steps
 *                  (a group with a step whose contracted and new elements
 *                  differ holds two buffers and stays within 2^min(value, 12)
 *                  elements). A narrow step that starts no longer group runs
 *                  alone in the same kernel. 0 turns fusion off: every
 *                  contraction then runs on the GEMM kernels
 *                  (tnc_contract_many never fuses)
 *  "stem_min_outer_log2" 0..30 (default 7): a fused group needs at least
 *                  2^value sub-tensors (CTAs) per slice
 *  "stem_coalesce_bits" 0..6 (default 3): the lowest-stride modes of a
 *                  group's input and output stem that stay inner, so that
 *                  each CTA reads and writes runs of 2^value elements
 *  "persistent"    0, 1 or 2 (default 2): the executor. 1: the persistent
 *                  executor. A call whose contractions all fit it (no fused
 *                  stem group in use, no tensor-core contraction cut into row
 *                  or K panels) runs each batch of slices as ONE launch of a
 *                  work-list kernel
 *                  with one CTA per SM: the tasks (FP32 GEMM tiles, operand
 *                  split blocks, 128 x 128 tensor-core tiles, K-split
 *                  reductions, root chunks and sums) are taken in list order
 *                  from an atomic ticket and each waits, on device counters,
 *                  for the tasks that produce its inputs (see
 *                  "persist_deps"). Results equal the per-level launches' up to
 *                  the order of FP32 additions in a K split; other calls, and
 *                  0, use one launch per tree level. 2: the persistent
 *                  executor when the per-level launches of a batch would
 *                  carry less than 0.1 us of work each on average (a
 *                  contraction estimated at the larger of its flops at 300
 *                  TFLOP/s and its 8 (MK + KN + MN) bytes per slice at 6
 *                  TB/s: calls of tiny contractions only, where launch gaps
 *                  are all the time), else one launch per level
 *                  (for tnc_contract_many: over the whole call, unless every
 *                  network has 1)
 *  "persist_deps"  0 or 1 (default 1): with 1, a tnc_contract batch run by
 *                  the persistent executor gives every tensor and temporary
 *                  of the batch bytes of their own for the launch when that
 *                  fits (the caller's workspace, or an own one of at most the
 *                  larger of 1 GiB and the reusing layout's size), and a task
 *                  of batch entry z then waits only on entry z of what it
 *                  reads, so tree levels of different entries overlap. With
 *                  0, or when it does not fit, the workspace reuses the bytes
 *                  of dead tensors and every task also waits for the whole
 *                  previous tree level. tnc_workspace_bytes reports the
 *                  reusing layout; tnc_arena_json with reuse = 0 gives the
 *                  size per-entry dependencies need, and tnc_stats
 *                  "last_workspace" both sizes for the last call. tnc_contract_many does the same
 *                  per network, its own workspace capped at the larger of
 *                  256 MiB and the reusing layout.
 *  "persist_wait_ms" 0..600000 (default 0 = 10 s): bound of one dependency
 *                  wait of the persistent executor; a wait that runs out
 *                  stops every CTA and tnc_check_device reports TNC_E_TIMEOUT
 *  "persist_test_stall" tests only: nonzero adds a task that waits on a
 *                  counter no task decrements, so that bound runs out
 *  "tc_spin_limit" polls before a bounded device-side wait gives up (0 = the
 *                  kernel default, 2^24)
 *  "tc_test_stall" tests only: nonzero makes the tensor-core producer issue no
 *                  loads, so the consumers' bounded waits run out and the
 *                  contraction reports TNC_E_TIMEOUT through tnc_check_device
 * Errors: TNC_E_INVALID for an unknown key or value. */
tnc_status tnc_set_option(tnc_net_t net, const char* key, int64_t value);

/* Autotuner: for every contraction of the current plan that the tensor
 * cores can take in `mode`, time one slice (`slice`) with that contraction on
 * the tensor cores with the network's default row width ("tc_row_bytes"), on
 * the tensor cores with the other row width, and on the FP32 CUDA cores (one
 * warm-up run, then the median of three timed runs each). A variant replaces
 * the default only if it is at least 3% faster, so near-equal timings do not
 * flip the choice. The choice is recorded per (mode, log2 M, log2 N, log2 K)
 * in a table shared by all networks of the process (results are the same up
 * to rounding either way). Later contractions of any network follow the
 * table. A plan without a tensor-core-eligible contraction returns at once. */
tnc_status tnc_autotune(tnc_net_t net, int mode, int64_t slice, void* stream);

/* The tuning table as JSON: [[mode, log2 M, log2 N, log2 K, choice], ...]
 * with choice 0 = FP32 CUDA cores, 32 / 64 = tensor-core row width. */
tnc_status tnc_tune_table(char* json, size_t cap);

/* Per-launch timing: when enabled, every kernel launch of tnc_contract is
 * bracketed by CUDA events recorded on the contraction's stream. Each call
 * clears the records and the launch counter, which then accumulate over all
 * following contractions. */
tnc_status tnc_set_timing(tnc_net_t net, int enable);

/* Launch records since the last tnc_set_timing (waits for their events): per timed
 * launch the node's tensor id, kernel kind (0 FP32 GEMM, 1 FP64 root reduction,
 * 2 GEMM root + FP64 slice sum, 3 tensor-core GEMM, 4 operand split,
 * 7 reduction of a tensor-core GEMM's K-split partials, 8 fused stem group (node = its
 * output tensor), 9 persistent executor (node -1; one launch per slice batch), -1 leaf
 * slice sum), slice batch, complex multiply-accumulates of the
 * launch (all its nodes and slices) and milliseconds; a grouped launch of
 * several nodes of one tree level reports node -1. Any output array may be NULL. *n_out receives the number
 * of records (TNC_E_INVALID if it exceeds cap); *n_launches (may be NULL) the
 * number of kernels launched since then (counted with timing on or off). */
tnc_status tnc_last_timings(tnc_net_t net, int* node, int* kind, int* batch, double* cmacs,
                            float* ms, int cap, int* n_out, int64_t* n_launches);

/* Peak-rate probe for the roofline denominators (not part of the paper's
 * method): launches, on `stream`, one kernel that keeps one execution unit
 * busy and returns in *flops_out the floating-point operations it performs;
 * the caller times the launch (e.g. with CUDA events on the same stream).
 *  kind 0: FP32 FMA chains on the CUDA cores (2048 threads per SM; iters x 128
 *          FMAs per thread)
 *  kind 1: tcgen05.mma kind::tf32, 128 x 256 x 8 per instruction, one CTA per SM
 *  kind 2: tcgen05.mma kind::f16 with BF16 operands, 128 x 256 x 16
 *  kind 3: tcgen05.mma kind::f16 with FP16 operands, 128 x 256 x 16
 * For the MMA kinds iters is the number of instructions per SM (rounded up to
 * a multiple of 64). Errors: TNC_E_INVALID for an unknown kind or iters
 * outside [1, 2^30]; TNC_E_CUDA if the launch fails. */
tnc_status tnc_peak_probe(int kind, int64_t iters, double* flops_out, void* stream);

/* Capacity, in complex doubles, of the static scratch of tnc_reduce_pair_noalloc. */
#define TNC_NOALLOC_MAX_PARTIALS 65536

/* Allocation-free final contraction. The paper has no counterpart: this entry
 * point exists for callers that may not allocate device memory, e.g. a host
 * program whose device memory is entirely owned by another allocator (a
 * framework pool, a fixed per-process budget), or a latency-critical caller
 * that cannot afford the device-wide synchronisation of cudaMalloc/cudaFree.
 *
 * Computes out[m*N + n] = sum_k A[m*K + k] * B[k*N + n] with A row-major
 * M x K and B row-major K x N (complex64, interleaved, device pointers), M =
 * 2^m_log2, N = 2^n_log2, K = 2^k_log2, M*N <= 64, K <= 2^31. The products are
 * summed in FP64, per chunk of K and then over the chunks in a fixed order -
 * the same kernels as the final reduction of tnc_contract - and out_c128
 * (device, 2*M*N doubles) is overwritten.
 *
 * No memory is allocated or freed, by this library or by any library it
 * calls: the partial sums live in one static device array of
 * TNC_NOALLOC_MAX_PARTIALS complex doubles (1 MiB) that every GPU loading
 * libtnc holds until the process exits. The first call on a device looks up
 * that array's device address (with the device current) and caches it; make
 * that first call before any stream capture. With CUDA's lazy module loading
 * that first call is also when the driver loads this library's device code
 * and the array onto the device, which the driver may back with device memory
 * of its own; a caller that must not see any device allocation after set-up
 * makes one call (e.g. with K = 1) during its own set-up. The cached address
 * belongs to the device's primary context (the one the CUDA runtime uses): it
 * is not valid in another driver context, nor after cudaDeviceReset. Every call on a device shares
 * the array, so calls whose work overlaps on the GPU (e.g. on two streams)
 * race; serialise them. Partial sums are fully rewritten by each call before
 * they are read. Errors: TNC_E_INVALID for NULL pointers or sizes beyond the
 * limits above (the number of partial sums, min(max(K/1024,1),1024) * M * N,
 * must fit the array); TNC_E_CUDA if the lookup or a launch fails. */
tnc_status tnc_reduce_pair_noalloc(const float* a_c64, const float* b_c64, int m_log2, int n_log2,
                                   int k_log2, double* out_c128, void* stream);

const char* tnc_last_error(void);
void tnc_destroy(tnc_net_t net);

#ifdef __cplusplus
}
#endif

#endif /* TNC_H */
