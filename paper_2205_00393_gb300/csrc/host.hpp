// Internal declarations of the host side of libtnc: the plan, the workspace
// arena, the level groups, the network handle and the functions that the
// planning and launch code (host_plan.cpp), the persistent executor
// (host_persist.cpp), the adjoint pass (host_backward.cpp), the many-network
// path (host_many.cpp) and the C ABI (tnc_api.cpp) share. Not installed.
#pragma once

#include "tnc.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <set>
#include <iomanip>
#include <sstream>
#include <string>
#include <vector>

#include "kernels.h"
#include "planner.hpp"

namespace tnc_host {

inline thread_local std::string g_err;

inline tnc_status fail(tnc_status st, const std::string& msg) {
    g_err = msg;
    return st;
}

#define CUDA_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess)                                                           \
            return fail(_e == cudaErrorMemoryAllocation ? TNC_E_OOM : TNC_E_CUDA,        \
                        std::string(#expr) + ": " + cudaGetErrorString(_e));             \
    } while (0)

constexpr int64_t kAlign = 256;

inline int64_t align_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Kernel chosen for a contraction node.
enum NodeKind {
    K_GEMM_F32 = 0, K_ROOT_F64 = 1, K_GEMM_ROOT_SUM = 2, K_TC = 3, K_SPLIT = 4, K_KRED = 7, K_STEM = 8, K_PERSIST = 9
};

// Tensor-core eligibility of a non-root node in a split mode: both output
// sides span whole 128-wide tiles and K spans whole 64-wide k-blocks.
inline bool tc_node(int mode, int mb, int nb, int kb, bool is_root) {
    return mode != TNC_FP32 && !is_root && mb >= 7 && nb >= 7 && kb >= tnc::tc_min_kb(mode);
}

// Autotuned kernel choice per (mode, log2 M, log2 N, log2 K): 0 = FP32 CUDA
// cores, 32 / 64 = tensor cores with that row width. Filled by
// tnc_autotune; shared by every network of the process.
inline std::map<std::tuple<int, int, int, int>, int>& tune_table() {
    static std::map<std::tuple<int, int, int, int>, int> t;
    return t;
}
inline uint64_t g_tune_version = 0;

struct NodePlan {
    int v = 0;            // tensor id produced
    int A = 0, B = 0;     // operand tensor ids
    int mb = 0, nb = 0, kb = 0;
    std::vector<int64_t> am, ak, bk, bn;
    std::vector<int> mm, km, nm;  // m, k, n binary modes, most significant first
    bool per_slice = true;
    bool is_root = false;
    int kind = K_GEMM_F32;
    int chunks = 1;       // root reduction chunks
};

// A fused stem group (secondary slicing, Sec. 5.2): consecutive narrow stem
// steps whose intermediates never leave shared memory (see kernels.h).
struct StemGroupPlan {
    std::vector<int> steps;   // indices into Plan::nodes, in order
    int in = -1, out = -1;    // tensor ids of T_0 and T_n
    std::vector<int> U;       // outer modes: live through every step of the group
    int max_inner = 0;        // largest inner bit count of any X_i
    bool per_slice = false;
};

struct Plan {
    bool valid = false;
    uint64_t version = 0;                                   // distinguishes rebuilt plans
    std::vector<int> slice_bit_of_mode;                     // by mode, -1 if not sliced
    std::vector<std::vector<int>> layout;                   // effective modes per tensor
    std::vector<std::vector<std::pair<int, int64_t>>> str;  // (mode, stride) per tensor
    std::vector<std::vector<std::pair<int, int64_t>>> sl;   // leaves: (slice bit, stride)
    std::vector<char> per_slice;
    std::vector<NodePlan> nodes;                            // SSA order
    std::vector<int64_t> out_stride;                        // result-order bit j -> root offset
    int obits = 0;
    // fused stem groups for the cap they were planned with (stem_cap = -1: not planned)
    int stem_cap = -1;
    std::vector<StemGroupPlan> stems;
    std::vector<int> stem_of;        // per node index: its group, or -1
};

struct Arena {
    std::vector<int64_t> off;      // byte offset per tensor (-1 = none)
    std::vector<int64_t> planes_a, planes_b;  // per node (tensor-core split planes)
    int64_t root_scratch_off = -1; // FP64 partials or FP32 per-slice root
    int64_t peak = 0;
    int64_t batch = 1;             // slices per batch the per-slice temporaries are sized for
    bool reuse = true;             // memory of dead tensors reused by later levels
};

// Level groups: nodes whose inputs are ready at the same time run in one
// launch. Invariant nodes are levelled over the invariant forest, per-slice
// nodes over per-slice dependencies; the root runs last on its own.
struct Group {
    bool per_slice = false;
    std::vector<int> fp32;   // node tensor ids run by one grouped FP32 launch
    std::vector<int> tc;     // nodes launched one by one: tensor-core nodes and large FP32 nodes
    std::vector<int> stems;  // fused stem groups ending at this level (Plan::stems indices)
    int first = 0;           // first entry of the group's parameters in the table
    int off_first = 0;       // first entry of its n + 1 tile offsets
    int64_t tiles = 0;
    double cmacs = 0.0;      // per slice
};

struct GroupPlan {
    std::vector<Group> inv, ps;
    std::vector<tnc::GemmParams> params;
    std::vector<int64_t> tile_off;
    std::vector<tnc::StemParams> stem_params;  // per Plan::stems entry (device copy in d_stem)
};

// Device copy of a work list: one allocation holding the tables, the initial
// counters, the counters themselves and the ticket.
struct DeviceWorkList {
    void* mem = nullptr;
    tnc::PersistParams prm{};
    int* init = nullptr;
    size_t n_counters = 0;
    double cmacs = 0.0;     // complex multiply-accumulates of one launch
    double tc_cmacs = 0.0;  // the part of them on the tensor cores
    bool tensor_tasks = false;  // any split, tensor-core tile or K-split task (else the FP32 variant runs it)
    ~DeviceWorkList() {
        if (mem) cudaFree(mem);
    }
};

inline int64_t stride_of(const std::vector<std::pair<int, int64_t>>& s, int mode) {
    for (auto& p : s)
        if (p.first == mode) return p.second;
    return -1;
}

}  // namespace tnc_host

using namespace tnc_host;


struct tnc_net {
    uint64_t uid = 0;               // process-unique id (cache keys)
    // network
    int n_leaves = 0;
    std::vector<std::vector<int64_t>> leaf_idx;
    std::vector<int> logd;          // by index id (0 for ids not present)
    std::vector<char> present;
    std::vector<int64_t> open_ids;
    std::vector<int> mode_base;     // first binary mode of an index id
    std::vector<int64_t> leaf_off;  // element offsets in the packed leaf buffer
    std::vector<int64_t> leaf_elems;
    std::vector<float> host_leaves; // packed complex64
    int64_t total_leaf_elems = 0;
    // device
    float2* d_leaves = nullptr;
    // leaf variants (tnc_set_leaf_variants): stacked copies of some leaves,
    // copy v addressed by the slice-id bits above those of the sliced indices
    int variant_bits = 0;
    int64_t n_variants = 0;
    std::vector<int64_t> var_off;   // per leaf: element offset in the variant buffer, -1 for an ordinary leaf
    std::vector<float> host_var;    // interleaved complex64, [leaf][variant][elements]
    float2* d_var = nullptr;
    size_t d_var_elems = 0;
    bool var_dirty = false;
    int* d_err = nullptr;           // device error word of bounded waits
    bool dev_dirty = true;
    // path and slices
    std::vector<tnc::Pair> path;
    std::unique_ptr<tnc::Tree> tree;
    std::vector<int64_t> S;         // as given
    std::vector<int64_t> S_sorted;
    Plan plan;
    // workspace
    void* ws_user = nullptr;
    size_t ws_user_bytes = 0;
    void* ws_own = nullptr;
    size_t ws_own_bytes = 0;
    int64_t last_batch = 0;
    int last_keep_every = 1;        // checkpoint spacing of the last backward pass
    size_t last_backward_bytes = 0;
    // tensor-core tile options (tnc_set_option)
    int tc_row_bytes = 64;
    int tc_group_m = 1;
    uint32_t tc_spin_limit = 0;  // 0 = kernel default
    int backward_keep_every = 0; // 0 = smallest spacing that fits the budget
    int plane_cap_log2 = 32;     // split-precision planes per operand <= 2^this bytes
    int force_choice = -1;       // autotuning: force 0 (FP32) or a tensor-core row width
    int stem_cap_log2 = 13;      // fused stem groups: inner sub-tensors up to 2^this elements (0 = off)
    int stem_min_outer = 7;      // fused stem groups: at least 2^this sub-tensors (CTAs) per slice
    int stem_coalesce_bits = 3;  // fused stem groups: lowest-stride modes of T_0 and T_n kept inner
    bool in_many = false;        // building a many-network call: no fused stem groups
    tnc::StemParams* d_stem = nullptr;
    size_t d_stem_cap = 0;
    bool cache_invariants = false;  // keep slice-invariant inputs of per-slice nodes across calls
    std::string inv_key;            // state under which the cached invariants were computed
    uint64_t leaf_version = 0;      // bumped whenever leaf data changes
    bool tuning = false;         // autotuning: every eligible node gets its own launch
    int tc_test_stall = 0;
    // cached level groups and their device parameter table
    std::string group_key;
    GroupPlan groups;
    tnc::GemmParams* d_params = nullptr;
    int64_t* d_tile_off = nullptr;
    size_t d_params_cap = 0, d_tile_cap = 0;
    int64_t* d_pg = nullptr;  // parameter-gradient offsets
    size_t pg_cap = 0;
    // per-launch timing (tnc_set_timing) and launch accounting
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    struct TimedLaunch { int node; int kind; int batch; double cmacs; size_t ev; };
    std::vector<TimedLaunch> timed;
    int64_t launches = 0;
    // persistent executor (one launch per slice batch); its device work lists by key
    int persistent = 2;  // 0 per-level launches, 1 persistent kernel, 2 automatic choice
    uint64_t persist_wait_ns = 0;    // bound of one dependency wait (0: 10 s)
    int persist_test_stall = 0;      // tests only: one task waits on a counter nothing signals
    int persist_deps = 1;            // per-slice node dependencies (no level chain) when their arena fits
    bool last_persist_deps = false;  // whether the last persistent call ran with them
    size_t last_arena_bytes[2] = {0, 0};  // last tnc_contract batch: reusing arena, arena without reuse (0: not needed)
    mutable std::map<std::string, Arena> arena_cache;  // plan_arena results by their inputs
    std::map<std::string, std::pair<double, double>> cost_cache;  // level_cost results (launches, seconds)
    std::map<std::string, std::unique_ptr<DeviceWorkList>> worklists;
    double timed_persist_tc_cmacs = 0.0;  // tensor-core share of the timed persistent launches
    unsigned long long* d_prof = nullptr;  // "persist_profile": per task type time, count, wait

    ~tnc_net() {
        if (d_leaves) cudaFree(d_leaves);
        if (d_err) cudaFree(d_err);
        if (d_params) cudaFree(d_params);
        if (d_tile_off) cudaFree(d_tile_off);
        if (d_pg) cudaFree(d_pg);
        if (d_stem) cudaFree(d_stem);
        if (ws_own) cudaFree(ws_own);
        if (d_prof) cudaFree(d_prof);
        if (d_var) cudaFree(d_var);
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    }
};


namespace tnc_host {

// How one tensor-core contraction is cut up:
//  - planes of one operand are capped (tc_plane_cap_log2): when K is the
//    largest dimension the contraction runs as 2^pK sequential K panels (each
//    launch keeps every output tile and adds into C after the first);
//    otherwise the top row bits of A (pA) and of B (pB) are fixed in panels;
//  - with fewer than four waves of output tiles (152 SMs), K is also split
//    across 2^ks CTAs of one launch (at least 4096 K per split) whose FP32
//    partials a reduction adds in a fixed order.
// The workspace holds, per operand, the planes of one panel (plus the split
// FP16x2 scale words), and for A also the partials of one launch.
struct TcCut {
    int pA = 0, pB = 0, pK = 0, ks = 0;
    int64_t a_bytes = 0, b_bytes = 0, partial_off = 0;
};

struct WorkList {
    std::vector<tnc::PersistTask> tasks;
    std::vector<int> counters;
    std::vector<tnc::GemmParams> gemm;
    std::vector<tnc::SplitParams> split;
    std::vector<tnc::TcNode> tc;
    std::vector<tnc::KredParams> kred;
    std::vector<tnc::RootParams> root;
    std::vector<tnc::AccParams> acc;
    std::vector<tnc::SumTaskParams> sum;
    double cmacs = 0.0, tc_cmacs = 0.0;
    int new_counter(int count) {
        counters.push_back(count);
        return (int)counters.size() - 1;
    }
    // tree-level chain of the network being emitted: tasks wait on the
    // previous level's counter and also count down the current level's;
    // level[i] is task i's level number within its network. Without the chain
    // (chain false: an arena without reuse, every tensor written once per
    // launch) tasks wait only on the counters of their own inputs.
    bool chain = true;
    int lvl_prev = -1, lvl_cur = -1, lvl_no = -1;
    std::vector<int> level;
    bool no_slot = false;  // a task had no wait slot left for the level chain
    void task(int type, int idx, int64_t item, int z, int net, int count, int w0, int w1, int w2, int signal) {
        tnc::PersistTask t{};
        t.type = type;
        t.idx = idx;
        t.item = item;
        t.z = z;
        t.net = net;
        t.count = count;
        t.wait[0] = w0;
        t.wait[1] = w1;
        t.wait[2] = w2;
        t.signal = signal;
        t.signal2 = chain ? lvl_cur : -1;
        // a slot left free takes the previous level (a task of a level waits
        // for the whole level before it: the workspace reuses memory across levels)
        if (chain && lvl_prev >= 0) {
            bool have = false;
            for (int q = 0; q < 3; ++q) have |= t.wait[q] == lvl_prev;
            for (int q = 0; q < 3 && !have; ++q)
                if (t.wait[q] < 0) {
                    t.wait[q] = lvl_prev;
                    have = true;
                }
            no_slot |= !have;
        }
        if (chain && lvl_cur >= 0) ++counters[lvl_cur];
        tasks.push_back(t);
        level.push_back(lvl_no);
    }
    void begin_level() {
        ++lvl_no;
        if (!chain) return;
        lvl_prev = lvl_cur;
        lvl_cur = new_counter(0);
    }
};

// The automatic executor choice: the persistent kernel when the per-level
// launches would carry less than 0.1 us of estimated work each on average.
// The estimate is nominal (peak rates); measured on GB300, the persistent
// kernel is ahead on calls whose every contraction is tiny (1.3-1.8x at
// 12-16 qubits, estimates of at most 0.03 us per launch), within about 10% of
// the per-level launches near 0.1 us, and 6-35% behind from 0.4 us up:
// there, each launch already runs for tens of microseconds and the
// one-CTA-per-SM tasks do the same work less efficiently than the separate
// kernels.
constexpr double kPersistAutoSecondsPerLaunch = 0.1e-6;

// planning, arena, level groups and launches (host_plan.cpp)
int net_plane_cap_log2(const tnc_net* net);
int shape_choice(const tnc_net* net, int mode, int mb, int nb, int kb, bool is_root);
void build_plan(tnc_net* net);
int64_t tensor_bytes(const Plan& P, int v);
bool stem_fusion(const tnc_net* net);
bool stem_step(const tnc_net* net, const NodePlan& np);
void plan_stems(tnc_net* net);
int64_t plane_data_bytes(int mode, int rb, int kb, int64_t batch);
int64_t full_planes_bytes(int mode, int rb, int kb, int64_t batch);
TcCut tc_cut(const tnc_net* net, int mode, int mb, int nb, int kb, int64_t batch);
int64_t tc_bytes_a(const tnc_net* net, int mode, int mb, int nb, int kb, int64_t batch);
int64_t tc_bytes_b(const tnc_net* net, int mode, int mb, int nb, int kb, int64_t batch);
Arena plan_arena(const tnc_net* net, int64_t nb, int mode, bool reuse = true);
// One allocation (op 0) or release (op 1) of plan_arena's simulation: kind 0
// a tensor (id: its tensor id), 1 / 2 the split planes of A / B of contraction
// id, 3 the final contraction's scratch; step: the level being simulated.
struct ArenaEvent {
    int op, kind, id;
    int64_t off, len;
    int step;
};
Arena plan_arena_log(const tnc_net* net, int64_t nb, int mode, bool reuse, std::vector<ArenaEvent>* log);
std::string group_key_of(const tnc_net* net, int mode, int64_t nb, const char* ws, bool reuse);
std::string plan_key(const tnc_net* net, int mode, int64_t nb);
int64_t cut_batch(const Arena& ar, const NodePlan& np, int64_t b);
tnc::Operand operand(const tnc_net* net, const Arena& ar, char* ws, int v, int64_t nb);
tnc::GemmParams gemm_params(const tnc_net* net, const Arena& ar, char* ws, const NodePlan& np, int64_t nb);
tnc_status ensure_plan(tnc_net* net);
tnc::StemParams stem_params(const tnc_net* net, const Arena& ar, char* ws, int gi, int64_t nb);
tnc_status ensure_leaves(tnc_net* net, cudaStream_t st);
int64_t slice_space(const tnc_net* net);
double node_cmacs(const tnc_net* net, int node);
cudaError_t timed_begin(tnc_net* net, int node, int kind, int batch, cudaStream_t s, double cmacs = -1.0);
cudaError_t timed_end(tnc_net* net, cudaStream_t s);
int64_t pick_batch(const tnc_net* net, int64_t want, size_t budget, int mode);
std::vector<Group> level_groups(const tnc_net* net, int mode, bool per_slice);
tnc_status ensure_groups(tnc_net* net, const Arena& ar, char* ws, int mode, int64_t nb, cudaStream_t s);
tnc_status launch_tc_contraction(tnc_net* net, const tnc::GemmParams& g, int b, int mode, void* pa, void* pb, int node, cudaStream_t s, int row_bytes, int64_t cut_b);
tnc_status launch_node(tnc_net* net, const Arena& ar, char* ws, const NodePlan& np, const tnc::GemmParams& g, int b, int mode, cudaStream_t s);
tnc_status run_group(tnc_net* net, const Arena& ar, char* ws, const Group& g, int b, int64_t slice0, int mode, cudaStream_t s);

// persistent executor (host_persist.cpp)
bool persist_eligible(tnc_net* net);
void level_cost(tnc_net* net, int mode, int64_t b, bool with_inv, double* launches, double* seconds);
bool wl_network(tnc_net* net, const Arena& ar, char* ws, int b, int mode, bool with_inv, int netidx, double* out, WorkList& W);
void wl_append(WorkList& W, const WorkList& Wi);
void wl_interleave_levels(WorkList& W);
tnc_status wl_upload(const WorkList& W, DeviceWorkList& D, int* err, uint64_t wait_ns, uint32_t spin, cudaStream_t s);
cudaError_t wl_launch(const DeviceWorkList& D, int mode, int64_t slice0, const int64_t* rs0, cudaStream_t s, unsigned long long* prof, double* out0);
bool wl_validate(const tnc_net* net, const WorkList& W, const char* ws, size_t ws_bytes, const double* out, int mode, std::string* why);
DeviceWorkList* contract_worklist(tnc_net* net, const Arena& ar, char* ws, int b, int mode, bool with_inv, double* out, cudaStream_t s, tnc_status* st);

// many-network calls (host_many.cpp)
void many_forget(uint64_t uid);

}  // namespace tnc_host
