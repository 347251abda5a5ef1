// C ABI of libtnc (declared in include/tnc.h) and the host-side executor.
//
// Execution of tnc_contract over slices [lo, hi) (Sec. 2.1.1: slicing turns
// the contraction into 2^|S| independent subtasks whose results are summed):
//  1. Contraction nodes whose subtree holds no sliced index give the same
//     tensor in every slice (Sec. 3.1: only tensors on a sliced index's
//     lifetime change); they run once per call, batch 1.
//  2. The remaining nodes run for a batch of consecutive slices per launch
//     (grid z = slice within the batch), in SSA order.
//  3. The root contraction reduces in FP64 and is accumulated into the
//     caller's complex128 result in a fixed order.
// Intermediates live in one workspace arena whose offsets are planned on the
// host by a first-fit simulation of the tensors' lifetimes.
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

namespace {

thread_local std::string g_err;

tnc_status fail(tnc_status st, const std::string& msg) {
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

int64_t align_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Kernel chosen for a contraction node.
enum NodeKind {
    K_GEMM_F32 = 0, K_ROOT_F64 = 1, K_GEMM_ROOT_SUM = 2, K_TC = 3, K_SPLIT = 4, K_KRED = 7, K_STEM = 8, K_PERSIST = 9
};

// Tensor-core eligibility of a non-root node in a split mode: both output
// sides span whole 128-wide tiles and K spans whole 64-wide k-blocks.
bool tc_node(int mode, int mb, int nb, int kb, bool is_root) {
    return mode != TNC_FP32 && !is_root && mb >= 7 && nb >= 7 && kb >= tnc::tc_min_kb(mode);
}

// Autotuned kernel choice per (mode, log2 M, log2 N, log2 K): 0 = FP32 CUDA
// cores, 32 / 64 = tensor cores with that row width. Filled by
// tnc_autotune; shared by every network of the process.
std::map<std::tuple<int, int, int, int>, int>& tune_table() {
    static std::map<std::tuple<int, int, int, int>, int> t;
    return t;
}
uint64_t g_tune_version = 0;

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
    ~DeviceWorkList() {
        if (mem) cudaFree(mem);
    }
};

int64_t stride_of(const std::vector<std::pair<int, int64_t>>& s, int mode) {
    for (auto& p : s)
        if (p.first == mode) return p.second;
    return -1;
}

}  // namespace

void tnc::set_last_error(const std::string& msg) { g_err = msg; }

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

namespace {

int net_plane_cap_log2(const tnc_net* net) { return net->plane_cap_log2; }

// Kernel for a contraction of this shape: 0 = FP32 CUDA cores, otherwise the
// tensor-core row width. Eligibility first, then a forced choice (autotuning
// runs), then the tuning table, then the network's default row width.
int shape_choice(const tnc_net* net, int mode, int mb, int nb, int kb, bool is_root) {
    if (!tc_node(mode, mb, nb, kb, is_root)) return 0;
    if (net->force_choice >= 0) return net->force_choice;
    auto it = tune_table().find(std::make_tuple(mode, mb, nb, kb));
    if (it != tune_table().end()) return it->second;
    return net->tc_row_bytes;
}

// ------------------------------------------------------------- planning ----

void build_plan(tnc_net* net) {
    static uint64_t counter = 0;
    Plan& P = net->plan;
    P = Plan();
    P.version = ++counter;
    const tnc::Tree& T = *net->tree;
    const int nt = T.n_tensors();
    int total_modes = net->mode_base.empty() ? 0 : net->mode_base.back();
    P.slice_bit_of_mode.assign(total_modes, -1);
    for (size_t j = 0; j < net->S_sorted.size(); ++j)
        // slice ids are int64: sliced indices beyond the 62nd take value 0 in
        // every addressable slice (bit 62 of an id below 2^62 is always 0)
        P.slice_bit_of_mode[net->mode_base[net->S_sorted[j]]] = (int)std::min<size_t>(j, 62);
    P.layout.resize(nt);
    P.str.resize(nt);
    P.sl.resize(nt);
    P.per_slice.assign(nt, 0);
    auto modes_of = [&](int64_t e) {
        std::vector<int> m;
        for (int b = 0; b < net->logd[e]; ++b) m.push_back(net->mode_base[e] + b);
        return m;
    };
    for (int v = 0; v < net->n_leaves; ++v) {
        std::vector<int> full;
        for (int64_t e : net->leaf_idx[v])
            for (int m : modes_of(e)) full.push_back(m);
        const int L = (int)full.size();
        for (int p = 0; p < L; ++p) {
            int64_t st = 1ll << (L - 1 - p);
            int sb = P.slice_bit_of_mode[full[p]];
            if (sb >= 0) {
                P.sl[v].emplace_back(sb, st);
                P.per_slice[v] = 1;
            } else {
                P.layout[v].push_back(full[p]);
                P.str[v].emplace_back(full[p], st);
            }
        }
        if (!net->var_off.empty() && net->var_off[v] >= 0) {
            // a variant leaf: copy number = slice-id bits [|S|, |S| + variant_bits)
            const int base = (int)net->S_sorted.size();
            if (base + net->variant_bits > 62)
                throw tnc::PlanError("sliced indices and variant bits exceed 62 slice-id bits");
            for (int j = 0; j < net->variant_bits; ++j) P.sl[v].emplace_back(base + j, net->leaf_elems[v] << j);
            P.per_slice[v] = 1;
        }
        if ((int)P.sl[v].size() > tnc::kMaxSliceBits)
            throw tnc::PlanError("leaf " + std::to_string(v) + " has more than 16 sliced modes and variant bits");
    }
    for (size_t i = 0; i < T.children.size(); ++i) {
        const int v = net->n_leaves + (int)i;
        int c0 = T.children[i].first, c1 = T.children[i].second;
        std::set<int> s0(P.layout[c0].begin(), P.layout[c0].end());
        std::set<int> s1(P.layout[c1].begin(), P.layout[c1].end());
        std::vector<int> f0, f1;
        for (int m : P.layout[c0])
            if (!s1.count(m)) f0.push_back(m);
        for (int m : P.layout[c1])
            if (!s0.count(m)) f1.push_back(m);
        NodePlan np;
        np.v = v;
        np.A = c0;
        np.B = c1;
        if (f1.size() > f0.size()) {
            std::swap(np.A, np.B);
            std::swap(f0, f1);
        }
        const std::set<int>& sB = (np.B == c1) ? s1 : s0;
        std::vector<int> kmodes;
        for (int m : P.layout[np.A])
            if (sB.count(m)) kmodes.push_back(m);
        np.mb = (int)f0.size();
        np.nb = (int)f1.size();
        np.kb = (int)kmodes.size();
        if (np.mb > tnc::kMaxBits || np.nb > tnc::kMaxBits || np.kb > tnc::kMaxBits)
            throw tnc::PlanError("contraction node " + std::to_string(i) + " exceeds 40 modes per side");
        for (int j = 0; j < np.mb; ++j) np.am.push_back(stride_of(P.str[np.A], f0[np.mb - 1 - j]));
        for (int j = 0; j < np.kb; ++j) {
            np.ak.push_back(stride_of(P.str[np.A], kmodes[np.kb - 1 - j]));
            np.bk.push_back(stride_of(P.str[np.B], kmodes[np.kb - 1 - j]));
        }
        for (int j = 0; j < np.nb; ++j) np.bn.push_back(stride_of(P.str[np.B], f1[np.nb - 1 - j]));
        np.mm = f0;
        np.km = kmodes;
        np.nm = f1;
        std::vector<int> out(f0);
        out.insert(out.end(), f1.begin(), f1.end());
        const int L = (int)out.size();
        if (L > 36)
            throw tnc::PlanError("intermediate " + std::to_string(v) + " keeps 2^" + std::to_string(L) +
                                 " elements after slicing; slice more indices");
        for (int p = 0; p < L; ++p) P.str[v].emplace_back(out[p], 1ll << (L - 1 - p));
        P.layout[v] = out;
        P.per_slice[v] = P.per_slice[c0] || P.per_slice[c1];
        np.is_root = (v == T.root);
        np.per_slice = P.per_slice[v] || np.is_root;
        if (np.is_root) {
            if (np.mb + np.nb <= 6) {
                np.kind = K_ROOT_F64;
                int64_t K = 1ll << np.kb;
                int64_t ch = K / 1024;
                if (ch < 1) ch = 1;
                if (ch > 1024) ch = 1024;
                np.chunks = (int)ch;
            } else {
                np.kind = K_GEMM_ROOT_SUM;
            }
        } else {
            np.kind = K_GEMM_F32;
        }
        P.nodes.push_back(np);
    }
    // result order: open_ids, each expanded MSB first; bit j counts from the last mode
    const int root = T.root;
    std::vector<int> omodes;
    for (int64_t e : net->open_ids)
        for (int m : modes_of(e)) omodes.push_back(m);
    P.obits = (int)omodes.size();
    if (P.obits > tnc::kMaxBits) throw tnc::PlanError("more than 40 open modes");
    for (int j = 0; j < P.obits; ++j) {
        int64_t st = stride_of(P.str[root], omodes[P.obits - 1 - j]);
        if (st < 0) throw tnc::PlanError("open mode missing from the result");
        P.out_stride.push_back(st);
    }
    P.valid = true;
}

int64_t tensor_bytes(const Plan& P, int v) { return (int64_t)8 << P.layout[v].size(); }

// ------------------------------------------------------ fused stem groups ----
//
// Secondary slicing (Sec. 5.2): along a chain of narrow stem steps (a big
// intermediate absorbing small branch tensors one after another), the modes of
// the stem that live through n consecutive steps are sliced for the GPU's
// shared memory (one CTA per assignment) and the other (inner) modes are
// carried through the n steps on chip. Following the paper, a group starts at
// a step and grows while every tensor of the sub-path, restricted to its
// inner modes, fits 2^cap elements; groups of at least two steps run fused.

bool stem_fusion(const tnc_net* net) {
    return net->stem_cap_log2 > 0 && !net->in_many && !net->tuning && net->plan.stem_cap == net->stem_cap_log2;
}

// A narrow stem step: the bigger operand A is an intermediate larger than
// one on-chip sub-tensor (2^cap elements) and the branch B brings at most 4
// contracted and 4 new modes.
bool stem_step(const tnc_net* net, const NodePlan& np) {
    return !np.is_root && np.kb <= 4 && np.nb <= 4 && np.A >= net->n_leaves &&
           (int)net->plan.layout[np.A].size() > net->stem_cap_log2;
}

constexpr int kStemTwoBufferCap = 12;

void plan_stems(tnc_net* net) {
    Plan& P = net->plan;
    const int cap = std::min(net->stem_cap_log2, tnc::kStemMaxInner);
    P.stems.clear();
    P.stem_of.assign(P.nodes.size(), -1);
    P.stem_cap = net->stem_cap_log2;
    if (cap <= 0) return;
    const int nl = net->n_leaves;
    const int nn = (int)P.nodes.size();
    std::vector<int> next(nn, -1);
    std::vector<char> has_prev(nn, 0);
    for (int j = 0; j < nn; ++j) {
        const NodePlan& nj = P.nodes[j];
        if (!stem_step(net, nj)) continue;
        const int i = nj.A - nl;  // the node whose output is this step's stem operand
        if (i >= 0 && stem_step(net, P.nodes[i]) && P.nodes[i].per_slice == nj.per_slice) {
            next[i] = j;
            has_prev[j] = 1;
        }
    }
    auto pos_stride = [](const std::vector<int>& L, int m) -> int64_t {
        for (size_t q = 0; q < L.size(); ++q)
            if (L[q] == m) return (int64_t)1 << (L.size() - 1 - q);
        return -1;
    };
    // the group chain[i .. i + n): outer modes U and the largest inner size.
    // The stem_coalesce_bits lowest-stride modes of T_0 and of T_n stay inner
    // (they would otherwise interleave the CTAs' reads and writes), so each
    // CTA moves runs of at least 2^stem_coalesce_bits consecutive elements.
    const int cb = net->stem_coalesce_bits;
    auto eval = [&](const std::vector<int>& chain, size_t i, size_t n, StemGroupPlan& g) -> bool {
        const std::vector<int>& L0 = P.layout[P.nodes[chain[i]].A];
        const std::vector<int>& Ln = P.layout[P.nodes[chain[i + n - 1]].v];
        std::set<int> contracted;
        for (size_t j = i; j < i + n; ++j)
            for (int m : P.nodes[chain[j]].km) contracted.insert(m);
        std::vector<int> U;
        for (int m : L0) {
            const int64_t s0 = pos_stride(L0, m), sn = pos_stride(Ln, m);
            if (!contracted.count(m) && s0 >= ((int64_t)1 << cb) && sn >= ((int64_t)1 << cb)) U.push_back(m);
        }
        const std::set<int> Us(U.begin(), U.end());
        int mx = (int)L0.size() - (int)U.size();
        for (size_t j = i; j < i + n; ++j) {
            int inner = 0;
            for (int m : P.layout[P.nodes[chain[j]].v])
                if (!Us.count(m)) ++inner;
            mx = std::max(mx, inner);
        }
        // a step that is not in place (contracted and new elements differ) makes
        // the kernel hold two buffers of the inner size: such groups stay within
        // 2^kStemTwoBufferCap elements, so that three CTAs still share an SM
        bool two = false;
        for (size_t j = i; j < i + n; ++j) {
            const NodePlan& np = P.nodes[chain[j]];
            two |= !(np.kb == np.nb && np.kb > 0);
        }
        const int lim = two ? std::min(cap, kStemTwoBufferCap) : cap;
        if (mx > lim || (int)U.size() < net->stem_min_outer || U.size() > 30) return false;
        g = StemGroupPlan();
        g.steps.assign(chain.begin() + i, chain.begin() + i + n);
        g.in = P.nodes[chain[i]].A;
        g.out = P.nodes[chain[i + n - 1]].v;
        g.U = U;
        g.max_inner = mx;
        g.per_slice = P.nodes[chain[i]].per_slice;
        return true;
    };
    for (int c0 = 0; c0 < nn; ++c0) {
        if (!stem_step(net, P.nodes[c0]) || has_prev[c0]) continue;
        std::vector<int> chain;
        for (int j = c0; j >= 0; j = next[j]) chain.push_back(j);
        size_t i = 0;
        while (i < chain.size()) {
            // the longest group from chain[i] that fits; a single step is the
            // streaming form of one narrow contraction
            size_t best = 0;
            StemGroupPlan bg;
            for (size_t n = 1; i + n <= chain.size() && (int)n <= tnc::kStemMaxSteps; ++n) {
                StemGroupPlan g;
                if (!eval(chain, i, n, g)) break;
                best = n;
                bg = g;
            }
            if (best < 1) {
                ++i;
                continue;
            }
            const int gi = (int)P.stems.size();
            for (int k : bg.steps) P.stem_of[k] = gi;
            P.stems.push_back(bg);
            i += best;
        }
    }
}

// Kernel parameters of fused stem group gi for a batch of nb slices (see kernels.h).
tnc::StemParams stem_params(const tnc_net* net, const Arena& ar, char* ws, int gi, int64_t nb);


std::vector<Group> level_groups(const tnc_net* net, int mode, bool per_slice);

// Plane data of one operand (rows x K, every plane, every batch entry); split
// FP16x2 keeps the operand's scale exponents (one byte per row and 256-wide K
// chunk, per batch entry) after it, 256-byte aligned. How a contraction whose
// planes exceed the cap is cut up: tc_cut below.
int64_t plane_data_bytes(int mode, int rb, int kb, int64_t batch) {
    return align_up(batch * (int64_t)tnc::tc_plane_count(mode) * tnc::tc_elem_bytes(mode) << (rb + kb));
}

int64_t full_planes_bytes(int mode, int rb, int kb, int64_t batch) {
    const int64_t scales = mode == TNC_SPLIT_FP16X2 ? align_up((batch * tnc::tc_scale_chunks(kb)) << rb) : 0;
    return plane_data_bytes(mode, rb, kb, batch) + scales;
}

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

TcCut tc_cut(const tnc_net* net, int mode, int mb, int nb, int kb, int64_t batch) {
    const int64_t cap = (int64_t)1 << net_plane_cap_log2(net);
    TcCut c;
    auto fits = [&](int rb, int k) { return full_planes_bytes(mode, rb, k, batch) <= cap; };
    if (kb > mb && kb > nb) {
        while (kb - c.pK > 6 && !(fits(mb, kb - c.pK) && fits(nb, kb - c.pK))) ++c.pK;
    }
    while (c.pA < mb - 7 && !fits(mb - c.pA, kb - c.pK)) ++c.pA;
    while (c.pB < nb - 7 && !fits(nb - c.pB, kb - c.pK)) ++c.pB;
    const int64_t tiles = batch << ((mb - c.pA - 7) + (nb - c.pB - 7));
    while (c.ks < 6 && (tiles << c.ks) < 4 * 152 && kb - c.pK - c.ks > 12) ++c.ks;
    c.partial_off = full_planes_bytes(mode, mb - c.pA, kb - c.pK, batch);
    const int64_t partials = c.ks ? (batch << (c.ks + (mb - c.pA) + (nb - c.pB))) * 8 : 0;
    c.a_bytes = c.partial_off + partials;
    c.b_bytes = full_planes_bytes(mode, nb - c.pB, kb - c.pK, batch);
    return c;
}

int64_t tc_bytes_a(const tnc_net* net, int mode, int mb, int nb, int kb, int64_t batch) {
    return tc_cut(net, mode, mb, nb, kb, batch).a_bytes;
}

int64_t tc_bytes_b(const tnc_net* net, int mode, int mb, int nb, int kb, int64_t batch) {
    return tc_cut(net, mode, mb, nb, kb, batch).b_bytes;
}

// First-fit simulation of the workspace for a batch of `nb` slices.
Arena plan_arena(const tnc_net* net, int64_t nb, int mode) {
    const Plan& P = net->plan;
    const tnc::Tree& T = *net->tree;
    Arena ar;
    ar.off.assign(T.n_tensors(), -1);
    ar.planes_a.assign(P.nodes.size(), -1);
    ar.planes_b.assign(P.nodes.size(), -1);
    std::map<int64_t, int64_t> used;  // off -> len
    int64_t top = 0;
    auto alloc = [&](int64_t len) {
        len = align_up(len);
        int64_t prev_end = 0;
        for (auto& kv : used) {
            if (kv.first - prev_end >= len) break;
            prev_end = kv.first + kv.second;
        }
        int64_t off = prev_end;
        used[off] = len;
        top = std::max(top, off + len);
        return off;
    };
    auto release = [&](int64_t off) { used.erase(off); };
    auto tc_planes = [&](const NodePlan& np, int64_t b) {
        const size_t i = np.v - net->n_leaves;
        ar.planes_a[i] = alloc(tc_bytes_a(net, mode, np.mb, np.nb, np.kb, b));
        ar.planes_b[i] = alloc(tc_bytes_b(net, mode, np.mb, np.nb, np.kb, b));
    };
    auto tc_release = [&](const NodePlan& np) {
        const size_t i = np.v - net->n_leaves;
        release(ar.planes_a[i]);
        release(ar.planes_b[i]);
    };
    // Lifetimes follow the executed order: one tree level at a time; all
    // outputs of a level are live together, inputs die after their level.
    auto run_level = [&](const Group& g, int64_t b) {
        for (int v : g.fp32) ar.off[v] = alloc(b * tensor_bytes(P, v));
        for (int v : g.tc) ar.off[v] = alloc(b * tensor_bytes(P, v));
        // fused stem groups: only T_n is stored; T_1 .. T_{n-1} stay on chip
        for (int gi : g.stems) ar.off[P.stems[gi].out] = alloc(b * tensor_bytes(P, P.stems[gi].out));
        // the split planes of a level's tensor-core contractions are live
        // together: the persistent executor runs a level's contractions at
        // the same time
        for (int v : g.tc) {
            const NodePlan& np = P.nodes[v - net->n_leaves];
            if (shape_choice(net, mode, np.mb, np.nb, np.kb, np.is_root)) tc_planes(np, b);
        }
        for (int v : g.tc) {
            const NodePlan& np = P.nodes[v - net->n_leaves];
            if (shape_choice(net, mode, np.mb, np.nb, np.kb, np.is_root)) tc_release(np);
        }
        for (auto* list : {&g.fp32, &g.tc})
            for (int v : *list) {
                const NodePlan& np = P.nodes[v - net->n_leaves];
                for (int c : {np.A, np.B})
                    if (c >= net->n_leaves && P.per_slice[c] == (char)g.per_slice) release(ar.off[c]);
            }
        for (int gi : g.stems) {
            const StemGroupPlan& sg = P.stems[gi];
            std::vector<int> ins{sg.in};
            for (int k : sg.steps) ins.push_back(P.nodes[k].B);
            for (int c : ins)
                if (c >= net->n_leaves && P.per_slice[c] == (char)g.per_slice) release(ar.off[c]);
        }
    };
    // phase 1: invariant levels (batch 1); invariant tensors consumed by
    // per-slice nodes stay live for the whole call
    for (const Group& g : level_groups(net, mode, false)) run_level(g, 1);
    // phase 2: one batch of per-slice levels, then the root
    for (const Group& g : level_groups(net, mode, true)) run_level(g, nb);
    for (const NodePlan& np : P.nodes) {
        if (!np.is_root) continue;
        int64_t bytes = np.kind == K_ROOT_F64 ? nb * np.chunks * (int64_t)16 << (np.mb + np.nb)
                                              : nb * tensor_bytes(P, np.v);
        ar.root_scratch_off = alloc(bytes);
    }
    ar.peak = top;
    ar.batch = nb;
    return ar;
}

// Batch whose cut (panels, K splits, plane and partial layout) a tensor-core
// contraction of np uses when it runs b slices: the batch its workspace
// temporaries were sized for. A smaller last batch keeps that cut, since its
// own could need more bytes (fewer panels, or deeper K splits with more
// partials) than the arena reserved.
int64_t cut_batch(const Arena& ar, const NodePlan& np, int64_t b) {
    return std::max<int64_t>(b, np.per_slice ? ar.batch : 1);
}

tnc::Operand operand(const tnc_net* net, const Arena& ar, char* ws, int v, int64_t nb) {
    const Plan& P = net->plan;
    tnc::Operand op{};
    if (v < net->n_leaves) {
        const bool var = !net->var_off.empty() && net->var_off[v] >= 0;
        op.ptr = var ? net->d_var + net->var_off[v] : net->d_leaves + net->leaf_off[v];
        op.batch_stride = 0;
        op.n_sl = (int)P.sl[v].size();
        for (int j = 0; j < op.n_sl; ++j) {
            op.sl_bit[j] = P.sl[v][j].first;
            op.sl_stride[j] = P.sl[v][j].second;
        }
    } else {
        op.ptr = reinterpret_cast<const float2*>(ws + ar.off[v]);
        op.batch_stride = P.per_slice[v] ? (tensor_bytes(P, v) / 8) : 0;
        op.n_sl = 0;
    }
    (void)nb;
    return op;
}

tnc::GemmParams gemm_params(const tnc_net* net, const Arena& ar, char* ws, const NodePlan& np, int64_t nb) {
    tnc::GemmParams g{};
    g.A = operand(net, ar, ws, np.A, nb);
    g.B = operand(net, ar, ws, np.B, nb);
    g.mb = np.mb;
    g.nb = np.nb;
    g.kb = np.kb;
    for (int j = 0; j < np.mb; ++j) g.am[j] = np.am[j];
    for (int j = 0; j < np.kb; ++j) {
        g.ak[j] = np.ak[j];
        g.bk[j] = np.bk[j];
    }
    for (int j = 0; j < np.nb; ++j) g.bn[j] = np.bn[j];
    return g;
}

tnc_status ensure_plan(tnc_net* net) {
    if (!net->tree) return fail(TNC_E_STATE, "no contraction path set (call tnc_set_path)");
    if (!net->plan.valid) {
        try {
            build_plan(net);
        } catch (const std::exception& e) {
            return fail(TNC_E_INVALID, e.what());
        }
    }
    if (net->plan.stem_cap != net->stem_cap_log2) plan_stems(net);
    return TNC_OK;
}

tnc::StemParams stem_params(const tnc_net* net, const Arena& ar, char* ws, int gi, int64_t nb) {
    const Plan& P = net->plan;
    const StemGroupPlan& g = P.stems[gi];
    tnc::StemParams sp{};
    const std::set<int> Us(g.U.begin(), g.U.end());
    sp.in = operand(net, ar, ws, g.in, nb);
    std::vector<int> X;  // modes of the current inner sub-tensor, most significant first
    for (int m : P.layout[g.in])
        if (!Us.count(m)) X.push_back(m);
    sp.n_in = (int)X.size();
    for (int b = 0; b < sp.n_in; ++b) sp.istr[b] = stride_of(P.str[g.in], X[sp.n_in - 1 - b]);
    sp.nu = (int)g.U.size();
    for (int b = 0; b < sp.nu; ++b) {
        sp.ustr_in[b] = stride_of(P.str[g.in], g.U[b]);
        sp.ustr_out[b] = stride_of(P.str[g.out], g.U[b]);
    }
    int boff = 0;
    sp.nsteps = (int)g.steps.size();
    for (int j = 0; j < sp.nsteps; ++j) {
        const NodePlan& np = P.nodes[g.steps[j]];
        tnc::StemStep& st = sp.steps[j];
        std::map<int, int> bit;  // mode -> bit position in X (least significant 0)
        for (size_t q = 0; q < X.size(); ++q) bit[X[q]] = (int)(X.size() - 1 - q);
        const std::set<int> K(np.km.begin(), np.km.end());
        std::vector<int> kept;
        for (int m : X)
            if (!K.count(m)) kept.push_back(m);
        st.nr = (int)kept.size();
        st.nk = np.kb;
        st.nn = np.nb;
        for (int b = 0; b < st.nr; ++b) st.rstr[b] = 1 << bit[kept[st.nr - 1 - b]];
        for (int b = 0; b < st.nk; ++b) {
            st.kstr_x[b] = 1 << bit[np.km[st.nk - 1 - b]];
            st.kstr_b[b] = (int)np.bk[b];
        }
        for (int b = 0; b < st.nn; ++b) st.nstr_b[b] = (int)np.bn[b];
        st.b_off = boff;
        boff += 1 << (st.nk + st.nn);
        st.br = operand(net, ar, ws, np.B, nb);
        st.inplace = st.nk == st.nn && st.nk > 0;
        if (st.inplace) {
            // new mode nm[t] takes the place of contracted mode km[t] (k bit b
            // and n bit b are km[nk-1-b] and nm[nn-1-b])
            std::vector<int> pos;
            for (int m : np.km) pos.push_back(bit[m]);
            std::sort(pos.begin(), pos.end());
            for (int t = 0; t < st.nk; ++t) st.ins[t] = pos[t];
            for (int t = 0; t < st.nk; ++t)
                for (int& m : X)
                    if (m == np.km[t]) m = np.nm[t];
        } else {
            sp.two_buffers = 1;
            X = kept;
            X.insert(X.end(), np.nm.begin(), np.nm.end());
        }
    }
    sp.b_total = boff;
    sp.n_out = (int)X.size();
    for (int b = 0; b < sp.n_out; ++b) sp.ostr[b] = stride_of(P.str[g.out], X[sp.n_out - 1 - b]);
    sp.out = reinterpret_cast<float2*>(ws + ar.off[g.out]);
    sp.out_batch_stride = g.per_slice ? tensor_bytes(P, g.out) / 8 : 0;
    return sp;
}

tnc_status ensure_leaves(tnc_net* net, cudaStream_t st) {
    if (!net->d_leaves) {
        CUDA_TRY(cudaMalloc(&net->d_leaves, std::max<int64_t>(8, net->total_leaf_elems * 8)));
        net->dev_dirty = true;
    }
    if (!net->d_err) {
        CUDA_TRY(cudaMalloc(&net->d_err, 256));
        CUDA_TRY(cudaMemsetAsync(net->d_err, 0, 256, st));
    }
    if (net->dev_dirty) {
        CUDA_TRY(cudaMemcpyAsync(net->d_leaves, net->host_leaves.data(), net->total_leaf_elems * 8,
                                 cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));  // pageable source: keep the host copy stable
        net->dev_dirty = false;
    }
    if (net->var_dirty) {
        const size_t elems = net->host_var.size() / 2;
        if (elems > net->d_var_elems) {
            if (net->d_var) CUDA_TRY(cudaFree(net->d_var));
            net->d_var = nullptr;
            net->d_var_elems = 0;
            CUDA_TRY(cudaMalloc(&net->d_var, elems * 8));
            net->d_var_elems = elems;
        }
        if (elems) {
            CUDA_TRY(cudaMemcpyAsync(net->d_var, net->host_var.data(), elems * 8, cudaMemcpyHostToDevice, st));
            CUDA_TRY(cudaStreamSynchronize(st));
        }
        net->var_dirty = false;
    }
    return TNC_OK;
}

// Slice ids a call may address: the 2^|S| slices of every leaf variant.
int64_t slice_space(const tnc_net* net) {
    return 1ll << std::min<size_t>(net->S_sorted.size() + net->variant_bits, 62);
}

// Event pair around one launch when timing is on; returns the pool slot.
double node_cmacs(const tnc_net* net, int node) {
    if (node < net->n_leaves) return 0.0;
    const NodePlan& np = net->plan.nodes[node - net->n_leaves];
    return std::ldexp(1.0, np.mb + np.nb + np.kb);
}

cudaError_t timed_begin(tnc_net* net, int node, int kind, int batch, cudaStream_t s, double cmacs = -1.0) {
    net->launches += 1;
    if (!net->timing) return cudaSuccess;
    if (cmacs < 0) cmacs = node_cmacs(net, node) * batch;
    size_t slot = net->timed.size() * 2;
    while (net->ev_pool.size() < slot + 2) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        net->ev_pool.push_back(e);
    }
    net->timed.push_back({node, kind, batch, cmacs, slot});
    return cudaEventRecord(net->ev_pool[slot], s);
}

cudaError_t timed_end(tnc_net* net, cudaStream_t s) {
    if (!net->timing) return cudaSuccess;
    return cudaEventRecord(net->ev_pool[net->timed.back().ev + 1], s);
}

int64_t pick_batch(const tnc_net* net, int64_t want, size_t budget, int mode) {
    int64_t lo = 1, hi = std::max<int64_t>(1, std::min<int64_t>(want, 65535));
    if ((size_t)plan_arena(net, 1, mode).peak > budget) return 0;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if ((size_t)plan_arena(net, mid, mode).peak <= budget) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

std::vector<Group> level_groups(const tnc_net* net, int mode, bool per_slice) {
    const Plan& P = net->plan;
    const bool fuse = stem_fusion(net);
    std::map<int, int> level;  // tensor id -> level
    std::map<int, Group> by_level;
    for (size_t ni = 0; ni < P.nodes.size(); ++ni) {
        const NodePlan& np = P.nodes[ni];
        if (np.per_slice != per_slice || np.is_root) continue;
        int l = 0;
        for (int c : {np.A, np.B}) {
            auto it = level.find(c);
            if (it != level.end()) l = std::max(l, it->second);
        }
        level[np.v] = l + 1;
        Group& g = by_level[l + 1];
        g.per_slice = per_slice;
        if (fuse && P.stem_of[ni] >= 0) {  // a fused stem group runs at the level of its last step
            const int gi = P.stem_of[ni];
            if (P.stems[gi].steps.back() == (int)ni) g.stems.push_back(gi);
            continue;
        }
        // large contractions keep their own launch (parameters in kernel parameter space)
        if (shape_choice(net, mode, np.mb, np.nb, np.kb, np.is_root) ||
            (net->tuning && tc_node(mode, np.mb, np.nb, np.kb, np.is_root)) ||
            tnc::gemm_f32_tiles(np.mb, np.nb) >= 256)
            g.tc.push_back(np.v);
        else
            g.fp32.push_back(np.v);
    }
    std::vector<Group> out;
    for (auto& kv : by_level) out.push_back(kv.second);
    return out;
}

// Build (or reuse) the level groups and upload their parameter table for this
// plan, mode, batch and workspace.
tnc_status ensure_groups(tnc_net* net, const Arena& ar, char* ws, int mode, int64_t nb, cudaStream_t s) {
    std::string key = std::to_string(mode) + ":" + std::to_string(nb) + ":" + std::to_string((uintptr_t)ws) +
                      ":" + std::to_string(net->plan.version) + ":" + std::to_string(g_tune_version) + ":" +
                      std::to_string(net->force_choice) + ":" + std::to_string(net->tuning ? 1 : 0) + ":" +
                      std::to_string(stem_fusion(net) ? net->stem_cap_log2 : 0) + ":" +
                      std::to_string(net->plane_cap_log2);
    if (key == net->group_key) return TNC_OK;
    // the persistent work lists address this arena: built again on next use
    net->worklists.clear();
    GroupPlan G;
    G.inv = level_groups(net, mode, false);
    G.ps = level_groups(net, mode, true);
    for (auto* list : {&G.inv, &G.ps}) {
        for (Group& g : *list) {
            g.first = (int)G.params.size();
            g.off_first = (int)G.tile_off.size();
            int64_t tiles = 0;
            for (int v : g.fp32) {
                const NodePlan& np = net->plan.nodes[v - net->n_leaves];
                tnc::GemmParams gp = gemm_params(net, ar, ws, np, g.per_slice ? nb : 1);
                gp.C = reinterpret_cast<float2*>(ws + ar.off[np.v]);
                gp.c_batch_stride = g.per_slice ? tensor_bytes(net->plan, np.v) / 8 : 0;
                gp.slice0 = 0;
                G.params.push_back(gp);
                G.tile_off.push_back(tiles);
                tiles += tnc::gemm_f32_tiles(np.mb, np.nb);
                g.cmacs += std::ldexp(1.0, np.mb + np.nb + np.kb);
            }
            G.tile_off.push_back(tiles);
            g.tiles = tiles;
        }
    }
    if (stem_fusion(net)) {
        G.stem_params.resize(net->plan.stems.size());
        for (const auto* list : {&G.inv, &G.ps})
            for (const Group& g : *list)
                for (int gi : g.stems) G.stem_params[gi] = stem_params(net, ar, ws, gi, g.per_slice ? nb : 1);
        if (G.stem_params.size() > net->d_stem_cap) {
            if (net->d_stem) CUDA_TRY(cudaFree(net->d_stem));
            net->d_stem = nullptr;
            CUDA_TRY(cudaMalloc(&net->d_stem, G.stem_params.size() * sizeof(tnc::StemParams)));
            net->d_stem_cap = G.stem_params.size();
        }
        if (!G.stem_params.empty())
            CUDA_TRY(cudaMemcpyAsync(net->d_stem, G.stem_params.data(), G.stem_params.size() * sizeof(tnc::StemParams),
                                     cudaMemcpyHostToDevice, s));
    }
    if (G.params.size() > net->d_params_cap) {
        if (net->d_params) CUDA_TRY(cudaFree(net->d_params));
        net->d_params = nullptr;
        CUDA_TRY(cudaMalloc(&net->d_params, std::max<size_t>(1, G.params.size()) * sizeof(tnc::GemmParams)));
        net->d_params_cap = G.params.size();
    }
    if (G.tile_off.size() > net->d_tile_cap) {
        if (net->d_tile_off) CUDA_TRY(cudaFree(net->d_tile_off));
        net->d_tile_off = nullptr;
        CUDA_TRY(cudaMalloc(&net->d_tile_off, std::max<size_t>(1, G.tile_off.size()) * sizeof(int64_t)));
        net->d_tile_cap = G.tile_off.size();
    }
    if (!G.params.empty())
        CUDA_TRY(cudaMemcpyAsync(net->d_params, G.params.data(), G.params.size() * sizeof(tnc::GemmParams),
                                 cudaMemcpyHostToDevice, s));
    if (!G.tile_off.empty())
        CUDA_TRY(cudaMemcpyAsync(net->d_tile_off, G.tile_off.data(), G.tile_off.size() * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));  // host staging vectors are freed below
    net->groups = std::move(G);
    net->group_key = key;
    return TNC_OK;
}

tnc_status run_group(tnc_net* net, const Arena& ar, char* ws, const Group& g, int b, int64_t slice0, int mode,
                     cudaStream_t s);

// Split + tensor-core GEMM for the contraction described by g (operands,
// per-bit strides, output), cut up as tc_cut() says; pa and pb are workspace
// temporaries of tc_bytes_a() and tc_bytes_b() bytes.
tnc_status launch_tc_contraction(tnc_net* net, const tnc::GemmParams& g, int b, int mode, void* pa, void* pb,
                                 int node, cudaStream_t s, int row_bytes, int64_t cut_b) {
    const TcCut cut = tc_cut(net, mode, g.mb, g.nb, g.kb, std::max<int64_t>(cut_b, b));
    const int pA = cut.pA, pB = cut.pB, pK = cut.pK;
    const int mbp = g.mb - pA, nbp = g.nb - pB, kbp = g.kb - pK;
    const int64_t N = 1ll << g.nb;
    // an operand that is the same for every slice of the batch (no sliced
    // modes, no batch stride) is split and scanned once
    const bool a_shared = b > 1 && g.A.batch_stride == 0 && g.A.n_sl == 0;
    const bool b_shared = b > 1 && g.B.batch_stride == 0 && g.B.n_sl == 0;
    const int nza = a_shared ? 1 : b, nzb = b_shared ? 1 : b;
    float2* partial = cut.ks ? reinterpret_cast<float2*>(static_cast<char*>(pa) + cut.partial_off) : nullptr;
    // split FP16x2: scale exponents per row and 256-wide K chunk of each
    // operand, written by the split after the (panel-sized) plane data
    int8_t* sexp_a = nullptr;
    int8_t* sexp_b = nullptr;
    if (mode == TNC_SPLIT_FP16X2) {
        sexp_a = reinterpret_cast<int8_t*>(static_cast<char*>(pa) + plane_data_bytes(mode, mbp, kbp, b));
        sexp_b = reinterpret_cast<int8_t*>(static_cast<char*>(pb) + plane_data_bytes(mode, nbp, kbp, b));
    }
    auto split = [&](const tnc::Operand& src, int rb, const int64_t* rs, const int64_t* ks, void* dst,
                     int8_t* sexp, int nz) -> tnc_status {
        tnc::SplitParams sp{};
        sp.src = src;
        sp.rb = rb;
        sp.kb = kbp;
        for (int j = 0; j < rb; ++j) sp.rs[j] = rs[j];
        for (int j = 0; j < kbp; ++j) sp.ks[j] = ks[j];
        sp.slice0 = g.slice0;
        sp.dst = dst;
        sp.sexp = sexp;
        CUDA_TRY(timed_begin(net, node, K_SPLIT, nz, s, 0.0));
        CUDA_TRY(tnc::launch_split(sp, mode, nz, s));
        CUDA_TRY(timed_end(net, s));
        return TNC_OK;
    };
    tnc_status st;
    for (int64_t qk = 0; qk < (1ll << pK); ++qk) {  // K panels: the top pK bits of k fixed
        tnc::Operand Ak = g.A, Bk = g.B;
        for (int j = 0; j < pK; ++j)
            if ((qk >> j) & 1) {
                Ak.ptr += g.ak[kbp + j];
                Bk.ptr += g.bk[kbp + j];
            }
        for (int64_t qb = 0; qb < (1ll << pB); ++qb) {  // row panels of B: top pB bits of n fixed
            tnc::Operand B = Bk;
            for (int j = 0; j < pB; ++j)
                if ((qb >> j) & 1) B.ptr += g.bn[nbp + j];
            if ((st = split(B, nbp, g.bn, g.bk, pb, sexp_b, nzb)) != TNC_OK) return st;
            for (int64_t qa = 0; qa < (1ll << pA); ++qa) {  // row panels of A: top pA bits of m fixed
                tnc::Operand A = Ak;
                for (int j = 0; j < pA; ++j)
                    if ((qa >> j) & 1) A.ptr += g.am[mbp + j];
                if (pB == 0 || qb == 0 || pA > 0)  // else the A planes of this K panel are still in place
                    if ((st = split(A, mbp, g.am, g.ak, pa, sexp_a, nza)) != TNC_OK) return st;
                tnc::TcGemmParams tp{};
                tp.mb = mbp;
                tp.nb = nbp;
                tp.kb = kbp;
                tp.C = g.C + (qa << mbp) * N + (qb << nbp);
                tp.c_batch_stride = g.c_batch_stride;
                tp.c_ld = N;
                tp.err = net->d_err;
                tp.row_bytes = row_bytes;
                tp.sexp_a = sexp_a;
                tp.sexp_b = sexp_b;
                tp.group_m = net->tc_group_m;
                tp.spin_limit = net->tc_spin_limit;
                tp.test_stall = net->tc_test_stall;
                tp.ksplit_bits = cut.ks;
                tp.partial = partial;
                tp.accumulate = (!cut.ks && qk > 0) ? 1 : 0;
                tp.a_shared = a_shared ? 1 : 0;
                tp.b_shared = b_shared ? 1 : 0;
                CUDA_TRY(timed_begin(net, node, K_TC, b, s, std::ldexp(1.0, mbp + nbp + kbp) * b));
                CUDA_TRY(tnc::launch_cgemm_tc(tp, mode, pa, pb, b, s));
                CUDA_TRY(timed_end(net, s));
                if (cut.ks) {  // add the K splits' partials into C, in split order
                    CUDA_TRY(timed_begin(net, node, K_KRED, b, s, 0.0));
                    CUDA_TRY(tnc::launch_ksplit_reduce(partial, cut.ks, b, mbp, nbp, tp.C, g.c_batch_stride, N,
                                                       qk > 0 ? 1 : 0, s));
                    CUDA_TRY(timed_end(net, s));
                }
            }
        }
    }
    return TNC_OK;
}

// One non-root contraction: FP32 CUDA-core GEMM, or (split modes, large
// nodes) operand split + tensor-core GEMM. `g` carries operands and output.
tnc_status launch_node(tnc_net* net, const Arena& ar, char* ws, const NodePlan& np, const tnc::GemmParams& g,
                       int b, int mode, cudaStream_t s) {
    const int choice = shape_choice(net, mode, np.mb, np.nb, np.kb, np.is_root);
    if (!choice) {
        CUDA_TRY(timed_begin(net, np.v, K_GEMM_F32, b, s));
        CUDA_TRY(tnc::launch_gemm_f32(g, b, s));
        CUDA_TRY(timed_end(net, s));
        return TNC_OK;
    }
    const size_t i = np.v - net->n_leaves;
    return launch_tc_contraction(net, g, b, mode, ws + ar.planes_a[i], ws + ar.planes_b[i], np.v, s, choice,
                                 cut_batch(ar, np, b));
}

tnc_status run_group(tnc_net* net, const Arena& ar, char* ws, const Group& g, int b, int64_t slice0, int mode,
                     cudaStream_t s) {
    tnc_status st;
    if (!g.fp32.empty()) {
        CUDA_TRY(timed_begin(net, -1, K_GEMM_F32, b, s, g.cmacs * b));
        CUDA_TRY(tnc::launch_gemm_f32_group(net->d_params + g.first, net->d_tile_off + g.off_first,
                                            (int)g.fp32.size(), g.tiles, slice0, b, s));
        CUDA_TRY(timed_end(net, s));
    }
    for (int v : g.tc) {
        const NodePlan& np = net->plan.nodes[v - net->n_leaves];
        tnc::GemmParams gp = gemm_params(net, ar, ws, np, b);
        gp.C = reinterpret_cast<float2*>(ws + ar.off[np.v]);
        gp.c_batch_stride = g.per_slice ? tensor_bytes(net->plan, np.v) / 8 : 0;
        gp.slice0 = slice0;
        if ((st = launch_node(net, ar, ws, np, gp, b, mode, s)) != TNC_OK) return st;
    }
    for (int gi : g.stems) {
        const StemGroupPlan& sg = net->plan.stems[gi];
        double cm = 0.0;
        for (int k : sg.steps) cm += node_cmacs(net, net->plan.nodes[k].v);
        CUDA_TRY(timed_begin(net, sg.out, K_STEM, b, s, cm * b));
        CUDA_TRY(tnc::launch_stem_fused(net->d_stem + gi, net->groups.stem_params[gi], sg.max_inner, slice0, b, s));
        CUDA_TRY(timed_end(net, s));
    }
    return TNC_OK;
}


// ------------------------------------------------------ persistent executor
//
// A work list is the whole computation of one launch: every contraction of a
// slice batch (and, in the first batch of a call, the slice-invariant ones)
// broken into tasks, in level order so that every task only waits on tasks
// before it (see kernels.h). Per node, one counter counts the tasks of its
// last stage; a task waits on the counters of the nodes that produce its
// inputs in the same launch.

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
    // level[i] is task i's level number within its network
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
        t.signal2 = lvl_cur;
        // a slot left free takes the previous level (a task of a level waits
        // for the whole level before it: the workspace reuses memory across levels)
        if (lvl_prev >= 0) {
            bool have = false;
            for (int q = 0; q < 3; ++q) have |= t.wait[q] == lvl_prev;
            for (int q = 0; q < 3 && !have; ++q)
                if (t.wait[q] < 0) {
                    t.wait[q] = lvl_prev;
                    have = true;
                }
            no_slot |= !have;
        }
        if (lvl_cur >= 0) ++counters[lvl_cur];
        tasks.push_back(t);
        level.push_back(lvl_no);
    }
    void begin_level() {
        ++lvl_no;
        lvl_prev = lvl_cur;
        lvl_cur = new_counter(0);
    }
};


constexpr int kSplitBlocksPerTask = 16;

// Tasks of one non-root contraction np for batch b into W; ctr maps a tensor
// produced in this launch to its counter. False if the contraction needs row
// or K panels (not run by the persistent executor).
bool wl_node(tnc_net* net, const Arena& ar, char* ws, const NodePlan& np, int b, int mode, int netidx, WorkList& W,
             std::map<int, int>& ctr) {
    const Plan& P = net->plan;
    tnc::GemmParams g = gemm_params(net, ar, ws, np, b);
    g.C = reinterpret_cast<float2*>(ws + ar.off[np.v]);
    g.c_batch_stride = np.per_slice ? tensor_bytes(P, np.v) / 8 : 0;
    // inputs come from earlier tree levels, which the level chain already waits for
    const int wa = -1, wb = -1;
    W.cmacs += std::ldexp(1.0, np.mb + np.nb + np.kb) * b;
    const int choice = shape_choice(net, mode, np.mb, np.nb, np.kb, np.is_root);
    if (!choice) {
        const int gi = (int)W.gemm.size();
        W.gemm.push_back(g);
        const int64_t tiles = tnc::gemm_f32_tiles(np.mb, np.nb);
        const int c = W.new_counter((int)(tiles * b));
        for (int z = 0; z < b; ++z)
            for (int64_t t = 0; t < tiles; ++t) W.task(tnc::PT_GEMM, gi, t, z, netidx, 0, wa, wb, -1, c);
        ctr[np.v] = c;
        return true;
    }
    const TcCut cut = tc_cut(net, mode, g.mb, g.nb, g.kb, cut_batch(ar, np, b));
    if (cut.pA || cut.pB || cut.pK) return false;
    W.tc_cmacs += std::ldexp(1.0, np.mb + np.nb + np.kb) * b;
    const size_t i = np.v - net->n_leaves;
    char* pa = ws + ar.planes_a[i];
    char* pb = ws + ar.planes_b[i];
    const bool a_shared = b > 1 && g.A.batch_stride == 0 && g.A.n_sl == 0;
    const bool b_shared = b > 1 && g.B.batch_stride == 0 && g.B.n_sl == 0;
    int8_t* sexp_a = nullptr;
    int8_t* sexp_b = nullptr;
    if (mode == TNC_SPLIT_FP16X2) {
        sexp_a = reinterpret_cast<int8_t*>(pa + plane_data_bytes(mode, g.mb, g.kb, b));
        sexp_b = reinterpret_cast<int8_t*>(pb + plane_data_bytes(mode, g.nb, g.kb, b));
    }
    auto split = [&](const tnc::Operand& src, int rb, const int64_t* rs, const int64_t* ks, void* dst, int8_t* sexp,
                     int nz, int wsrc) {
        tnc::SplitParams sp{};
        sp.src = src;
        sp.rb = rb;
        sp.kb = g.kb;
        for (int j = 0; j < rb; ++j) sp.rs[j] = rs[j];
        for (int j = 0; j < g.kb; ++j) sp.ks[j] = ks[j];
        sp.dst = dst;
        sp.sexp = sexp;
        const int64_t blocks = tnc::tc_split_prepare(sp);
        if (blocks <= 0) return -2;
        const int si = (int)W.split.size();
        W.split.push_back(sp);
        const int64_t per = (blocks + kSplitBlocksPerTask - 1) / kSplitBlocksPerTask;
        const int c = W.new_counter((int)(per * nz));
        for (int z = 0; z < nz; ++z)
            for (int64_t q = 0; q < blocks; q += kSplitBlocksPerTask)
                W.task(tnc::PT_SPLIT, si, q, z, netidx,
                       (int)std::min<int64_t>(kSplitBlocksPerTask, blocks - q), wsrc, -1, -1, c);
        return c;
    };
    const int ca = split(g.A, g.mb, g.am, g.ak, pa, sexp_a, a_shared ? 1 : b, wa);
    const int cb = split(g.B, g.nb, g.bn, g.bk, pb, sexp_b, b_shared ? 1 : b, wb);
    if (ca == -2 || cb == -2) return false;
    tnc::TcGemmParams tp{};
    tp.mb = g.mb;
    tp.nb = g.nb;
    tp.kb = g.kb;
    tp.C = g.C;
    tp.c_batch_stride = g.c_batch_stride;
    tp.c_ld = 1ll << g.nb;
    tp.err = net->d_err;
    tp.row_bytes = 64;
    tp.group_m = net->tc_group_m;
    tp.spin_limit = net->tc_spin_limit;
    tp.test_stall = net->tc_test_stall;
    tp.sexp_a = sexp_a;
    tp.sexp_b = sexp_b;
    tp.ksplit_bits = cut.ks;
    tp.partial = cut.ks ? reinterpret_cast<float2*>(pa + cut.partial_off) : nullptr;
    tp.accumulate = 0;
    tp.a_shared = a_shared ? 1 : 0;
    tp.b_shared = b_shared ? 1 : 0;
    tnc::TcNode nd{};
    if (!tnc::tc_make_node(&nd, tp, mode, pa, pb, b)) return false;
    const int ti = (int)W.tc.size();
    W.tc.push_back(nd);
    const int64_t tiles = tnc::tc_node_tiles(tp);
    const int ct = W.new_counter((int)(tiles * b));
    for (int z = 0; z < b; ++z)
        for (int64_t t = 0; t < tiles; ++t) W.task(tnc::PT_TC, ti, t, z, netidx, 0, ca, cb, -1, ct);
    if (!cut.ks) {
        ctr[np.v] = ct;
        return true;
    }
    tnc::KredParams kp{};
    kp.partial = tp.partial;
    kp.nsplit = 1 << cut.ks;
    kp.batch = b;
    kp.nb = g.nb;
    kp.mn2 = (1ll << (g.mb + g.nb)) / 2;
    kp.C = g.C;
    kp.c_batch_stride = g.c_batch_stride;
    kp.c_ld = 1ll << g.nb;
    kp.accumulate = 0;
    const int ki = (int)W.kred.size();
    W.kred.push_back(kp);
    const int64_t chunks = (kp.mn2 + 16383) / 16384;
    const int ck = W.new_counter((int)(chunks * b));
    for (int z = 0; z < b; ++z)
        for (int64_t q = 0; q < chunks; ++q) W.task(tnc::PT_KRED, ki, q, z, netidx, 0, ct, -1, -1, ck);
    ctr[np.v] = ck;
    return true;
}

// Tasks of the final contraction of network netidx for batch b: FP64 chunk
// sums then their ordered sum into out (at most 64 outputs), or an FP32 root
// tensor then its FP64 slice sum.
bool wl_root(tnc_net* net, const Arena& ar, char* ws, const NodePlan& np, int b, int netidx, double* out, WorkList& W,
             std::map<int, int>& ctr) {
    const Plan& P = net->plan;
    const int wa = -1, wb = -1;  // the level chain waits for the inputs
    tnc::GemmParams g = gemm_params(net, ar, ws, np, b);
    tnc::PermParams pp{};
    pp.obits = P.obits;
    for (int j = 0; j < P.obits; ++j) pp.ostride[j] = P.out_stride[j];
    W.cmacs += std::ldexp(1.0, np.mb + np.nb + np.kb) * b;
    if (np.kind == K_ROOT_F64) {
        tnc::RootParams rp{};
        rp.g = g;
        rp.chunks = np.chunks;
        const int ri = (int)W.root.size();
        W.root.push_back(rp);
        tnc::AccParams ap{};
        ap.partials = reinterpret_cast<const double2*>(ws + ar.root_scratch_off);
        ap.count = b * np.chunks;
        ap.pp = pp;
        ap.out = reinterpret_cast<double2*>(out);
        const int ai = (int)W.acc.size();
        W.acc.push_back(ap);
        const int cr = W.new_counter(b * np.chunks);
        for (int z = 0; z < b; ++z)
            for (int c = 0; c < np.chunks; ++c) W.task(tnc::PT_ROOT, ri, c, z, netidx, ai, wa, wb, -1, cr);
        const int cdone = W.new_counter(1);
        W.task(tnc::PT_ACC, ai, 0, 0, netidx, 0, cr, -1, -1, cdone);
        return true;
    }
    g.C = reinterpret_cast<float2*>(ws + ar.root_scratch_off);
    g.c_batch_stride = tensor_bytes(P, np.v) / 8;
    const int gi = (int)W.gemm.size();
    W.gemm.push_back(g);
    const int64_t tiles = tnc::gemm_f32_tiles(np.mb, np.nb);
    const int cg = W.new_counter((int)(tiles * b));
    for (int z = 0; z < b; ++z)
        for (int64_t t = 0; t < tiles; ++t) W.task(tnc::PT_GEMM, gi, t, z, netidx, 0, wa, wb, -1, cg);
    tnc::SumTaskParams st{};
    st.sp.src.ptr = g.C;
    st.sp.src.batch_stride = g.c_batch_stride;
    st.sp.obits = P.obits;
    for (int j = 0; j < P.obits; ++j) st.sp.ostride[j] = P.out_stride[j];
    st.batch = b;
    st.out = reinterpret_cast<double2*>(out);
    const int si = (int)W.sum.size();
    W.sum.push_back(st);
    const int cdone = W.new_counter(1);
    W.task(tnc::PT_SUM, si, 0, 0, netidx, 0, cg, -1, -1, cdone);
    return true;
}

// Whether the persistent executor can run this network's contraction in
// mode: at least one contraction, no fused stem groups in use.
bool persist_eligible(tnc_net* net) {
    return net->persistent && !net->plan.nodes.empty() && !(stem_fusion(net) && !net->plan.stems.empty()) &&
           !net->tuning;
}

// Launches and estimated seconds of one batch of b slices on the per-level
// executor (the slice-invariant levels included when with_inv): one grouped
// launch per level for its FP32 contractions, three per tensor-core
// contraction (two operand splits and the GEMM), two for the final
// contraction. A contraction's time is estimated as the larger of its flops
// at 300 TFLOP/s and its operand and result bytes, 8 (MK + KN + MN) per
// slice, at 6 TB/s.
void level_cost(tnc_net* net, int mode, int64_t b, bool with_inv, double* launches, double* seconds) {
    const Plan& P = net->plan;
    auto node_s = [](const NodePlan& np, double bb) {
        const double M = std::ldexp(1.0, np.mb), N = std::ldexp(1.0, np.nb), K = std::ldexp(1.0, np.kb);
        return std::max(8.0 * M * N * K * bb / 3e14, 8.0 * (M * K + K * N + M * N) * bb / 6e12);
    };
    for (bool per : {false, true}) {
        if (!per && !with_inv) continue;
        for (const Group& g : level_groups(net, mode, per)) {
            if (!g.fp32.empty()) *launches += 1;
            for (int v : g.tc) {
                const NodePlan& np = P.nodes[v - net->n_leaves];
                *launches += shape_choice(net, mode, np.mb, np.nb, np.kb, np.is_root) ? 3 : 1;
            }
            for (auto* list : {&g.fp32, &g.tc})
                for (int v : *list) *seconds += node_s(P.nodes[v - net->n_leaves], per ? (double)b : 1.0);
        }
    }
    for (const NodePlan& np : P.nodes)
        if (np.is_root) {
            *launches += 2;
            *seconds += node_s(np, (double)b);
        }
}

// The automatic executor choice: the persistent kernel when the per-level
// launches would carry less than 60 us of estimated work each on average,
// i.e. when launch gaps and tail effects, not the contractions, would
// dominate.
constexpr double kPersistAutoSecondsPerLaunch = 60e-6;

// Tasks of one network for a batch b: the slice-invariant levels (if with_inv),
// the per-slice levels and the final contraction.
bool wl_network(tnc_net* net, const Arena& ar, char* ws, int b, int mode, bool with_inv, int netidx, double* out,
                WorkList& W) {
    std::map<int, int> ctr;
    const Plan& P = net->plan;
    W.lvl_prev = W.lvl_cur = W.lvl_no = -1;
    for (bool per : {false, true}) {
        if (!per && !with_inv) continue;
        for (const Group& g : level_groups(net, mode, per)) {
            W.begin_level();
            for (auto* list : {&g.fp32, &g.tc})
                for (int v : *list)
                    if (!wl_node(net, ar, ws, P.nodes[v - net->n_leaves], per ? b : 1, mode, netidx, W, ctr)) return false;
        }
    }
    W.begin_level();
    for (const NodePlan& np : P.nodes)
        if (np.is_root && !wl_root(net, ar, ws, np, b, netidx, out, W, ctr)) return false;
    return !W.no_slot;
}

// Appends the work list Wi (one network's tasks, its own tables and
// counters) to W: table indices and counter ids move by W's sizes so far.
void wl_append(WorkList& W, const WorkList& Wi) {
    const int o_gemm = (int)W.gemm.size(), o_split = (int)W.split.size(), o_tc = (int)W.tc.size(),
              o_kred = (int)W.kred.size(), o_root = (int)W.root.size(), o_acc = (int)W.acc.size(),
              o_sum = (int)W.sum.size(), o_ctr = (int)W.counters.size();
    for (size_t i = 0; i < Wi.tasks.size(); ++i) {
        tnc::PersistTask t = Wi.tasks[i];
        switch (t.type) {
            case tnc::PT_GEMM: t.idx += o_gemm; break;
            case tnc::PT_SPLIT: t.idx += o_split; break;
            case tnc::PT_TC: t.idx += o_tc; break;
            case tnc::PT_KRED: t.idx += o_kred; break;
            case tnc::PT_ROOT:
                t.idx += o_root;
                t.count += o_acc;  // the AccParams entry its chunk sums go to
                break;
            case tnc::PT_ACC: t.idx += o_acc; break;
            case tnc::PT_SUM: t.idx += o_sum; break;
            default: break;
        }
        for (int& c : t.wait)
            if (c >= 0) c += o_ctr;
        t.signal += o_ctr;
        if (t.signal2 >= 0) t.signal2 += o_ctr;
        W.tasks.push_back(t);
        W.level.push_back(Wi.level[i]);
    }
    W.counters.insert(W.counters.end(), Wi.counters.begin(), Wi.counters.end());
    W.gemm.insert(W.gemm.end(), Wi.gemm.begin(), Wi.gemm.end());
    W.split.insert(W.split.end(), Wi.split.begin(), Wi.split.end());
    W.tc.insert(W.tc.end(), Wi.tc.begin(), Wi.tc.end());
    W.kred.insert(W.kred.end(), Wi.kred.begin(), Wi.kred.end());
    W.root.insert(W.root.end(), Wi.root.begin(), Wi.root.end());
    W.acc.insert(W.acc.end(), Wi.acc.begin(), Wi.acc.end());
    W.sum.insert(W.sum.end(), Wi.sum.begin(), Wi.sum.end());
    W.cmacs += Wi.cmacs;
    W.tc_cmacs += Wi.tc_cmacs;
}

// Phase of a task type within its level: operand splits and root chunks
// first, then FP32 tiles (which wait on nothing of their level), then the
// tensor-core tiles (waiting on the splits), then reductions of tiles or
// chunks. A task only waits on tasks of an earlier phase of its level or on
// the level before.
int wl_phase(int type) {
    switch (type) {
        case tnc::PT_SPLIT:
        case tnc::PT_ROOT: return 0;
        case tnc::PT_GEMM: return 1;
        case tnc::PT_TC: return 2;
        case tnc::PT_KRED: return 3;
        default: return 4;
    }
}

// Orders the tasks (of one or several networks) by their level within their
// network, then by phase (stable, so each network keeps its own order
// otherwise): the CTAs take level L of every network before level L + 1 of
// any, and every split of a level well before the tiles that wait on it.
// Every wait still names tasks earlier in the list, since a task only waits
// on its own network's earlier levels and earlier phases of its level.
void wl_interleave_levels(WorkList& W) {
    std::vector<size_t> ord(W.tasks.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) {
        if (W.level[a] != W.level[b]) return W.level[a] < W.level[b];
        return wl_phase(W.tasks[a].type) < wl_phase(W.tasks[b].type);
    });
    std::vector<tnc::PersistTask> t(ord.size());
    std::vector<int> l(ord.size());
    for (size_t i = 0; i < ord.size(); ++i) {
        t[i] = W.tasks[ord[i]];
        l[i] = W.level[ord[i]];
    }
    W.tasks.swap(t);
    W.level.swap(l);
}

tnc_status wl_upload(const WorkList& W, DeviceWorkList& D, int* err, uint64_t wait_ns, uint32_t spin,
                     cudaStream_t s) {
    size_t off = 0;
    auto slot = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t o_tasks = slot(W.tasks.size() * sizeof(tnc::PersistTask));
    const size_t o_init = slot(W.counters.size() * sizeof(int));
    const size_t o_ctr = slot(W.counters.size() * sizeof(int) + sizeof(int));  // + ticket
    const size_t o_gemm = slot(W.gemm.size() * sizeof(tnc::GemmParams));
    const size_t o_split = slot(W.split.size() * sizeof(tnc::SplitParams));
    const size_t o_tc = slot(W.tc.size() * sizeof(tnc::TcNode));
    const size_t o_kred = slot(W.kred.size() * sizeof(tnc::KredParams));
    const size_t o_root = slot(W.root.size() * sizeof(tnc::RootParams));
    const size_t o_acc = slot(W.acc.size() * sizeof(tnc::AccParams));
    const size_t o_sum = slot(W.sum.size() * sizeof(tnc::SumTaskParams));
    CUDA_TRY(cudaMalloc(&D.mem, std::max<size_t>(off, 256)));
    char* base = static_cast<char*>(D.mem);
    auto up = [&](size_t o, const void* src, size_t bytes) -> cudaError_t {
        return bytes ? cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    CUDA_TRY(up(o_tasks, W.tasks.data(), W.tasks.size() * sizeof(tnc::PersistTask)));
    CUDA_TRY(up(o_init, W.counters.data(), W.counters.size() * sizeof(int)));
    CUDA_TRY(up(o_gemm, W.gemm.data(), W.gemm.size() * sizeof(tnc::GemmParams)));
    CUDA_TRY(up(o_split, W.split.data(), W.split.size() * sizeof(tnc::SplitParams)));
    CUDA_TRY(up(o_tc, W.tc.data(), W.tc.size() * sizeof(tnc::TcNode)));
    CUDA_TRY(up(o_kred, W.kred.data(), W.kred.size() * sizeof(tnc::KredParams)));
    CUDA_TRY(up(o_root, W.root.data(), W.root.size() * sizeof(tnc::RootParams)));
    CUDA_TRY(up(o_acc, W.acc.data(), W.acc.size() * sizeof(tnc::AccParams)));
    CUDA_TRY(up(o_sum, W.sum.data(), W.sum.size() * sizeof(tnc::SumTaskParams)));
    CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors may go
    tnc::PersistParams& P = D.prm;
    P = tnc::PersistParams{};
    P.tasks = reinterpret_cast<const tnc::PersistTask*>(base + o_tasks);
    P.ntasks = (int)W.tasks.size();
    P.counters = reinterpret_cast<int*>(base + o_ctr);
    P.ticket = P.counters + W.counters.size();
    P.err = err;
    P.gemm = reinterpret_cast<const tnc::GemmParams*>(base + o_gemm);
    P.split = reinterpret_cast<const tnc::SplitParams*>(base + o_split);
    P.tc = reinterpret_cast<const tnc::TcNode*>(base + o_tc);
    P.kred = reinterpret_cast<const tnc::KredParams*>(base + o_kred);
    P.root = reinterpret_cast<const tnc::RootParams*>(base + o_root);
    P.acc = reinterpret_cast<const tnc::AccParams*>(base + o_acc);
    P.sum = reinterpret_cast<const tnc::SumTaskParams*>(base + o_sum);
    P.wait_ns = wait_ns;
    P.spin_limit = spin;
    D.init = reinterpret_cast<int*>(base + o_init);
    D.n_counters = W.counters.size();
    D.cmacs = W.cmacs;
    D.tc_cmacs = W.tc_cmacs;
    return TNC_OK;
}

// Reset the counters and the ticket, then launch (stream-ordered; capturable).
cudaError_t wl_launch(const DeviceWorkList& D, int mode, int64_t slice0, const int64_t* rs0, cudaStream_t s,
                      unsigned long long* prof, double* out0) {
    cudaError_t e = cudaMemcpyAsync(D.prm.counters, D.init, D.n_counters * sizeof(int), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.prm.ticket, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    tnc::PersistParams p = D.prm;
    p.slice0 = slice0;
    p.rs0 = rs0;
    p.prof = prof;
    p.out0 = reinterpret_cast<double2*>(out0);
    return tnc::launch_persist(p, mode, s);
}

// Host-side check of a work list before its first launch: every range a task
// reads or writes (operands through their strides and slice offsets, outputs,
// split planes and scales, K-split partials, final sums) lies inside the
// workspace, the packed leaves or the result. A violation is a planning bug;
// the call then fails instead of launching.
bool wl_validate(const tnc_net* net, const WorkList& W, const char* ws, size_t ws_bytes, const double* out, int mode,
                 std::string* why) {
    const char* lv = reinterpret_cast<const char*>(net->d_leaves);
    const size_t lv_bytes = (size_t)net->total_leaf_elems * 8;
    const char* ob = reinterpret_cast<const char*>(out);
    const size_t out_bytes = (size_t)16 << net->plan.obits;
    const char* vb = reinterpret_cast<const char*>(net->d_var);
    const size_t vb_bytes = net->host_var.size() * 4;
    auto inside = [&](const void* p, int64_t bytes, const char* what) {
        const char* c = static_cast<const char*>(p);
        const bool ok = bytes >= 0 && ((c >= ws && c + bytes <= ws + ws_bytes) || (c >= lv && c + bytes <= lv + lv_bytes) ||
                                       (c >= ob && c + bytes <= ob + out_bytes) ||
                                       (vb && c >= vb && c + bytes <= vb + vb_bytes));
        if (!ok) *why = std::string("work list range outside its buffers: ") + what;
        return ok;
    };
    auto sum_of = [](const int64_t* st, int n) {
        int64_t t = 0;
        for (int j = 0; j < n; ++j) t += st[j];
        return t;
    };
    auto operand_ok = [&](const tnc::Operand& op, const int64_t* s1, int n1, const int64_t* s2, int n2, int nz,
                          const char* what) {
        int64_t hi = (int64_t)(nz - 1) * op.batch_stride + sum_of(s1, n1) + sum_of(s2, n2);
        for (int j = 0; j < op.n_sl; ++j) hi += op.sl_stride[j];
        return inside(op.ptr, (hi + 1) * 8, what);
    };
    std::map<std::pair<int, int>, int> nz;  // (type, idx) -> largest z + 1
    for (const tnc::PersistTask& t : W.tasks) {
        int& v = nz[{t.type, t.idx}];
        v = std::max(v, t.z + 1);
    }
    const int64_t pe = (int64_t)tnc::tc_plane_count(mode) * tnc::tc_elem_bytes(mode);
    for (size_t i = 0; i < W.gemm.size(); ++i) {
        const tnc::GemmParams& g = W.gemm[i];
        const int z = std::max(1, nz[{tnc::PT_GEMM, (int)i}]);
        if (!operand_ok(g.A, g.am, g.mb, g.ak, g.kb, z, "FP32 tile operand A") ||
            !operand_ok(g.B, g.bk, g.kb, g.bn, g.nb, z, "FP32 tile operand B") ||
            !inside(g.C, ((int64_t)(z - 1) * g.c_batch_stride + (1ll << (g.mb + g.nb))) * 8, "FP32 tile output"))
            return false;
    }
    for (size_t i = 0; i < W.split.size(); ++i) {
        const tnc::SplitParams& sp = W.split[i];
        const int z = std::max(1, nz[{tnc::PT_SPLIT, (int)i}]);
        if (!operand_ok(sp.src, sp.rs, sp.rb, sp.ks, sp.kb, z, "split source") ||
            !inside(sp.dst, (int64_t)z * pe << (sp.rb + sp.kb), "split planes") ||
            (sp.sexp && !inside(sp.sexp, ((int64_t)z * tnc::tc_scale_chunks(sp.kb)) << sp.rb, "split scales")))
            return false;
    }
    for (size_t i = 0; i < W.tc.size(); ++i) {
        const tnc::TcGemmParams& tp = W.tc[i].p;
        const int nb = W.tc[i].nbatch;
        const int64_t M = 1ll << tp.mb, N = 1ll << tp.nb;
        if (!inside(tp.C, ((int64_t)(nb - 1) * tp.c_batch_stride + (M - 1) * (tp.c_ld ? tp.c_ld : N) + N) * 8,
                    "tensor-core output") ||
            (tp.ksplit_bits && !inside(tp.partial, ((int64_t)nb << tp.ksplit_bits) * M * N * 8, "K-split partials")))
            return false;
    }
    for (const tnc::KredParams& kp : W.kred)
        if (!inside(kp.C, ((int64_t)(kp.batch - 1) * kp.c_batch_stride + 2 * kp.mn2) * 8, "K-split output") ||
            !inside(kp.partial, (int64_t)kp.nsplit * kp.batch * kp.mn2 * 16, "K-split partial sums"))
            return false;
    for (size_t i = 0; i < W.root.size(); ++i) {
        const tnc::GemmParams& g = W.root[i].g;
        const int z = std::max(1, nz[{tnc::PT_ROOT, (int)i}]);
        if (!operand_ok(g.A, g.am, g.mb, g.ak, g.kb, z, "final contraction operand A") ||
            !operand_ok(g.B, g.bk, g.kb, g.bn, g.nb, z, "final contraction operand B"))
            return false;
    }
    for (const tnc::AccParams& ap : W.acc)
        if (!inside(ap.partials, (int64_t)ap.count * 16 << ap.pp.obits, "final chunk sums") ||
            !inside(ap.out, (int64_t)16 << ap.pp.obits, "result"))
            return false;
    for (const tnc::SumTaskParams& st : W.sum)
        if (!operand_ok(st.sp.src, st.sp.ostride, st.sp.obits, nullptr, 0, st.batch, "root tensor") ||
            !inside(st.out, (int64_t)16 << st.sp.obits, "result"))
            return false;
    for (const tnc::PersistTask& t : W.tasks)
        for (int c : {t.wait[0], t.wait[1], t.wait[2], t.signal, t.signal2})
            if (c >= (int)W.counters.size()) {
                *why = "work list counter out of range";
                return false;
            }
    return true;
}

// The work list of one tnc_contract batch (b slices, invariants included or
// not), built and uploaded on first use; null if the persistent executor
// cannot run it.
DeviceWorkList* contract_worklist(tnc_net* net, const Arena& ar, char* ws, int b, int mode, bool with_inv,
                                  double* out, cudaStream_t s, tnc_status* st) {
    *st = TNC_OK;
    // the result pointer is not part of the list: launches pass it (out0)
    const std::string key = net->group_key + "|" + std::to_string(b) + ":" + std::to_string(with_inv ? 1 : 0) + ":" +
                            std::to_string(net->tc_spin_limit) + ":" +
                            std::to_string(net->tc_test_stall) + ":" + std::to_string(net->persist_test_stall) + ":" +
                            std::to_string(net->persist_wait_ns) + ":" + std::to_string(net->tc_group_m);
    auto it = net->worklists.find(key);
    if (it != net->worklists.end()) return it->second.get();
    WorkList W;
    if (!wl_network(net, ar, ws, b, mode, with_inv, 0, out, W)) return nullptr;
    wl_interleave_levels(W);
    if (net->persist_test_stall) {  // a task that waits on a counter no task decrements
        const int never = W.new_counter(1);
        const int c = W.new_counter(1);
        W.tasks.insert(W.tasks.begin(), tnc::PersistTask{tnc::PT_STALL, 0, 0, 0, 0, 0, {never, -1, -1}, c, -1});
    }
    std::string why;
    const size_t ws_bytes = net->ws_user ? net->ws_user_bytes : net->ws_own_bytes;
    if (!wl_validate(net, W, ws, ws_bytes, out, mode, &why)) {
        *st = fail(TNC_E_STATE, why);
        return nullptr;
    }
    auto D = std::make_unique<DeviceWorkList>();
    if ((*st = wl_upload(W, *D, net->d_err, net->persist_wait_ns, net->tc_spin_limit, s)) != TNC_OK) return nullptr;
    if (net->worklists.size() > 16) net->worklists.clear();
    DeviceWorkList* raw = D.get();
    net->worklists[key] = std::move(D);
    return raw;
}

// ------------------------------------------------------------ adjoint pass

// First-fit allocator over a workspace (also used as a dry run to size it).
struct FitAlloc {
    std::map<int64_t, int64_t> used;
    int64_t top = 0;
    int64_t alloc(int64_t len) {
        len = align_up(std::max<int64_t>(len, 1));
        int64_t prev_end = 0;
        for (auto& kv : used) {
            if (kv.first - prev_end >= len) break;
            prev_end = kv.first + kv.second;
        }
        used[prev_end] = len;
        top = std::max(top, prev_end + len);
        return prev_end;
    }
    void release(int64_t off) { used.erase(off); }
};

struct Backward {
    tnc_net* net;
    int mode;
    int64_t nb;
    bool exec;
    char* ws = nullptr;
    cudaStream_t s = nullptr;
    FitAlloc A;
    Arena fwd;                                     // offsets of forward intermediates and planes
    std::vector<char> needs;                       // per tensor: environment required
    std::vector<std::vector<int>> env_layout;      // per tensor
    std::vector<int64_t> env_off;                  // per tensor (current env buffer)
    std::vector<int64_t> inv_acc;                  // per invariant tensor: FP64 env accumulator
    int64_t leaf_grad = -1;                        // FP64 gradients of all leaves, packed
    // per-level checkpointing of per-slice intermediates
    int keep_every = 1;                            // keep tensors at levels divisible by this
    std::vector<char> keep, present;               // per tensor
    int64_t recomputed = 0;                        // nodes recomputed in the reverse walk
};

int64_t layout_stride(const std::vector<int>& layout, int mode) {
    const int L = (int)layout.size();
    for (int p = 0; p < L; ++p)
        if (layout[p] == mode) return 1ll << (L - 1 - p);
    return -1;
}

// Environment of child `c` of node np from the node's environment.
tnc_status env_child(Backward& bw, const NodePlan& np, int c, int64_t b, int64_t slice0) {
    tnc_net* net = bw.net;
    const Plan& P = net->plan;
    const bool is_a = (c == np.A);
    const int sib = is_a ? np.B : np.A;
    std::vector<int> lay;
    if (is_a) {
        lay = np.mm;
        lay.insert(lay.end(), np.km.begin(), np.km.end());
    } else {
        lay = np.km;
        lay.insert(lay.end(), np.nm.begin(), np.nm.end());
    }
    bw.env_layout[c] = lay;
    const bool per = P.per_slice[c] != 0;
    const int64_t elems = 1ll << lay.size();
    const int64_t bb = per ? b : b;  // per-slice environments of every child, batch b
    int64_t off = bw.A.alloc(bb * elems * 8);
    bw.env_off[c] = off;
    // GEMM dims of this environment: E_A is (mb, kb) over nb; E_B is (kb, nb) over mb
    const int gmb = is_a ? np.mb : np.kb, gnb = is_a ? np.kb : np.nb, gkb = is_a ? np.nb : np.mb;
    const int env_choice = shape_choice(net, bw.mode, gmb, gnb, gkb, false);
    const bool tc = env_choice != 0;
    int64_t pa = -1, pb = -1;
    if (tc) {  // split-precision planes (allocated in the sizing pass too)
        pa = bw.A.alloc(tc_bytes_a(bw.net, bw.mode, gmb, gnb, gkb, b));
        pb = bw.A.alloc(tc_bytes_b(bw.net, bw.mode, gmb, gnb, gkb, b));
    }
    if (!bw.exec) {
        if (tc) {
            bw.A.release(pa);
            bw.A.release(pb);
        }
        return TNC_OK;
    }
    tnc::GemmParams g{};
    const std::vector<int>& ev = bw.env_layout[np.v];
    tnc::Operand E{};
    E.ptr = reinterpret_cast<const float2*>(bw.ws + bw.env_off[np.v]);
    E.batch_stride = P.per_slice[np.v] || np.is_root ? ((int64_t)1 << ev.size()) : 0;
    tnc::Operand S = operand(net, bw.fwd, bw.ws, sib, b);
    if (is_a) {
        // E_A[m, k] = sum_n E_v[m, n] B[k, n]
        g.A = E;
        g.B = S;
        g.mb = np.mb;
        g.nb = np.kb;
        g.kb = np.nb;
        for (int j = 0; j < np.mb; ++j) g.am[j] = layout_stride(ev, np.mm[np.mb - 1 - j]);
        for (int j = 0; j < np.nb; ++j) {
            g.ak[j] = layout_stride(ev, np.nm[np.nb - 1 - j]);
            g.bk[j] = np.bn[j];
        }
        for (int j = 0; j < np.kb; ++j) g.bn[j] = np.bk[j];
    } else {
        // E_B[k, n] = sum_m A[m, k] E_v[m, n]
        g.A = S;
        g.B = E;
        g.mb = np.kb;
        g.nb = np.nb;
        g.kb = np.mb;
        for (int j = 0; j < np.kb; ++j) g.am[j] = np.ak[j];
        for (int j = 0; j < np.mb; ++j) {
            g.ak[j] = np.am[j];
            g.bk[j] = layout_stride(ev, np.mm[np.mb - 1 - j]);
        }
        for (int j = 0; j < np.nb; ++j) g.bn[j] = layout_stride(ev, np.nm[np.nb - 1 - j]);
    }
    g.C = reinterpret_cast<float2*>(bw.ws + off);
    g.c_batch_stride = elems;
    g.slice0 = slice0;
    if (tc) {
        // split precision with FP32 accumulation, as in the forward
        tnc_status st =
            launch_tc_contraction(net, g, (int)b, bw.mode, bw.ws + pa, bw.ws + pb, np.v, bw.s, env_choice, b);
        bw.A.release(pa);
        bw.A.release(pb);
        return st;
    }
    CUDA_TRY(timed_begin(net, np.v, K_GEMM_F32, (int)b, bw.s, std::ldexp(1.0, g.mb + g.nb + g.kb) * b));
    CUDA_TRY(tnc::launch_gemm_f32(g, (int)b, bw.s));
    CUDA_TRY(timed_end(net, bw.s));
    return TNC_OK;
}

// Fold the environment of child c (batch b) into its destination: leaves
// accumulate into their FP64 gradient; invariant tensors reached from a
// per-slice parent accumulate (over slices) into their FP64 environment;
// anything else keeps its environment for its own children.
tnc_status env_fold(Backward& bw, int c, int64_t b, int64_t slice0, bool from_per_slice) {
    tnc_net* net = bw.net;
    const Plan& P = net->plan;
    const int64_t elems = 1ll << bw.env_layout[c].size();
    if (c < net->n_leaves) {
        if (bw.exec) {
            tnc::LeafEnvParams lp{};
            lp.env = reinterpret_cast<const float2*>(bw.ws + bw.env_off[c]);
            lp.env_batch_stride = elems;
            int q = 0;
            for (int64_t e : net->leaf_idx[c])
                for (int bit = 0; bit < net->logd[e]; ++bit, ++q) {
                    const int mode = net->mode_base[e] + bit;
                    lp.sl_bit[q] = P.slice_bit_of_mode[mode];
                    lp.env_stride[q] = lp.sl_bit[q] >= 0 ? 0 : layout_stride(bw.env_layout[c], mode);
                }
            lp.L = q;
            lp.slice0 = slice0;
            lp.grad = reinterpret_cast<double2*>(bw.ws + bw.leaf_grad) + net->leaf_off[c];
            CUDA_TRY(timed_begin(net, c, -2, (int)b, bw.s, 0.0));
            CUDA_TRY(tnc::launch_leaf_env_accum(lp, (int)b, bw.s));
            CUDA_TRY(timed_end(net, bw.s));
        }
        bw.A.release(bw.env_off[c]);
    } else if (from_per_slice && !P.per_slice[c]) {
        if (bw.exec) {
            CUDA_TRY(tnc::launch_accum_batch_f64(reinterpret_cast<const float2*>(bw.ws + bw.env_off[c]), elems,
                                                 (int)b, elems,
                                                 reinterpret_cast<double2*>(bw.ws + bw.inv_acc[c]), bw.s));
            net->launches += 1;
        }
        bw.A.release(bw.env_off[c]);
    }
    return TNC_OK;
}

tnc_status fwd_node(Backward& bw, const NodePlan& np, int64_t b, int64_t slice0);

// Make the value of per-slice tensor v available, recomputing it (and, as
// needed, its own per-slice inputs) from the nearest kept tensors.
tnc_status materialize(Backward& bw, int v, int64_t b, int64_t slice0) {
    tnc_net* net = bw.net;
    if (v < net->n_leaves || !net->plan.per_slice[v] || bw.present[v]) return TNC_OK;
    const NodePlan& np = net->plan.nodes[v - net->n_leaves];
    tnc_status st;
    for (int c : {np.A, np.B})
        if ((st = materialize(bw, c, b, slice0)) != TNC_OK) return st;
    if ((st = fwd_node(bw, np, b, slice0)) != TNC_OK) return st;
    bw.present[v] = 1;
    bw.recomputed += 1;
    for (int c : {np.A, np.B})
        if (c >= net->n_leaves && net->plan.per_slice[c] && !bw.keep[c]) {
            bw.A.release(bw.fwd.off[c]);
            bw.present[c] = 0;
        }
    return TNC_OK;
}

// Reverse walk over the nodes of one class (per-slice or invariant).
tnc_status reverse_walk(Backward& bw, bool per_slice, int64_t b, int64_t slice0) {
    tnc_net* net = bw.net;
    const Plan& P = net->plan;
    tnc_status st;
    for (int i = (int)P.nodes.size() - 1; i >= 0; --i) {
        const NodePlan& np = P.nodes[i];
        const bool node_per = np.per_slice;
        if (node_per != per_slice) continue;
        if (!bw.needs[np.v]) continue;
        if (per_slice) {  // siblings feed the environment contractions
            if (bw.needs[np.A] && (st = materialize(bw, np.B, b, slice0)) != TNC_OK) return st;
            if (bw.needs[np.B] && (st = materialize(bw, np.A, b, slice0)) != TNC_OK) return st;
        }
        for (int c : {np.A, np.B}) {
            if (!bw.needs[c]) continue;
            if ((st = env_child(bw, np, c, b, slice0)) != TNC_OK) return st;
            if ((st = env_fold(bw, c, b, slice0, per_slice)) != TNC_OK) return st;
        }
        bw.A.release(bw.env_off[np.v]);
        if (per_slice)  // the children's values are not needed again
            for (int c : {np.A, np.B})
                if (c >= net->n_leaves && P.per_slice[c] && bw.present[c]) {
                    bw.A.release(bw.fwd.off[c]);
                    bw.present[c] = 0;
                }
    }
    return TNC_OK;
}

// One forward node kept for the reverse walk (all per-slice intermediates live).
tnc_status fwd_node(Backward& bw, const NodePlan& np, int64_t b, int64_t slice0) {
    tnc_net* net = bw.net;
    const Plan& P = net->plan;
    const bool per = np.per_slice;
    bw.fwd.off[np.v] = bw.A.alloc((per ? b : 1) * tensor_bytes(P, np.v));
    const bool tc = shape_choice(net, bw.mode, np.mb, np.nb, np.kb, np.is_root) != 0;
    const size_t i = np.v - net->n_leaves;
    if (tc) {
        bw.fwd.planes_a[i] = bw.A.alloc(tc_bytes_a(net, bw.mode, np.mb, np.nb, np.kb, per ? b : 1));
        bw.fwd.planes_b[i] = bw.A.alloc(tc_bytes_b(net, bw.mode, np.mb, np.nb, np.kb, per ? b : 1));
    }
    if (bw.exec) {
        tnc::GemmParams g = gemm_params(net, bw.fwd, bw.ws, np, b);
        g.C = reinterpret_cast<float2*>(bw.ws + bw.fwd.off[np.v]);
        g.c_batch_stride = per ? tensor_bytes(P, np.v) / 8 : 0;
        g.slice0 = slice0;
        tnc_status st = launch_node(net, bw.fwd, bw.ws, np, g, per ? (int)b : 1, bw.mode, bw.s);
        if (st != TNC_OK) return st;
    }
    if (tc) {
        bw.A.release(bw.fwd.planes_a[i]);
        bw.A.release(bw.fwd.planes_b[i]);
    }
    return TNC_OK;
}

// The whole backward computation; with exec == false only the workspace is sized.
tnc_status backward_run(Backward& bw, int64_t lo, int64_t hi, const double* grad_out) {
    tnc_net* net = bw.net;
    const Plan& P = net->plan;
    const tnc::Tree& T = *net->tree;
    tnc_status st;
    bw.fwd.off.assign(T.n_tensors(), -1);
    bw.fwd.planes_a.assign(P.nodes.size(), -1);
    bw.fwd.planes_b.assign(P.nodes.size(), -1);
    bw.env_layout.assign(T.n_tensors(), {});
    bw.env_off.assign(T.n_tensors(), -1);
    bw.inv_acc.assign(T.n_tensors(), -1);
    // checkpoint levels: per-slice dependency depth; the root's inputs are kept
    bw.keep.assign(T.n_tensors(), 0);
    bw.present.assign(T.n_tensors(), 0);
    {
        std::vector<int> level(T.n_tensors(), 0);
        for (const NodePlan& np : P.nodes) {
            if (!np.per_slice || np.is_root) continue;
            int l = 0;
            for (int c : {np.A, np.B})
                if (c >= net->n_leaves && P.per_slice[c]) l = std::max(l, level[c]);
            level[np.v] = l + 1;
            bw.keep[np.v] = (level[np.v] % std::max(1, bw.keep_every)) == 0;
        }
        if (!P.nodes.empty())
            for (int c : {P.nodes.back().A, P.nodes.back().B}) bw.keep[c] = 1;
    }
    bw.leaf_grad = bw.A.alloc(net->total_leaf_elems * 16);
    if (bw.exec) CUDA_TRY(cudaMemsetAsync(bw.ws + bw.leaf_grad, 0, net->total_leaf_elems * 16, bw.s));
    // invariant forward, kept for the whole call
    for (const NodePlan& np : P.nodes)
        if (!np.per_slice && !np.is_root)
            if ((st = fwd_node(bw, np, 1, 0)) != TNC_OK) return st;
    // FP64 environment accumulators of invariant tensors whose parent is per-slice
    for (int v = net->n_leaves; v < T.n_tensors(); ++v) {
        if (P.per_slice[v] || v == T.root || !bw.needs[v]) continue;
        const int par = T.parent[v];
        if (par < 0 || !(P.per_slice[par] || par == T.root)) continue;
        const int64_t bytes = (int64_t)16 << P.layout[v].size();
        bw.inv_acc[v] = bw.A.alloc(bytes);
        if (bw.exec) CUDA_TRY(cudaMemsetAsync(bw.ws + bw.inv_acc[v], 0, bytes, bw.s));
    }
    const int root = T.root;
    for (int64_t s0 = lo; s0 < hi; s0 += bw.nb) {
        const int64_t b = std::min<int64_t>(bw.nb, hi - s0);
        FitAlloc saved = bw.A;
        // per-slice forward, root excluded; tensors off the checkpoint levels are
        // dropped once consumed and recomputed in the reverse walk
        std::fill(bw.present.begin(), bw.present.end(), 0);
        for (const NodePlan& np : P.nodes) {
            if (!np.per_slice || np.is_root) continue;
            if ((st = fwd_node(bw, np, b, s0)) != TNC_OK) return st;
            bw.present[np.v] = 1;
            for (int c : {np.A, np.B})
                if (c >= net->n_leaves && P.per_slice[c] && !bw.keep[c] && bw.present[c]) {
                    bw.A.release(bw.fwd.off[c]);
                    bw.present[c] = 0;
                }
        }
        // seed: the root's environment is grad_out (in the root's layout)
        bw.env_layout[root] = P.layout[root];
        const int64_t relems = 1ll << P.layout[root].size();
        bw.env_off[root] = bw.A.alloc(b * relems * 8);
        if (bw.exec) {
            tnc::SeedParams sp{};
            sp.grad = reinterpret_cast<const double2*>(grad_out);
            sp.obits = P.obits;
            for (int j = 0; j < P.obits; ++j) sp.ostride[j] = P.out_stride[j];
            sp.E = reinterpret_cast<float2*>(bw.ws + bw.env_off[root]);
            sp.batch_stride = relems;
            CUDA_TRY(tnc::launch_env_seed(sp, (int)b, bw.s));
            net->launches += 1;
        }
        if (root < net->n_leaves) {
            if ((st = env_fold(bw, root, b, s0, true)) != TNC_OK) return st;
        } else if ((st = reverse_walk(bw, true, b, s0)) != TNC_OK) {
            return st;
        }
        bw.A.used = saved.used;  // the batch's buffers are dead; keep the peak
    }
    // invariant reverse walk from the accumulated environments (batch 1)
    for (int v = net->n_leaves; v < T.n_tensors(); ++v) {
        if (bw.inv_acc[v] < 0) continue;
        // the accumulator holds the environment in the layout its per-slice
        // parent produced (env_layout[v], set by env_child; same size as v)
        const int64_t elems = (int64_t)1 << P.layout[v].size();
        if (bw.env_layout[v].empty() && !P.layout[v].empty()) bw.env_layout[v] = P.layout[v];
        bw.env_off[v] = bw.A.alloc(elems * 8);
        if (bw.exec)
            CUDA_TRY(tnc::launch_f64_to_f32(reinterpret_cast<const double2*>(bw.ws + bw.inv_acc[v]), elems,
                                            reinterpret_cast<float2*>(bw.ws + bw.env_off[v]), bw.s));
    }
    if ((st = reverse_walk(bw, false, 1, 0)) != TNC_OK) return st;
    return TNC_OK;
}


// ------------------------------------------------------- many networks

// Several networks contracted together: their level groups merge into shared
// launches (level L of every network in one grouped launch), each network
// advancing through its own slice range one batch per round; the final
// reductions of all networks share two launches per round. The whole launch
// sequence is captured once into a CUDA graph and replayed for identical calls.
struct ManyCall {
    struct MGroup {
        int first = 0, n = 0, off_first = 0;
        int64_t tiles = 0;
        int max_b = 1;
        std::vector<std::pair<int, int>> singles;  // (network, node) launched one by one
    };
    std::vector<tnc_net*> nets;
    std::vector<uint64_t> uids;
    std::vector<int64_t> lo, hi, nb;
    std::vector<double*> outs;
    std::vector<Arena> arenas;
    std::vector<char*> wss;
    int mode = 0, rounds = 0;
    std::vector<MGroup> inv, ps;
    std::vector<int64_t> h_rs0;
    std::vector<int> h_rb;
    int64_t root_blocks = 0;
    int max_nb = 1;
    // device tables
    void* d_mem = nullptr;
    tnc::GemmParams* d_params = nullptr;
    int64_t* d_tile_off = nullptr;
    int* d_net = nullptr;
    int64_t* d_rs0 = nullptr;
    int* d_rb = nullptr;
    tnc::RootParams* d_roots = nullptr;
    double2** d_partials = nullptr;
    int64_t* d_blk_off = nullptr;
    tnc::PermParams* d_perms = nullptr;
    double2** d_outs = nullptr;
    // persistent executor: one work list (one launch) per round, empty when
    // the call runs on the merged level launches
    std::vector<std::unique_ptr<DeviceWorkList>> wls;
    cudaGraphExec_t graph = nullptr;
    bool warmed = false;
    int64_t kernels = 0;
    ~ManyCall() {
        if (graph) cudaGraphExecDestroy(graph);
        if (d_mem) cudaFree(d_mem);
    }
};

std::map<std::string, std::unique_ptr<ManyCall>>& many_cache() {
    static std::map<std::string, std::unique_ptr<ManyCall>> c;
    return c;
}

void many_forget(uint64_t uid) {
    auto& c = many_cache();
    for (auto it = c.begin(); it != c.end();) {
        bool hit = false;
        for (uint64_t u : it->second->uids) hit |= (u == uid);
        if (hit) it = c.erase(it);
        else ++it;
    }
}

// Launch sequence of one many-network call (recorded into a graph by the caller).
tnc_status many_run(ManyCall& mc, cudaStream_t s) {
    tnc_status st;
    const int n = (int)mc.nets.size();
    for (int i = 0; i < n; ++i) {
        CUDA_TRY(cudaMemsetAsync(mc.outs[i], 0, ((size_t)16) << mc.nets[i]->plan.obits, s));
        CUDA_TRY(cudaMemsetAsync(mc.nets[i]->d_err, 0, sizeof(int), s));
    }
    mc.kernels = 0;
    if (!mc.wls.empty()) {
        for (size_t r = 0; r < mc.wls.size(); ++r) {
            CUDA_TRY(wl_launch(*mc.wls[r], mc.mode, 0, mc.d_rs0 + (int64_t)r * n, s, mc.nets[0]->d_prof, nullptr));
            mc.kernels += 1;
        }
        return TNC_OK;
    }
    auto run_groups = [&](const std::vector<ManyCall::MGroup>& groups, const int64_t* rs0, const int* rb,
                          const int64_t* h_rs0, const int* h_rb, bool per_slice) -> tnc_status {
        for (const auto& g : groups) {
            if (g.n > 0) {
                CUDA_TRY(tnc::launch_gemm_f32_group_multi(mc.d_params + g.first, mc.d_tile_off + g.off_first, g.n,
                                                          g.tiles, mc.d_net + g.first, rs0, rb, g.max_b, s));
                mc.kernels += 1;
            }
            for (auto [i, v] : g.singles) {
                const int b = h_rb[i];
                if (b < 1) continue;
                tnc_net* net = mc.nets[i];
                const NodePlan& np = net->plan.nodes[v - net->n_leaves];
                tnc::GemmParams gp = gemm_params(net, mc.arenas[i], mc.wss[i], np, b);
                gp.C = reinterpret_cast<float2*>(mc.wss[i] + mc.arenas[i].off[np.v]);
                gp.c_batch_stride = per_slice ? tensor_bytes(net->plan, np.v) / 8 : 0;
                gp.slice0 = h_rs0[i];
                int64_t before = net->launches;
                if ((st = launch_node(net, mc.arenas[i], mc.wss[i], np, gp, b, mc.mode, s)) != TNC_OK) return st;
                mc.kernels += net->launches - before;
            }
        }
        return TNC_OK;
    };
    const int R = mc.rounds;
    if ((st = run_groups(mc.inv, mc.d_rs0 + (int64_t)R * n, mc.d_rb + (int64_t)R * n, mc.h_rs0.data() + (int64_t)R * n,
                         mc.h_rb.data() + (int64_t)R * n, false)) != TNC_OK)
        return st;
    for (int r = 0; r < R; ++r) {
        const int64_t* rs0 = mc.d_rs0 + (int64_t)r * n;
        const int* rb = mc.d_rb + (int64_t)r * n;
        if ((st = run_groups(mc.ps, rs0, rb, mc.h_rs0.data() + (int64_t)r * n, mc.h_rb.data() + (int64_t)r * n,
                             true)) != TNC_OK)
            return st;
        CUDA_TRY(tnc::launch_root_multi(mc.d_roots, mc.d_partials, mc.d_blk_off, n, mc.root_blocks, mc.d_perms,
                                        mc.d_outs, rs0, rb, mc.max_nb, s));
        mc.kernels += 2;
    }
    return TNC_OK;
}

tnc_status many_build(ManyCall& mc, cudaStream_t s) {
    tnc_status st;
    const int n = (int)mc.nets.size();
    // the merged level launches of many networks take no fused stem groups
    struct NoFuse {
        std::vector<tnc_net*>& nets;
        explicit NoFuse(std::vector<tnc_net*>& v) : nets(v) { for (auto* t : nets) t->in_many = true; }
        ~NoFuse() { for (auto* t : nets) t->in_many = false; }
    } no_fuse(mc.nets);
    mc.arenas.resize(n);
    mc.wss.resize(n);
    mc.nb.resize(n);
    int max_inv = 0, max_ps = 0;
    for (int i = 0; i < n; ++i) {
        tnc_net* net = mc.nets[i];
        if ((st = ensure_plan(net)) != TNC_OK) return st;
        if ((st = ensure_leaves(net, s)) != TNC_OK) return st;
        const Plan& P = net->plan;
        if (P.nodes.empty()) return fail(TNC_E_INVALID, "network " + std::to_string(i) + " has a single tensor");
        if (P.nodes.back().kind != K_ROOT_F64)
            return fail(TNC_E_INVALID, "network " + std::to_string(i) + " has more than 64 outputs");
        const int64_t want = mc.hi[i] - mc.lo[i];
        int64_t nb = 0;
        char* ws = nullptr;
        if (net->ws_user) {
            nb = pick_batch(net, std::max<int64_t>(want, 1), net->ws_user_bytes, mc.mode);
            if (nb < 1) return fail(TNC_E_OOM, "workspace too small for one slice");
            ws = (char*)net->ws_user;
        } else {
            size_t one = (size_t)plan_arena(net, 1, mc.mode).peak;
            nb = pick_batch(net, std::min<int64_t>(std::max<int64_t>(want, 1), 1024),
                            std::max<size_t>(one, (size_t)256 << 20), mc.mode);
            size_t need = (size_t)plan_arena(net, nb, mc.mode).peak;
            if (net->ws_own_bytes < need) {
                if (net->ws_own) CUDA_TRY(cudaFree(net->ws_own));
                net->ws_own = nullptr;
                net->ws_own_bytes = 0;
                CUDA_TRY(cudaMalloc(&net->ws_own, std::max<size_t>(need, kAlign)));
                net->ws_own_bytes = need;
                net->group_key.clear();
            }
            ws = (char*)net->ws_own;
        }
        mc.nb[i] = nb;
        mc.wss[i] = ws;
        net->inv_key.clear();
        mc.arenas[i] = plan_arena(net, nb, mc.mode);
        if ((st = ensure_groups(net, mc.arenas[i], ws, mc.mode, nb, s)) != TNC_OK) return st;
        max_inv = std::max(max_inv, (int)net->groups.inv.size());
        max_ps = std::max(max_ps, (int)net->groups.ps.size());
        mc.max_nb = std::max<int>(mc.max_nb, (int)nb);
        net->last_batch = nb;
    }
    // merged groups and their parameter tables
    std::vector<tnc::GemmParams> params;
    std::vector<int64_t> tile_off;
    std::vector<int> netidx;
    auto merge = [&](bool per_slice, int levels, std::vector<ManyCall::MGroup>& out) {
        for (int L = 0; L < levels; ++L) {
            ManyCall::MGroup mg;
            mg.first = (int)params.size();
            mg.off_first = (int)tile_off.size();
            int64_t tiles = 0;
            for (int i = 0; i < n; ++i) {
                tnc_net* net = mc.nets[i];
                const auto& list = per_slice ? net->groups.ps : net->groups.inv;
                if (L >= (int)list.size()) continue;
                const Group& g = list[L];
                for (size_t k = 0; k < g.fp32.size(); ++k) {
                    const NodePlan& np = net->plan.nodes[g.fp32[k] - net->n_leaves];
                    params.push_back(net->groups.params[g.first + k]);
                    netidx.push_back(i);
                    tile_off.push_back(tiles);
                    tiles += tnc::gemm_f32_tiles(np.mb, np.nb);
                }
                for (int v : g.tc) mg.singles.emplace_back(i, v);
                if (per_slice) mg.max_b = std::max<int>(mg.max_b, (int)mc.nb[i]);
            }
            tile_off.push_back(tiles);
            mg.n = (int)params.size() - mg.first;
            mg.tiles = tiles;
            out.push_back(mg);
        }
    };
    merge(false, max_inv, mc.inv);
    merge(true, max_ps, mc.ps);
    // round tables: rounds 0..R-1, then the invariant slot R (slice 0, batch 1)
    int R = 0;
    for (int i = 0; i < n; ++i) R = std::max<int>(R, (int)((mc.hi[i] - mc.lo[i] + mc.nb[i] - 1) / mc.nb[i]));
    mc.rounds = R;
    mc.h_rs0.assign((size_t)(R + 1) * n, 0);
    mc.h_rb.assign((size_t)(R + 1) * n, 0);
    for (int r = 0; r < R; ++r)
        for (int i = 0; i < n; ++i) {
            const int64_t s0 = mc.lo[i] + r * mc.nb[i];
            mc.h_rs0[(size_t)r * n + i] = s0;
            mc.h_rb[(size_t)r * n + i] = (int)std::max<int64_t>(0, std::min<int64_t>(mc.nb[i], mc.hi[i] - s0));
        }
    for (int i = 0; i < n; ++i) mc.h_rb[(size_t)R * n + i] = 1;
    // root tables
    std::vector<tnc::RootParams> roots(n);
    std::vector<double2*> partials(n), outs(n);
    std::vector<tnc::PermParams> perms(n);
    std::vector<int64_t> blk_off(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        tnc_net* net = mc.nets[i];
        const NodePlan& np = net->plan.nodes.back();
        roots[i].g = gemm_params(net, mc.arenas[i], mc.wss[i], np, mc.nb[i]);
        roots[i].chunks = np.chunks;
        partials[i] = reinterpret_cast<double2*>(mc.wss[i] + mc.arenas[i].root_scratch_off);
        outs[i] = reinterpret_cast<double2*>(mc.outs[i]);
        perms[i].obits = net->plan.obits;
        for (int j = 0; j < net->plan.obits; ++j) perms[i].ostride[j] = net->plan.out_stride[j];
        blk_off[i + 1] = blk_off[i] + np.chunks;
    }
    mc.root_blocks = blk_off[n];
    // one device allocation for every table
    size_t off = 0;
    auto slot = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t o_params = slot(params.size() * sizeof(tnc::GemmParams));
    const size_t o_tile = slot(tile_off.size() * sizeof(int64_t));
    const size_t o_net = slot(netidx.size() * sizeof(int));
    const size_t o_rs0 = slot(mc.h_rs0.size() * sizeof(int64_t));
    const size_t o_rb = slot(mc.h_rb.size() * sizeof(int));
    const size_t o_roots = slot(roots.size() * sizeof(tnc::RootParams));
    const size_t o_part = slot(partials.size() * sizeof(double2*));
    const size_t o_blk = slot(blk_off.size() * sizeof(int64_t));
    const size_t o_perm = slot(perms.size() * sizeof(tnc::PermParams));
    const size_t o_outs = slot(outs.size() * sizeof(double2*));
    CUDA_TRY(cudaMalloc(&mc.d_mem, std::max<size_t>(off, 256)));
    char* base = (char*)mc.d_mem;
    mc.d_params = reinterpret_cast<tnc::GemmParams*>(base + o_params);
    mc.d_tile_off = reinterpret_cast<int64_t*>(base + o_tile);
    mc.d_net = reinterpret_cast<int*>(base + o_net);
    mc.d_rs0 = reinterpret_cast<int64_t*>(base + o_rs0);
    mc.d_rb = reinterpret_cast<int*>(base + o_rb);
    mc.d_roots = reinterpret_cast<tnc::RootParams*>(base + o_roots);
    mc.d_partials = reinterpret_cast<double2**>(base + o_part);
    mc.d_blk_off = reinterpret_cast<int64_t*>(base + o_blk);
    mc.d_perms = reinterpret_cast<tnc::PermParams*>(base + o_perm);
    mc.d_outs = reinterpret_cast<double2**>(base + o_outs);
    auto up = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    CUDA_TRY(up(mc.d_params, params.data(), params.size() * sizeof(tnc::GemmParams)));
    CUDA_TRY(up(mc.d_tile_off, tile_off.data(), tile_off.size() * sizeof(int64_t)));
    CUDA_TRY(up(mc.d_net, netidx.data(), netidx.size() * sizeof(int)));
    CUDA_TRY(up(mc.d_rs0, mc.h_rs0.data(), mc.h_rs0.size() * sizeof(int64_t)));
    CUDA_TRY(up(mc.d_rb, mc.h_rb.data(), mc.h_rb.size() * sizeof(int)));
    CUDA_TRY(up(mc.d_roots, roots.data(), roots.size() * sizeof(tnc::RootParams)));
    CUDA_TRY(up(mc.d_partials, partials.data(), partials.size() * sizeof(double2*)));
    CUDA_TRY(up(mc.d_blk_off, blk_off.data(), blk_off.size() * sizeof(int64_t)));
    CUDA_TRY(up(mc.d_perms, perms.data(), perms.size() * sizeof(tnc::PermParams)));
    CUDA_TRY(up(mc.d_outs, outs.data(), outs.size() * sizeof(double2*)));
    CUDA_TRY(cudaStreamSynchronize(s));
    // persistent executor (when every network has it on): per round one work
    // list with every network's tasks, levels interleaved; slice ids per
    // network come from the round's row of the device table d_rs0. A network
    // it cannot run keeps the whole call on the merged level launches.
    bool pers = true, forced = true;
    for (tnc_net* net : mc.nets) {
        pers &= net->persistent != 0;
        forced &= net->persistent == 1;
    }
    if (pers && !forced) {  // automatic choice over the whole call
        double launches = 0, seconds = 0;
        for (int i = 0; i < n; ++i) level_cost(mc.nets[i], mc.mode, mc.nb[i], true, &launches, &seconds);
        pers = seconds < kPersistAutoSecondsPerLaunch * std::max(launches, 1.0);
    }
    for (int r = 0; r < R && pers; ++r) {
        WorkList W;
        for (int i = 0; i < n && pers; ++i) {
            const int b = mc.h_rb[(size_t)r * n + i];
            if (b < 1) continue;
            tnc_net* net = mc.nets[i];
            WorkList Wi;
            if (!wl_network(net, mc.arenas[i], mc.wss[i], b, mc.mode, r == 0, i, mc.outs[i], Wi)) {
                pers = false;
                break;
            }
            std::string why;
            const size_t ws_bytes = net->ws_user ? net->ws_user_bytes : net->ws_own_bytes;
            if (!wl_validate(net, Wi, mc.wss[i], ws_bytes, mc.outs[i], mc.mode, &why))
                return fail(TNC_E_STATE, "network " + std::to_string(i) + ": " + why);
            wl_append(W, Wi);
        }
        if (!pers) break;
        wl_interleave_levels(W);
        auto D = std::make_unique<DeviceWorkList>();
        if ((st = wl_upload(W, *D, mc.nets[0]->d_err, mc.nets[0]->persist_wait_ns, mc.nets[0]->tc_spin_limit, s)) !=
            TNC_OK)
            return st;
        mc.wls.push_back(std::move(D));
    }
    if (!pers) mc.wls.clear();
    return TNC_OK;
}

}  // namespace

// =================================================================== C ABI

extern "C" {

const char* tnc_last_error(void) { return g_err.c_str(); }

tnc_status tnc_create_network(int n_tensors, const int* ranks, const int64_t* const* index_ids,
                              int64_t n_indices, const int64_t* index_dims, const float* const* data_c64,
                              int n_open, const int64_t* open_ids, tnc_net_t* out) {
    if (!out) return fail(TNC_E_INVALID, "out is NULL");
    *out = nullptr;
    if (n_tensors < 1) return fail(TNC_E_INVALID, "n_tensors must be >= 1");
    if (n_indices < 0 || n_indices > (1ll << 30)) return fail(TNC_E_INVALID, "n_indices out of range");
    if (!ranks || !index_ids || !data_c64 || (n_indices > 0 && !index_dims))
        return fail(TNC_E_INVALID, "NULL argument");
    std::unique_ptr<tnc_net> net(new tnc_net());
    static uint64_t next_uid = 0;
    net->uid = ++next_uid;
    net->n_leaves = n_tensors;
    net->logd.assign(n_indices, 0);
    net->present.assign(n_indices, 0);
    for (int64_t e = 0; e < n_indices; ++e) {
        int64_t d = index_dims[e];
        if (d < 1 || (d & (d - 1))) return fail(TNC_E_INVALID, "index " + std::to_string(e) + " has a dimension that is not a power of two");
        net->logd[e] = 63 - __builtin_clzll((unsigned long long)d);
    }
    std::vector<int> count(n_indices, 0);
    for (int i = 0; i < n_tensors; ++i) {
        if (ranks[i] < 0) return fail(TNC_E_INVALID, "negative rank");
        if (ranks[i] > 0 && !index_ids[i]) return fail(TNC_E_INVALID, "NULL index list");
        std::vector<int64_t> idx(index_ids[i], index_ids[i] + ranks[i]);
        std::set<int64_t> seen;
        int bits = 0;
        for (int64_t e : idx) {
            if (e < 0 || e >= n_indices) return fail(TNC_E_INVALID, "index id out of range in tensor " + std::to_string(i));
            if (!seen.insert(e).second) return fail(TNC_E_INVALID, "index repeated within tensor " + std::to_string(i));
            count[e] += 1;
            net->present[e] = 1;
            bits += net->logd[e];
        }
        if (bits > 31) return fail(TNC_E_INVALID, "tensor " + std::to_string(i) + " exceeds 2^31 elements");
        net->leaf_idx.push_back(idx);
        net->leaf_off.push_back(net->total_leaf_elems);
        net->leaf_elems.push_back(1ll << bits);
        net->total_leaf_elems += 1ll << bits;
    }
    for (int64_t e = 0; e < n_indices; ++e)
        if (count[e] > 2) return fail(TNC_E_INVALID, "index " + std::to_string(e) + " joins more than two tensors");
    std::set<int64_t> open_set;
    if (n_open < 0 || (n_open > 0 && !open_ids)) return fail(TNC_E_INVALID, "bad open index list");
    for (int j = 0; j < n_open; ++j) {
        int64_t e = open_ids[j];
        if (e < 0 || e >= n_indices || count[e] != 1) return fail(TNC_E_INVALID, "open index " + std::to_string(e) + " must belong to exactly one tensor");
        if (!open_set.insert(e).second) return fail(TNC_E_INVALID, "open index repeated");
        net->open_ids.push_back(e);
    }
    for (int64_t e = 0; e < n_indices; ++e)
        if (count[e] == 1 && !open_set.count(e)) return fail(TNC_E_INVALID, "index " + std::to_string(e) + " belongs to one tensor but is not open");
    net->mode_base.assign(n_indices + 1, 0);
    for (int64_t e = 0; e < n_indices; ++e) net->mode_base[e + 1] = net->mode_base[e] + net->logd[e];
    net->host_leaves.resize(net->total_leaf_elems * 2);
    for (int i = 0; i < n_tensors; ++i) {
        if (!data_c64[i]) return fail(TNC_E_INVALID, "NULL tensor data");
        std::memcpy(net->host_leaves.data() + 2 * net->leaf_off[i], data_c64[i], net->leaf_elems[i] * 8);
    }
    *out = net.release();
    return TNC_OK;
}

tnc_status tnc_set_leaf_variants(tnc_net_t net, int n, const int* leaf_ids, int64_t n_variants,
                                 const float* const* data_c64) {
    if (!net) return fail(TNC_E_INVALID, "NULL network");
    if (n == 0) {  // back to ordinary leaves
        net->var_off.clear();
        net->host_var.clear();
        net->variant_bits = 0;
        net->n_variants = 0;
        net->plan.valid = false;
        net->inv_key.clear();
        return TNC_OK;
    }
    if (n < 0 || n > net->n_leaves || !leaf_ids || !data_c64) return fail(TNC_E_INVALID, "bad variant leaf list");
    if (n_variants < 1 || n_variants > (1ll << 24)) return fail(TNC_E_INVALID, "n_variants must be in [1, 2^24]");
    int m = 0;
    while ((1ll << m) < n_variants) ++m;
    std::vector<int64_t> off(net->n_leaves, -1);
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        const int leaf = leaf_ids[i];
        if (leaf < 0 || leaf >= net->n_leaves) return fail(TNC_E_INVALID, "variant leaf out of range");
        if (off[leaf] >= 0) return fail(TNC_E_INVALID, "variant leaf repeated");
        if (!data_c64[i]) return fail(TNC_E_INVALID, "NULL variant data");
        off[leaf] = total;
        total += net->leaf_elems[leaf] << m;
    }
    if (total > (1ll << 34)) return fail(TNC_E_INVALID, "variant data above 2^34 elements");
    std::vector<float> host((size_t)total * 2, 0.0f);  // copies past n_variants stay zero
    for (int i = 0; i < n; ++i) {
        const int leaf = leaf_ids[i];
        std::memcpy(host.data() + 2 * off[leaf], data_c64[i], (size_t)n_variants * net->leaf_elems[leaf] * 8);
    }
    net->var_off = std::move(off);
    net->host_var = std::move(host);
    net->variant_bits = m;
    net->n_variants = n_variants;
    net->var_dirty = true;
    net->plan.valid = false;
    net->inv_key.clear();
    return TNC_OK;
}

tnc_status tnc_contract_variants(tnc_net_t net, int64_t v_lo, int64_t v_hi, int64_t lo, int64_t hi, int mode,
                                 double* out_c128, void* stream) {
    if (!net) return fail(TNC_E_INVALID, "NULL network");
    if (!out_c128) return fail(TNC_E_INVALID, "NULL output");
    tnc_status st = ensure_plan(net);
    if (st != TNC_OK) return st;
    if (!net->n_variants) return fail(TNC_E_STATE, "no leaf variants (call tnc_set_leaf_variants)");
    if (v_lo < 0 || v_hi < v_lo || v_hi > net->n_variants) return fail(TNC_E_INVALID, "variant range out of bounds");
    const int sbits = (int)std::min<size_t>(net->S_sorted.size(), 62);
    const int64_t ns = 1ll << sbits;
    if (lo < 0 || hi < lo || hi > ns) return fail(TNC_E_INVALID, "slice range outside [0, 2^|S|]");
    const int64_t n_out = 1ll << net->plan.obits;
    // the slice-invariant tensors are computed by the first variant and kept
    // in the workspace for the others
    const int keep = net->cache_invariants;
    if (!keep) net->inv_key.clear();  // computed afresh by this call's first variant
    net->cache_invariants = 1;
    for (int64_t v = v_lo; v < v_hi && st == TNC_OK; ++v)
        st = tnc_contract(net, (v << sbits) + lo, (v << sbits) + hi, mode, out_c128 + 2 * (v - v_lo) * n_out, stream);
    net->cache_invariants = keep;
    return st;
}

tnc_status tnc_set_tensor_data(tnc_net_t net, int tensor, const float* data_c64) {
    if (!net || !data_c64) return fail(TNC_E_INVALID, "NULL argument");
    if (tensor < 0 || tensor >= net->n_leaves) return fail(TNC_E_INVALID, "tensor out of range");
    std::memcpy(net->host_leaves.data() + 2 * net->leaf_off[tensor], data_c64, net->leaf_elems[tensor] * 8);
    net->dev_dirty = true;
    net->leaf_version += 1;
    return TNC_OK;
}

tnc_status tnc_leaf_bytes(tnc_net_t net, size_t* bytes) {
    if (!net || !bytes) return fail(TNC_E_INVALID, "NULL argument");
    *bytes = (size_t)net->total_leaf_elems * 8;
    return TNC_OK;
}

tnc_status tnc_upload_leaves(tnc_net_t net, const float* packed, void* stream) {
    if (!net || !packed) return fail(TNC_E_INVALID, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    if (!net->d_leaves) CUDA_TRY(cudaMalloc(&net->d_leaves, std::max<int64_t>(8, net->total_leaf_elems * 8)));
    std::memcpy(net->host_leaves.data(), packed, net->total_leaf_elems * 8);
    CUDA_TRY(cudaMemcpyAsync(net->d_leaves, packed, net->total_leaf_elems * 8, cudaMemcpyHostToDevice, st));
    net->dev_dirty = false;
    net->leaf_version += 1;
    return TNC_OK;
}

tnc_status tnc_greedy_path(tnc_net_t net, int* pairs_out) {
    if (!net || (!pairs_out && net->n_leaves > 1)) return fail(TNC_E_INVALID, "NULL argument");
    try {
        auto p = tnc::greedy_path(net->leaf_idx, net->logd);
        for (size_t i = 0; i < p.size(); ++i) {
            pairs_out[2 * i] = p[i].first;
            pairs_out[2 * i + 1] = p[i].second;
        }
    } catch (const std::exception& e) {
        return fail(TNC_E_INVALID, e.what());
    }
    return TNC_OK;
}

tnc_status tnc_set_path(tnc_net_t net, int n_steps, const int* pairs) {
    if (!net) return fail(TNC_E_INVALID, "NULL network");
    if (n_steps != net->n_leaves - 1) return fail(TNC_E_INVALID, "path must have n_tensors - 1 steps");
    if (n_steps > 0 && !pairs) return fail(TNC_E_INVALID, "NULL pairs");
    std::vector<tnc::Pair> path;
    for (int i = 0; i < n_steps; ++i) path.emplace_back(pairs[2 * i], pairs[2 * i + 1]);
    try {
        auto tree = std::make_unique<tnc::Tree>(net->leaf_idx, net->logd, net->open_ids, path);
        for (int v = 0; v < tree->n_tensors(); ++v)
            if (tree->size_log(v) > 120) return fail(TNC_E_INVALID, "an intermediate tensor exceeds 2^120 elements");
        net->tree = std::move(tree);
    } catch (const std::exception& e) {
        return fail(TNC_E_INVALID, e.what());
    }
    net->path = path;
    net->S.clear();
    net->S_sorted.clear();
    net->plan.valid = false;
    return TNC_OK;
}

tnc_status tnc_find_slices(tnc_net_t net, int target_log2, uint64_t seed, double T0, double Tf, double alpha,
                           int64_t* out_ids, int* n_out, int cap) {
    if (!net || !n_out) return fail(TNC_E_INVALID, "NULL argument");
    if (!net->tree) return fail(TNC_E_STATE, "no contraction path set (call tnc_set_path)");
    if (T0 <= 0) T0 = 1.0;
    if (Tf <= 0) Tf = 1e-4;
    if (alpha <= 0 || alpha >= 1) alpha = 0.9;
    try {
        auto S1 = tnc::slice_finder(*net->tree, target_log2);
        auto S = tnc::slice_refiner(*net->tree, target_log2, S1, seed, T0, Tf, alpha);
        *n_out = (int)S.size();
        if ((int)S.size() > cap || (!out_ids && !S.empty()))
            return fail(TNC_E_INVALID, "out_ids capacity too small: need " + std::to_string(S.size()));
        for (size_t i = 0; i < S.size(); ++i) out_ids[i] = S[i];
    } catch (const std::exception& e) {
        return fail(TNC_E_INVALID, e.what());
    }
    return TNC_OK;
}

tnc_status tnc_set_slices(tnc_net_t net, int n, const int64_t* ids) {
    if (!net) return fail(TNC_E_INVALID, "NULL network");
    if (!net->tree) return fail(TNC_E_STATE, "no contraction path set (call tnc_set_path)");
    if (n < 0 || n > 120 || (n > 0 && !ids)) return fail(TNC_E_INVALID, "bad slice count");
    std::set<int64_t> seen;
    for (int j = 0; j < n; ++j) {
        int64_t e = ids[j];
        if (e < 0 || e >= (int64_t)net->logd.size() || !net->present[e]) return fail(TNC_E_INVALID, "sliced index " + std::to_string(e) + " not in the network");
        if (net->tree->is_open[e]) return fail(TNC_E_INVALID, "sliced index " + std::to_string(e) + " is open");
        if (net->logd[e] != 1) return fail(TNC_E_INVALID, "sliced index " + std::to_string(e) + " must have dimension 2");
        if (!seen.insert(e).second) return fail(TNC_E_INVALID, "sliced index repeated");
    }
    net->S.assign(ids, ids + n);
    net->S_sorted.assign(seen.begin(), seen.end());
    net->plan.valid = false;
    return TNC_OK;
}

tnc_status tnc_workspace_bytes(tnc_net_t net, int64_t max_batch, size_t* bytes) {
    if (!net || !bytes || max_batch < 1) return fail(TNC_E_INVALID, "bad argument");
    tnc_status st = ensure_plan(net);
    if (st != TNC_OK) return st;
    size_t b = 0;
    for (int mode = TNC_FP32; mode <= TNC_SPLIT_FP16X2; ++mode)
        b = std::max(b, (size_t)plan_arena(net, max_batch, mode).peak);
    *bytes = b;
    return TNC_OK;
}

tnc_status tnc_set_workspace(tnc_net_t net, void* dev_ptr, size_t bytes) {
    if (!net) return fail(TNC_E_INVALID, "NULL network");
    if (((uintptr_t)dev_ptr) % kAlign) return fail(TNC_E_INVALID, "workspace must be 256-byte aligned");
    net->ws_user = dev_ptr;
    net->ws_user_bytes = dev_ptr ? bytes : 0;
    net->inv_key.clear();
    return TNC_OK;
}

tnc_status tnc_contract(tnc_net_t net, int64_t lo, int64_t hi, int mode, double* out_c128, void* stream) {
    if (!net) return fail(TNC_E_INVALID, "NULL network");
    if (!out_c128) return fail(TNC_E_INVALID, "NULL output");
    if (mode < TNC_FP32 || mode > TNC_SPLIT_FP16X2) return fail(TNC_E_INVALID, "unknown mode");
    tnc_status st = ensure_plan(net);
    if (st != TNC_OK) return st;
    const int64_t n_slices = slice_space(net);
    if (lo < 0 || hi < lo || hi > n_slices)
        return fail(TNC_E_INVALID, "slice range outside [0, 2^(|S| + variant bits)]");
    cudaStream_t s = (cudaStream_t)stream;
    const Plan& P = net->plan;
    const int64_t R = 1ll << P.obits;
    CUDA_TRY(cudaMemsetAsync(out_c128, 0, R * 16, s));
    if (hi == lo) return TNC_OK;
    if ((st = ensure_leaves(net, s)) != TNC_OK) return st;

    // workspace and batch
    char* ws = nullptr;
    int64_t nb = 0;
    const int64_t want = hi - lo;
    if (net->ws_user) {
        nb = pick_batch(net, want, net->ws_user_bytes, mode);
        if (nb < 1) return fail(TNC_E_OOM, "workspace too small for one slice");
        ws = (char*)net->ws_user;
    } else {
        size_t one = (size_t)plan_arena(net, 1, mode).peak;
        size_t budget = std::max<size_t>(one, (size_t)1 << 30);
        nb = pick_batch(net, std::min<int64_t>(want, 1024), budget, mode);
        size_t need = (size_t)plan_arena(net, nb, mode).peak;
        if (net->ws_own_bytes < need) {
            if (net->ws_own) CUDA_TRY(cudaFree(net->ws_own));
            net->ws_own = nullptr;
            net->ws_own_bytes = 0;
            CUDA_TRY(cudaMalloc(&net->ws_own, std::max<size_t>(need, kAlign)));
            net->ws_own_bytes = need;
        }
        ws = (char*)net->ws_own;
    }
    net->last_batch = nb;
    const Arena ar = plan_arena(net, nb, mode);
    CUDA_TRY(cudaMemsetAsync(net->d_err, 0, sizeof(int), s));

    if ((st = ensure_groups(net, ar, ws, mode, nb, s)) != TNC_OK) return st;
    const std::string ikey = net->group_key + "|" + std::to_string(net->leaf_version);
    // persistent executor: one launch per batch of slices, the slice-invariant
    // contractions in the first one (unless cached). Every batch's work list is
    // prepared before the first launch, so a call that it cannot run falls back
    // to the launches below as a whole.
    bool use_persist = persist_eligible(net);
    if (use_persist && net->persistent == 2) {
        const bool inv_cached = net->cache_invariants && net->inv_key == ikey;
        double launches = 0, seconds = 0;
        level_cost(net, mode, nb, !inv_cached, &launches, &seconds);
        use_persist = seconds < kPersistAutoSecondsPerLaunch * std::max(launches, 1.0);
    }
    if (use_persist) {
        const bool inv_cached = net->cache_invariants && net->inv_key == ikey;
        std::vector<std::pair<DeviceWorkList*, int64_t>> rounds;
        bool ok = true;
        for (int64_t s0 = lo; s0 < hi && ok; s0 += nb) {
            const int b = (int)std::min<int64_t>(nb, hi - s0);
            DeviceWorkList* wl = contract_worklist(net, ar, ws, b, mode, s0 == lo && !inv_cached, out_c128, s, &st);
            if (st != TNC_OK) return st;
            if (!wl) ok = false;
            else rounds.emplace_back(wl, s0);
        }
        if (ok) {
            for (auto& [wl, s0] : rounds) {
                const int b = (int)std::min<int64_t>(nb, hi - s0);
                CUDA_TRY(timed_begin(net, -1, K_PERSIST, b, s, wl->cmacs));
                if (net->timing) net->timed_persist_tc_cmacs += wl->tc_cmacs;
                CUDA_TRY(wl_launch(*wl, mode, s0, nullptr, s, net->d_prof, out_c128));
                CUDA_TRY(timed_end(net, s));
            }
            net->inv_key = net->cache_invariants ? ikey : std::string();
            return TNC_OK;
        }
    }
    // invariant nodes once, one launch per level (or reused from an earlier
    // call when caching is on and nothing they depend on has changed)
    if (!(net->cache_invariants && net->inv_key == ikey)) {
        for (const Group& g : net->groups.inv)
            if ((st = run_group(net, ar, ws, g, 1, 0, mode, s)) != TNC_OK) return st;
        net->inv_key = net->cache_invariants ? ikey : std::string();
    }
    tnc::PermParams pp{};
    pp.obits = P.obits;
    for (int j = 0; j < P.obits; ++j) pp.ostride[j] = P.out_stride[j];
    double2* out = reinterpret_cast<double2*>(out_c128);

    for (int64_t s0 = lo; s0 < hi; s0 += nb) {
        const int b = (int)std::min<int64_t>(nb, hi - s0);
        if (P.nodes.empty()) {  // a single leaf: the result is the leaf itself
            tnc::SumParams sp{};
            sp.src = operand(net, ar, ws, 0, b);
            sp.obits = P.obits;
            for (int j = 0; j < P.obits; ++j) sp.ostride[j] = P.out_stride[j];
            sp.slice0 = s0;
            CUDA_TRY(timed_begin(net, 0, -1, b, s));
            CUDA_TRY(tnc::launch_slice_sum_f32(sp, b, out, s));
            CUDA_TRY(timed_end(net, s));
            continue;
        }
        for (const Group& g : net->groups.ps)
            if ((st = run_group(net, ar, ws, g, b, s0, mode, s)) != TNC_OK) return st;
        for (const NodePlan& np : P.nodes) {
            if (!np.is_root) continue;
            tnc::GemmParams g = gemm_params(net, ar, ws, np, b);
            g.slice0 = s0;
            CUDA_TRY(timed_begin(net, np.v, np.kind, b, s));
            if (np.kind == K_ROOT_F64) {
                tnc::RootParams rp{};
                rp.g = g;
                rp.chunks = np.chunks;
                double2* partials = reinterpret_cast<double2*>(ws + ar.root_scratch_off);
                CUDA_TRY(tnc::launch_root_partials(rp, b, partials, s));
                net->launches += 1;
                CUDA_TRY(tnc::launch_accumulate_partials(partials, b * np.chunks, pp, out, s));
            } else {
                float2* rootbuf = reinterpret_cast<float2*>(ws + ar.root_scratch_off);
                g.C = rootbuf;
                g.c_batch_stride = tensor_bytes(P, np.v) / 8;
                CUDA_TRY(tnc::launch_gemm_f32(g, b, s));
                net->launches += 1;
                tnc::SumParams sp{};
                sp.src.ptr = rootbuf;
                sp.src.batch_stride = g.c_batch_stride;
                sp.src.n_sl = 0;
                sp.obits = P.obits;
                for (int j = 0; j < P.obits; ++j) sp.ostride[j] = P.out_stride[j];
                sp.slice0 = s0;
                CUDA_TRY(tnc::launch_slice_sum_f32(sp, b, out, s));
            }
            CUDA_TRY(timed_end(net, s));
        }
    }
    return TNC_OK;
}

tnc_status tnc_autotune(tnc_net_t net, int mode, int64_t slice, void* stream) {
    if (!net) return fail(TNC_E_INVALID, "NULL network");
    if (mode == TNC_FP32) return TNC_OK;  // nothing to choose
    tnc_status st = ensure_plan(net);
    if (st != TNC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_slices = slice_space(net);
    if (slice < 0 || slice >= n_slices) return fail(TNC_E_INVALID, "slice out of range");
    bool any = false;  // nothing to choose without a tensor-core-eligible contraction
    for (const NodePlan& np : net->plan.nodes) any |= tc_node(mode, np.mb, np.nb, np.kb, np.is_root);
    if (!any) return TNC_OK;
    const int R = 1 << net->plan.obits;
    double* out = nullptr;
    CUDA_TRY(cudaMalloc(&out, (size_t)R * 16));
    // variants: the network's default row width (first), the other row width,
    // FP32 CUDA cores
    constexpr int NV = 3, kReps = 3;
    const int variants[NV] = {net->tc_row_bytes, net->tc_row_bytes == 64 ? 32 : 64, 0};
    std::map<int, std::array<double, kReps>> t[NV];  // per node and timed repeat: ms of all its launches
    const bool timing = net->timing;
    net->tuning = true;
    for (int vi = 0; vi < NV && st == TNC_OK; ++vi) {
        net->force_choice = variants[vi];
        for (int rep = 0; rep <= kReps && st == TNC_OK; ++rep) {  // run 0 warms up
            net->timing = true;
            net->timed.clear();
            st = tnc_contract(net, slice, slice + 1, mode, out, stream);
            if (st != TNC_OK) break;
            CUDA_TRY(cudaStreamSynchronize(s));
            if (rep > 0)
                for (const auto& r : net->timed) {
                    float ms = 0.f;
                    CUDA_TRY(cudaEventElapsedTime(&ms, net->ev_pool[r.ev], net->ev_pool[r.ev + 1]));
                    if (r.node >= net->n_leaves) t[vi][r.node][rep - 1] += ms;
                }
        }
    }
    net->force_choice = -1;
    net->tuning = false;
    net->timing = timing;
    net->timed.clear();
    cudaFree(out);
    if (st != TNC_OK) return st;
    // per shape: the sum over its nodes of each repeat, then the median repeat
    std::map<std::tuple<int, int, int, int>, std::array<std::array<double, kReps>, NV>> by_shape;
    for (const NodePlan& np : net->plan.nodes) {
        if (!tc_node(mode, np.mb, np.nb, np.kb, np.is_root)) continue;
        auto& acc = by_shape[std::make_tuple(mode, np.mb, np.nb, np.kb)];
        for (int vi = 0; vi < NV; ++vi)
            for (int r = 0; r < kReps; ++r) acc[vi][r] += t[vi][np.v][r];
    }
    // the default stays unless another variant is faster by kMargin: timings
    // of near-equal variants differ by noise, and a choice should not flip on it
    constexpr double kMargin = 0.03;
    for (auto& kv : by_shape) {
        double med[NV];
        for (int vi = 0; vi < NV; ++vi) {
            std::array<double, kReps> v = kv.second[vi];
            std::sort(v.begin(), v.end());
            med[vi] = v[kReps / 2];
        }
        int best = 0;
        for (int vi = 1; vi < NV; ++vi)
            if (med[vi] < (1.0 - kMargin) * med[0] && med[vi] < med[best]) best = vi;
        tune_table()[kv.first] = variants[best];
    }
    ++g_tune_version;
    net->group_key.clear();
    return TNC_OK;
}

tnc_status tnc_tune_table(char* json, size_t cap) {
    if (!json) return fail(TNC_E_INVALID, "NULL argument");
    std::ostringstream o;
    o << "[";
    bool first = true;
    for (auto& kv : tune_table()) {
        o << (first ? "" : ",") << "[" << std::get<0>(kv.first) << "," << std::get<1>(kv.first) << ","
          << std::get<2>(kv.first) << "," << std::get<3>(kv.first) << "," << kv.second << "]";
        first = false;
    }
    o << "]";
    std::string str = o.str();
    if (str.size() + 1 > cap) return fail(TNC_E_INVALID, "json capacity too small");
    std::memcpy(json, str.c_str(), str.size() + 1);
    return TNC_OK;
}

tnc_status tnc_check_device(tnc_net_t net, void* stream) {
    if (!net) return fail(TNC_E_INVALID, "NULL network");
    if (!net->d_err) return TNC_OK;
    int h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, net->d_err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    if (h == TNC_E_TIMEOUT) return fail(TNC_E_TIMEOUT, "a device-side wait gave up (tensor-core pipeline)");
    if (h) return fail(TNC_E_CUDA, "device error word " + std::to_string(h));
    return TNC_OK;
}

tnc_status tnc_set_option(tnc_net_t net, const char* key, int64_t value) {
    if (!net || !key) return fail(TNC_E_INVALID, "NULL argument");
    std::string k(key);
    if (k == "tc_row_bytes") {
        if (value != 32 && value != 64) return fail(TNC_E_INVALID, "tc_row_bytes must be 32 or 64");
        net->tc_row_bytes = (int)value;
    } else if (k == "tc_group_m") {
        if (value < 1 || value > 64) return fail(TNC_E_INVALID, "tc_group_m must be in [1, 64]");
        net->tc_group_m = (int)value;
    } else if (k == "backward_keep_every") {
        if (value < 0 || value > 64) return fail(TNC_E_INVALID, "backward_keep_every must be in [0, 64]");
        net->backward_keep_every = (int)value;
    } else if (k == "tc_plane_cap_log2") {
        if (value < 16 || value > 40) return fail(TNC_E_INVALID, "tc_plane_cap_log2 must be in [16, 40]");
        net->plane_cap_log2 = (int)value;
        net->group_key.clear();
    } else if (k == "persistent") {
        if (value < 0 || value > 2) return fail(TNC_E_INVALID, "persistent must be 0, 1 or 2");
        net->persistent = (int)value;
    } else if (k == "persist_wait_ms") {
        if (value < 0 || value > 600000) return fail(TNC_E_INVALID, "persist_wait_ms must be in [0, 600000]");
        net->persist_wait_ns = (uint64_t)value * 1000000ull;
    } else if (k == "persist_profile") {
        if (value != 0 && value != 1) return fail(TNC_E_INVALID, "persist_profile must be 0 or 1");
        if (value && !net->d_prof) {
            CUDA_TRY(cudaMalloc(&net->d_prof, tnc::kPersistProfWords * sizeof(unsigned long long)));
            CUDA_TRY(cudaMemset(net->d_prof, 0, tnc::kPersistProfWords * sizeof(unsigned long long)));
        } else if (!value && net->d_prof) {
            CUDA_TRY(cudaDeviceSynchronize());
            CUDA_TRY(cudaFree(net->d_prof));
            net->d_prof = nullptr;
        }
    } else if (k == "persist_test_stall") {
        net->persist_test_stall = value != 0;
    } else if (k == "stem_cap_log2") {
        // a group with a step that is not in place holds two buffers of
        // 2^value complex elements: 2 x 64 KB at 13 fits a CTA, 2 x 128 KB does not
        if (value != 0 && (value < 2 || value > tnc::kStemMaxInner - 1))
            return fail(TNC_E_INVALID, "stem_cap_log2 must be 0 or in [2, 13]");
        net->stem_cap_log2 = (int)value;
        net->plan.stem_cap = -1;
        net->group_key.clear();
        net->inv_key.clear();
    } else if (k == "stem_coalesce_bits") {
        if (value < 0 || value > 6) return fail(TNC_E_INVALID, "stem_coalesce_bits must be in [0, 6]");
        net->stem_coalesce_bits = (int)value;
        net->plan.stem_cap = -1;
        net->group_key.clear();
        net->inv_key.clear();
    } else if (k == "stem_min_outer_log2") {
        if (value < 0 || value > 30) return fail(TNC_E_INVALID, "stem_min_outer_log2 must be in [0, 30]");
        net->stem_min_outer = (int)value;
        net->plan.stem_cap = -1;
        net->group_key.clear();
        net->inv_key.clear();
    } else if (k == "cache_invariants") {
        net->cache_invariants = value != 0;
        net->inv_key.clear();
    } else if (k == "tc_spin_limit") {
        if (value < 0 || value > 0xFFFFFFFFll) return fail(TNC_E_INVALID, "tc_spin_limit out of range");
        net->tc_spin_limit = (uint32_t)value;
    } else if (k == "tc_test_stall") {
        net->tc_test_stall = value != 0;
    } else {
        return fail(TNC_E_INVALID, "unknown option " + k);
    }
    return TNC_OK;
}

tnc_status tnc_set_timing(tnc_net_t net, int enable) {
    if (!net) return fail(TNC_E_INVALID, "NULL network");
    net->timing = enable != 0;
    net->timed.clear();
    net->launches = 0;
    net->timed_persist_tc_cmacs = 0.0;
    if (net->d_prof) {
        CUDA_TRY(cudaDeviceSynchronize());
        CUDA_TRY(cudaMemset(net->d_prof, 0, tnc::kPersistProfWords * sizeof(unsigned long long)));
    }
    return TNC_OK;
}

tnc_status tnc_last_timings(tnc_net_t net, int* node, int* kind, int* batch, double* cmacs,
                            float* ms, int cap, int* n_out, int64_t* n_launches) {
    if (!net || !n_out) return fail(TNC_E_INVALID, "NULL argument");
    if (n_launches) *n_launches = net->launches;
    *n_out = (int)net->timed.size();
    if ((int)net->timed.size() > cap) return fail(TNC_E_INVALID, "capacity too small");
    for (size_t i = 0; i < net->timed.size(); ++i) {
        const auto& t = net->timed[i];
        float v = 0.f;
        CUDA_TRY(cudaEventSynchronize(net->ev_pool[t.ev + 1]));
        CUDA_TRY(cudaEventElapsedTime(&v, net->ev_pool[t.ev], net->ev_pool[t.ev + 1]));
        if (node) node[i] = t.node;
        if (kind) kind[i] = t.kind;
        if (batch) batch[i] = t.batch;
        if (ms) ms[i] = v;
        if (cmacs) cmacs[i] = t.cmacs;
    }
    return TNC_OK;
}

tnc_status tnc_contract_backward(tnc_net_t net, int64_t lo, int64_t hi, int mode, const double* grad_out_c128,
                                 float* grad_leaves_c64, const unsigned char* leaf_mask, size_t budget_bytes,
                                 void* stream) {
    if (!net) return fail(TNC_E_INVALID, "NULL network");
    if (!grad_out_c128 || !grad_leaves_c64) return fail(TNC_E_INVALID, "NULL gradient buffer");
    if (mode < TNC_FP32 || mode > TNC_SPLIT_FP16X2) return fail(TNC_E_INVALID, "unknown mode");
    tnc_status st = ensure_plan(net);
    if (st != TNC_OK) return st;
    if (net->variant_bits || net->n_variants)
        return fail(TNC_E_STATE, "the adjoint pass does not take leaf variants (tnc_set_leaf_variants)");
    const int64_t n_slices = 1ll << std::min<size_t>(net->S_sorted.size(), 62);
    if (lo < 0 || hi < lo || hi > n_slices) return fail(TNC_E_INVALID, "slice range outside [0, 2^|S|]");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_leaves(net, s)) != TNC_OK) return st;
    const tnc::Tree& T = *net->tree;
    Backward bw;
    bw.net = net;
    bw.mode = mode;
    bw.s = s;
    bw.needs.assign(T.n_tensors(), 0);
    for (int v = 0; v < net->n_leaves; ++v) bw.needs[v] = leaf_mask ? (leaf_mask[v] != 0) : 1;
    for (size_t i = 0; i < T.children.size(); ++i) {
        const int v = net->n_leaves + (int)i;
        bw.needs[v] = bw.needs[T.children[i].first] || bw.needs[T.children[i].second];
    }
    if (budget_bytes == 0) budget_bytes = (size_t)32 << 30;
    if (hi == lo) {
        CUDA_TRY(cudaMemsetAsync(grad_leaves_c64, 0, net->total_leaf_elems * 8, s));
        return TNC_OK;
    }
    // checkpoint spacing, then the largest slice batch, that fit the budget (dry runs)
    int keep_every = 1;
    auto need_for = [&](int64_t nb) {
        Backward d = bw;
        d.exec = false;
        d.nb = nb;
        d.keep_every = keep_every;
        backward_run(d, lo, std::min(hi, lo + nb), grad_out_c128);
        return (size_t)d.A.top;
    };
    int64_t nb = 1;
    if (net->backward_keep_every > 0) keep_every = net->backward_keep_every;
    else
        while (need_for(1) > budget_bytes && keep_every < 64) keep_every *= 2;
    if (need_for(1) > budget_bytes)
        return fail(TNC_E_OOM, "backward workspace for one slice exceeds the budget (" +
                                   std::to_string(need_for(1)) + " bytes)");
    net->last_keep_every = keep_every;
    int64_t hi_b = std::min<int64_t>(hi - lo, 1024);
    while (nb < hi_b) {
        int64_t nx = std::min<int64_t>(nb * 2, hi_b);
        if (need_for(nx) > budget_bytes) break;
        nb = nx;
    }
    const size_t need = need_for(nb);
    net->last_backward_bytes = need;
    char* ws = nullptr;
    if (net->ws_user && net->ws_user_bytes >= need) {
        ws = (char*)net->ws_user;
    } else {
        if (net->ws_own_bytes < need) {
            if (net->ws_own) CUDA_TRY(cudaFree(net->ws_own));
            net->ws_own = nullptr;
            net->ws_own_bytes = 0;
            CUDA_TRY(cudaMalloc(&net->ws_own, need));
            net->ws_own_bytes = need;
        }
        ws = (char*)net->ws_own;
    }
    net->last_batch = nb;
    net->group_key.clear();  // the workspace may now hold other data
    net->inv_key.clear();
    CUDA_TRY(cudaMemsetAsync(net->d_err, 0, sizeof(int), s));
    bw.exec = true;
    bw.nb = nb;
    bw.ws = ws;
    bw.keep_every = keep_every;
    if ((st = backward_run(bw, lo, hi, grad_out_c128)) != TNC_OK) return st;
    CUDA_TRY(tnc::launch_f64_to_f32(reinterpret_cast<const double2*>(ws + bw.leaf_grad), net->total_leaf_elems,
                                    reinterpret_cast<float2*>(grad_leaves_c64), s));
    net->launches += 1;
    return TNC_OK;
}

tnc_status tnc_param_grads(tnc_net_t net, int n_params, const int* leaf_ids, const float* dleaf_c64,
                           const float* env_packed_c64, double* out_c128, void* stream) {
    if (!net) return fail(TNC_E_INVALID, "NULL network");
    if (n_params < 0 || (n_params > 0 && (!leaf_ids || !dleaf_c64 || !env_packed_c64 || !out_c128)))
        return fail(TNC_E_INVALID, "bad argument");
    if (n_params == 0) return TNC_OK;
    std::vector<int64_t> host(3 * (size_t)n_params);
    int64_t doff = 0;
    for (int q = 0; q < n_params; ++q) {
        const int l = leaf_ids[q];
        if (l < 0 || l >= net->n_leaves) return fail(TNC_E_INVALID, "leaf id out of range");
        host[q] = net->leaf_off[l];
        host[n_params + q] = doff;
        host[2 * n_params + q] = net->leaf_elems[l];
        doff += net->leaf_elems[l];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = host.size() * sizeof(int64_t);
    if (net->pg_cap < bytes) {
        if (net->d_pg) CUDA_TRY(cudaFree(net->d_pg));
        net->d_pg = nullptr;
        net->pg_cap = 0;
        CUDA_TRY(cudaMalloc(&net->d_pg, bytes));
        net->pg_cap = bytes;
    }
    CUDA_TRY(cudaMemcpyAsync(net->d_pg, host.data(), bytes, cudaMemcpyHostToDevice, s));
    CUDA_TRY(tnc::launch_param_grads(n_params, net->d_pg, net->d_pg + n_params, net->d_pg + 2 * n_params,
                                     reinterpret_cast<const float2*>(env_packed_c64),
                                     reinterpret_cast<const float2*>(dleaf_c64),
                                     reinterpret_cast<double2*>(out_c128), s));
    CUDA_TRY(cudaStreamSynchronize(s));  // the staged offsets above are host memory
    return TNC_OK;
}


tnc_status tnc_contract_many(int n, const tnc_net_t* nets, const int64_t* slice_lo, const int64_t* slice_hi,
                             int mode, double* const* outs_c128, int use_graph, void* stream) {
    if (n < 1 || !nets || !slice_lo || !slice_hi || !outs_c128) return fail(TNC_E_INVALID, "bad argument");
    if (mode < TNC_FP32 || mode > TNC_SPLIT_FP16X2) return fail(TNC_E_INVALID, "unknown mode");
    cudaStream_t s = (cudaStream_t)stream;
    std::ostringstream key;
    key << mode << ":" << use_graph << ":" << (uintptr_t)s;
    for (int i = 0; i < n; ++i) {
        tnc_net* net = nets[i];
        if (!net) return fail(TNC_E_INVALID, "NULL network");
        if (!outs_c128[i]) return fail(TNC_E_INVALID, "NULL output");
        tnc_status st = ensure_plan(net);
        if (st != TNC_OK) return st;
        const int64_t ns = slice_space(net);
        if (slice_lo[i] < 0 || slice_hi[i] < slice_lo[i] || slice_hi[i] > ns)
            return fail(TNC_E_INVALID, "slice range of network " + std::to_string(i) +
                                           " outside [0, 2^(|S| + variant bits)]");
        for (int j = 0; j < i; ++j)
            if (nets[j] == net) return fail(TNC_E_INVALID, "a network appears twice");
        key << "|" << net->uid << ":" << net->plan.version << ":" << slice_lo[i] << ":" << slice_hi[i] << ":"
            << (uintptr_t)outs_c128[i] << ":" << (uintptr_t)net->ws_user << ":" << net->ws_user_bytes << ":"
            << net->persistent << ":" << net->persist_wait_ns << ":" << net->plane_cap_log2 << ":" << g_tune_version
            << ":" << net->force_choice << ":" << net->tc_group_m << ":" << net->tc_spin_limit << ":"
            << net->tc_row_bytes << ":" << (uintptr_t)net->d_prof;
    }
    tnc_status st;
    // device copies of leaf data must be current before a cached sequence replays
    for (int i = 0; i < n; ++i)
        if ((st = ensure_leaves(nets[i], s)) != TNC_OK) return st;
    auto& cache = many_cache();
    auto it = cache.find(key.str());
    if (it != cache.end()) {
        // a network's own workspace may have been reallocated by a later call
        // of its own: the cached sequence addresses the old one
        for (int i = 0; i < n && it != cache.end(); ++i) {
            const tnc_net* net = nets[i];
            const char* cur = static_cast<const char*>(net->ws_user ? net->ws_user : net->ws_own);
            if (cur != it->second->wss[i]) {
                cache.erase(it);
                it = cache.end();
            }
        }
    }
    ManyCall* mc = nullptr;
    if (it == cache.end()) {
        if (cache.size() >= 8) cache.clear();
        auto fresh = std::make_unique<ManyCall>();
        fresh->mode = mode;
        for (int i = 0; i < n; ++i) {
            fresh->nets.push_back(nets[i]);
            fresh->uids.push_back(nets[i]->uid);
            fresh->lo.push_back(slice_lo[i]);
            fresh->hi.push_back(slice_hi[i]);
            fresh->outs.push_back(outs_c128[i]);
        }
        if ((st = many_build(*fresh, s)) != TNC_OK) return st;
        mc = fresh.get();
        cache[key.str()] = std::move(fresh);
    } else {
        mc = it->second.get();
    }
    const bool graph = use_graph && s != nullptr;
    // the first run of a sequence is eager: one-time set-up (kernel attributes,
    // driver entry points) never happens inside a capture
    if (!graph || !mc->warmed) {
        mc->warmed = true;
        // the call's kernels are counted on the first network, as for a replay
        std::vector<int64_t> before(n);
        for (int i = 0; i < n; ++i) before[i] = nets[i]->launches;
        st = many_run(*mc, s);
        for (int i = 0; i < n; ++i) nets[i]->launches = before[i];
        nets[0]->launches += mc->kernels;
        return st;
    }
    if (!mc->graph) {
        cudaGraph_t g = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        std::vector<bool> timing(n);
        for (int i = 0; i < n; ++i) {
            timing[i] = nets[i]->timing;
            nets[i]->timing = false;  // no event records inside the graph
        }
        tnc_status rst = many_run(*mc, s);
        for (int i = 0; i < n; ++i) nets[i]->timing = timing[i];
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (rst != TNC_OK) {
            if (g) cudaGraphDestroy(g);
            return rst;
        }
        if (e != cudaSuccess) return fail(TNC_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&mc->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(TNC_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    CUDA_TRY(cudaGraphLaunch(mc->graph, s));
    nets[0]->launches += mc->kernels;
    return TNC_OK;
}

tnc_status tnc_stats(tnc_net_t net, char* json, size_t cap) {
    if (!net || !json) return fail(TNC_E_INVALID, "NULL argument");
    if (!net->tree) return fail(TNC_E_STATE, "no contraction path set (call tnc_set_path)");
    const tnc::Tree& T = *net->tree;
    std::ostringstream o;
    tnc::Wide e1 = T.eq1(), e3 = T.eq3(net->S);
    o << "{\"n_leaves\":" << net->n_leaves << ",\"n_nodes\":" << T.children.size();
    o << ",\"eq1\":\"" << e1.to_string() << "\",\"eq3\":\"" << e3.to_string() << "\"";
    o << ",\"overhead\":" << (e3.to_double() / e1.to_double());
    o << ",\"sliced\":[";
    for (size_t i = 0; i < net->S.size(); ++i) o << (i ? "," : "") << net->S[i];
    o << "]";
    std::vector<char> sl(T.logd.size(), 0);
    for (int64_t e : net->S) sl[e] = 1;
    int w = 0;
    for (int v = 0; v < T.n_tensors(); ++v) w = std::max(w, T.dim(v, sl));
    o << ",\"max_log2_size\":" << w;
    std::string perr;
    if (!net->plan.valid) {
        try {
            build_plan(net);
        } catch (const std::exception& e) {
            perr = e.what();
        }
    }
    if (net->plan.valid) {
        o << ",\"workspace_batch1\":" << plan_arena(net, 1, TNC_FP32).peak;
        o << ",\"last_batch\":" << net->last_batch;
        o << ",\"backward_keep_every\":" << net->last_keep_every;
        o << ",\"backward_workspace\":" << net->last_backward_bytes;
        o << ",\"nodes\":[";
        bool first = true;
        for (const NodePlan& np : net->plan.nodes) {
            o << (first ? "" : ",") << "[" << np.mb << "," << np.nb << "," << np.kb << ","
              << (np.per_slice ? 1 : 0) << "," << np.kind << "]";
            first = false;
        }
        o << "]";
        // how each tensor-core-eligible contraction is cut up in the split
        // modes, for the last batch size (1 before any call)
        const int64_t cb = net->last_batch > 0 ? net->last_batch : 1;
        o << ",\"tc_cut_batch\":" << cb << ",\"tc_cuts\":{";
        const int cut_modes[4] = {TNC_SPLIT_TF32, TNC_SPLIT_BF16, TNC_SPLIT_BF16X2, TNC_SPLIT_FP16X2};
        for (int mi = 0; mi < 4; ++mi) {
            const int mode = cut_modes[mi];
            o << (mi ? "," : "") << "\"" << mode << "\":[";
            bool f2 = true;
            for (size_t i = 0; i < net->plan.nodes.size(); ++i) {
                const NodePlan& np = net->plan.nodes[i];
                if (!tc_node(mode, np.mb, np.nb, np.kb, np.is_root)) continue;
                const TcCut c = tc_cut(net, mode, np.mb, np.nb, np.kb, np.per_slice ? cb : 1);
                o << (f2 ? "" : ",") << "[" << i << "," << c.pA << "," << c.pB << "," << c.pK << "," << c.ks << "]";
                f2 = false;
            }
            o << "]";
        }
        o << "}";
        // fused stem groups for the current cap: [first node, steps, outer bits, inner bits, per slice]
        if (net->plan.stem_cap != net->stem_cap_log2) plan_stems(net);
        o << ",\"stem_cap_log2\":" << net->stem_cap_log2 << ",\"stem_groups\":[";
        for (size_t gi = 0; gi < net->plan.stems.size(); ++gi) {
            const StemGroupPlan& g = net->plan.stems[gi];
            o << (gi ? "," : "") << "[" << g.steps.front() << "," << g.steps.size() << "," << g.U.size() << ","
              << g.max_inner << "," << (g.per_slice ? 1 : 0) << "," << net->plan.layout[g.in].size() << ","
              << net->plan.layout[g.out].size() << "]";
        }
        o << "]";
    } else {
        o << ",\"plan_error\":\"" << perr << "\"";
    }
    o << ",\"persistent\":" << net->persistent << ",\"timed_persist_tc_cmacs\":" << std::setprecision(17)
      << net->timed_persist_tc_cmacs;
    if (net->d_prof) {  // [run ns, tasks, wait ns] per task type since tnc_set_timing
        unsigned long long h[tnc::kPersistProfWords];
        if (cudaDeviceSynchronize() == cudaSuccess &&
            cudaMemcpy(h, net->d_prof, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess) {
            o << ",\"persist_profile\":[";
            for (int t = 0; t < tnc::kPersistProfWords / 3; ++t)
                o << (t ? "," : "") << "[" << h[3 * t] << "," << h[3 * t + 1] << "," << h[3 * t + 2] << "]";
            o << "]";
        }
    }
    o << "}";
    std::string s = o.str();
    if (s.size() + 1 > cap) return fail(TNC_E_INVALID, "json capacity too small: need " + std::to_string(s.size() + 1));
    std::memcpy(json, s.c_str(), s.size() + 1);
    return TNC_OK;
}

void tnc_destroy(tnc_net_t net) {
    if (!net) return;
    many_forget(net->uid);
    delete net;
}

}  // extern "C"
