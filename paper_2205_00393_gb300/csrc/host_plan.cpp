// Host side of libtnc: the contraction plan (binary modes, per-bit strides,
// per-slice classification), fused stem groups, tensor-core cuts, the
// workspace arena, level groups and the per-level launches.
#include "host.hpp"

namespace tnc_host {


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

static Arena plan_arena_uncached(const tnc_net* net, int64_t nb, int mode, bool reuse,
                                 std::vector<ArenaEvent>* log = nullptr);

// Everything the level groups and the arena of a batch of nb slices depend
// on: the plan, the kernel choices and the options that shape groups and
// tensor-core temporaries. Key of the host-side caches below.
std::string plan_key(const tnc_net* net, int mode, int64_t nb) {
    return std::to_string(mode) + ":" + std::to_string(nb) + ":" + std::to_string(net->plan.version) + ":" +
           std::to_string(g_tune_version) + ":" + std::to_string(net->force_choice) + ":" +
           std::to_string(net->tc_row_bytes) + ":" + std::to_string(net->tuning ? 1 : 0) + ":" +
           std::to_string(net->in_many ? 1 : 0) + ":" + std::to_string(net->stem_cap_log2) + ":" +
           std::to_string(net->plan.stem_cap) + ":" + std::to_string(net_plane_cap_log2(net));
}

// First-fit simulation of the workspace for a batch of `nb` slices, cached
// by plan_key.
Arena plan_arena(const tnc_net* net, int64_t nb, int mode, bool reuse) {
    const std::string key = plan_key(net, mode, nb) + (reuse ? ":r" : ":f");
    auto it = net->arena_cache.find(key);
    if (it != net->arena_cache.end()) return it->second;
    if (net->arena_cache.size() >= 64) net->arena_cache.clear();
    return net->arena_cache[key] = plan_arena_uncached(net, nb, mode, reuse);
}

static Arena plan_arena_uncached(const tnc_net* net, int64_t nb, int mode, bool reuse,
                                 std::vector<ArenaEvent>* log) {
    const Plan& P = net->plan;
    const tnc::Tree& T = *net->tree;
    Arena ar;
    ar.off.assign(T.n_tensors(), -1);
    ar.planes_a.assign(P.nodes.size(), -1);
    ar.planes_b.assign(P.nodes.size(), -1);
    std::map<int64_t, int64_t> used;  // off -> len
    int64_t top = 0;
    int step = 0;  // level being simulated (for the optional event log)
    auto alloc = [&](int64_t len, int kind, int id) {
        len = align_up(len);
        int64_t prev_end = 0;
        for (auto& kv : used) {
            if (kv.first - prev_end >= len) break;
            prev_end = kv.first + kv.second;
        }
        int64_t off = prev_end;
        used[off] = len;
        top = std::max(top, off + len);
        if (log) log->push_back(ArenaEvent{0, kind, id, off, len, step});
        return off;
    };
    // without reuse every tensor and temporary keeps its bytes for the whole
    // launch, so tasks of different levels may run at the same time
    auto release = [&](int64_t off, int kind, int id) {
        if (!reuse) return;
        auto it = used.find(off);
        if (it == used.end()) return;
        if (log) log->push_back(ArenaEvent{1, kind, id, off, it->second, step});
        used.erase(it);
    };
    auto tc_planes = [&](const NodePlan& np, int64_t b) {
        const size_t i = np.v - net->n_leaves;
        ar.planes_a[i] = alloc(tc_bytes_a(net, mode, np.mb, np.nb, np.kb, b), 1, np.v);
        ar.planes_b[i] = alloc(tc_bytes_b(net, mode, np.mb, np.nb, np.kb, b), 2, np.v);
    };
    auto tc_release = [&](const NodePlan& np) {
        const size_t i = np.v - net->n_leaves;
        release(ar.planes_a[i], 1, np.v);
        release(ar.planes_b[i], 2, np.v);
    };
    // Lifetimes follow the executed order: one tree level at a time; all
    // outputs of a level are live together, inputs die after their level.
    auto run_level = [&](const Group& g, int64_t b) {
        for (int v : g.fp32) ar.off[v] = alloc(b * tensor_bytes(P, v), 0, v);
        for (int v : g.tc) ar.off[v] = alloc(b * tensor_bytes(P, v), 0, v);
        // fused stem groups: only T_n is stored; T_1 .. T_{n-1} stay on chip
        for (int gi : g.stems)
            ar.off[P.stems[gi].out] = alloc(b * tensor_bytes(P, P.stems[gi].out), 0, P.stems[gi].out);
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
                    if (c >= net->n_leaves && P.per_slice[c] == (char)g.per_slice) release(ar.off[c], 0, c);
            }
        for (int gi : g.stems) {
            const StemGroupPlan& sg = P.stems[gi];
            std::vector<int> ins{sg.in};
            for (int k : sg.steps) ins.push_back(P.nodes[k].B);
            for (int c : ins)
                if (c >= net->n_leaves && P.per_slice[c] == (char)g.per_slice) release(ar.off[c], 0, c);
        }
        ++step;
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
        ar.root_scratch_off = alloc(bytes, 3, np.v);
    }
    ar.peak = top;
    ar.batch = nb;
    ar.reuse = reuse;
    return ar;
}

// plan_arena's simulation with its events recorded (not cached).
Arena plan_arena_log(const tnc_net* net, int64_t nb, int mode, bool reuse, std::vector<ArenaEvent>* log) {
    return plan_arena_uncached(net, nb, mode, reuse, log);
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

cudaError_t timed_begin(tnc_net* net, int node, int kind, int batch, cudaStream_t s, double cmacs) {
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
// Key of the launch groups (and persistent work lists) of a call: they address
// the workspace at the offsets of its arena.
std::string group_key_of(const tnc_net* net, int mode, int64_t nb, const char* ws, bool reuse) {
    return std::to_string(mode) + ":" + std::to_string(nb) + ":" + std::to_string((uintptr_t)ws) + ":" +
           std::to_string(net->plan.version) + ":" + std::to_string(g_tune_version) + ":" +
           std::to_string(net->force_choice) + ":" + std::to_string(net->tuning ? 1 : 0) + ":" +
           std::to_string(stem_fusion(net) ? net->stem_cap_log2 : 0) + ":" + std::to_string(net->plane_cap_log2) +
           ":" + std::to_string(reuse ? 1 : 0);
}

tnc_status ensure_groups(tnc_net* net, const Arena& ar, char* ws, int mode, int64_t nb, cudaStream_t s) {
    const std::string key = group_key_of(net, mode, nb, ws, ar.reuse);
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



}  // namespace tnc_host
