// Host side of the adjoint pass (tnc_contract_backward) and the gate-parameter
// chain rule (tnc_param_grads).
#include "host.hpp"

namespace tnc_host {

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



}  // namespace tnc_host

extern "C" {

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


}  // extern "C"
