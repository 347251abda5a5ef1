// C ABI of libtnc (declared in include/tnc.h), except the adjoint entry
// points (host_backward.cpp) and tnc_contract_many (host_many.cpp).
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
// host by a first-fit simulation of the tensors' lifetimes (host_plan.cpp).
// A launch-bound call runs each batch as one persistent launch instead
// (host_persist.cpp).
#include "host.hpp"

#include <iomanip>
#include <sstream>

void tnc::set_last_error(const std::string& msg) { g_err = msg; }

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
    CUDA_TRY(cudaMemsetAsync(net->d_err, 0, sizeof(int), s));

    // persistent executor: one launch per batch of slices, the slice-invariant
    // contractions in the first one (unless cached). Its tasks wait only on
    // their own inputs when the arena without memory reuse fits: the given
    // workspace, or an own one of at most the larger of 1 GiB and what the
    // reusing arena needs.
    bool use_persist = persist_eligible(net);
    Arena ar_flat;
    bool deps = false;
    net->last_arena_bytes[0] = (size_t)plan_arena(net, nb, mode).peak;
    net->last_arena_bytes[1] = 0;
    net->last_persist_deps = false;
    if (use_persist && net->persist_deps) {
        ar_flat = plan_arena(net, nb, mode, false);
        net->last_arena_bytes[1] = (size_t)ar_flat.peak;
        const size_t cap = net->ws_user ? net->ws_user_bytes : std::max<size_t>(net->last_arena_bytes[0], (size_t)1 << 30);
        deps = (size_t)ar_flat.peak <= cap;
    }
    const bool grow = deps && !net->ws_user && net->ws_own_bytes < (size_t)ar_flat.peak;
    if (use_persist && net->persistent == 2) {
        const std::string k = group_key_of(net, mode, nb, ws, !deps) + "|" + std::to_string(net->leaf_version);
        const bool inv_cached = !grow && net->cache_invariants && net->inv_key == k;
        double launches = 0, seconds = 0;
        level_cost(net, mode, nb, !inv_cached, &launches, &seconds);
        use_persist = seconds < kPersistAutoSecondsPerLaunch * std::max(launches, 1.0);
    }
    deps = deps && use_persist;
    if (deps && grow) {  // a failed allocation keeps the reusing arena
        void* p = nullptr;
        if (cudaMalloc(&p, (size_t)ar_flat.peak) == cudaSuccess) {
            if (net->ws_own) CUDA_TRY(cudaFree(net->ws_own));
            net->ws_own = p;
            net->ws_own_bytes = (size_t)ar_flat.peak;
            ws = (char*)net->ws_own;
        } else {
            (void)cudaGetLastError();
            deps = false;
        }
    }
    const Arena ar = deps ? ar_flat : plan_arena(net, nb, mode);

    if ((st = ensure_groups(net, ar, ws, mode, nb, s)) != TNC_OK) return st;
    const std::string ikey = net->group_key + "|" + std::to_string(net->leaf_version);
    // Every batch's work list is prepared before the first launch, so a call
    // that the persistent executor cannot run falls back to the launches
    // below as a whole.
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
            net->last_persist_deps = deps;
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
    } else if (k == "persist_deps") {
        if (value != 0 && value != 1) return fail(TNC_E_INVALID, "persist_deps must be 0 or 1");
        net->persist_deps = (int)value;
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
        // the automatic executor choice's estimate for that batch, invariants
        // included: [per-level launches, estimated seconds] per mode
        o << ",\"level_cost\":{";
        for (int mode = TNC_FP32; mode <= TNC_SPLIT_FP16X2; ++mode) {
            double launches = 0, seconds = 0;
            level_cost(net, mode, cb, true, &launches, &seconds);
            o << (mode ? "," : "") << "\"" << mode << "\":[" << launches << "," << seconds
              << "]";
        }
        o << "}";
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
    o << ",\"persistent\":" << net->persistent << ",\"persist_deps\":" << net->persist_deps
      << ",\"last_persist_deps\":" << (net->last_persist_deps ? 1 : 0) << ",\"last_workspace\":["
      << net->last_arena_bytes[0] << "," << net->last_arena_bytes[1] << "],\"timed_persist_tc_cmacs\":" << std::setprecision(17)
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

// Work list of networks nets[0..n) for one batch each, as the persistent
// executor would run it in one launch (one network: as tnc_contract; several:
// merged and interleaved by level as tnc_contract_many), built against
// stand-in workspaces, then written as JSON.
static tnc_status worklist_json(int n, const tnc_net_t* nets, int64_t batch, int mode, int deps, char* json,
                                size_t cap) {
    if (n < 1 || !nets || !json) return fail(TNC_E_INVALID, "bad argument");
    if (mode < TNC_FP32 || mode > TNC_SPLIT_FP16X2) return fail(TNC_E_INVALID, "unknown mode");
    if (batch < 1 || batch > 1024) return fail(TNC_E_INVALID, "batch must be in [1, 1024]");
    if (deps != 0 && deps != 1) return fail(TNC_E_INVALID, "deps must be 0 or 1");
    WorkList W;
    for (int i = 0; i < n; ++i) {
        tnc_net* net = nets[i];
        if (!net) return fail(TNC_E_INVALID, "NULL network");
        for (int j = 0; j < i; ++j)
            if (nets[j] == net) return fail(TNC_E_INVALID, "a network appears twice");
        tnc_status st = ensure_plan(net);
        if (st != TNC_OK) return st;
        if (net->plan.nodes.empty() || (stem_fusion(net) && !net->plan.stems.empty()) || net->tuning)
            return fail(TNC_E_STATE, "the persistent executor does not run network " + std::to_string(i) +
                                         " (fused stem groups in use?)");
        // the list addresses an arena at a stand-in base: nothing is read or written
        const Arena ar = plan_arena(net, batch, mode, deps == 0);
        char* const base = reinterpret_cast<char*>(uintptr_t(i + 1) << 40);
        WorkList Wi;
        if (!wl_network(net, ar, base, (int)batch, mode, true, i, nullptr, Wi))
            return fail(TNC_E_STATE, "no work list for network " + std::to_string(i) +
                                         ": a contraction needs panels, or tensor maps need the CUDA driver");
        if (n == 1) W = std::move(Wi);
        else wl_append(W, Wi);
    }
    wl_interleave_levels(W);
    std::ostringstream o;
    o << "{\"chain\":" << (deps ? 0 : 1) << ",\"counters\":[";
    for (size_t i = 0; i < W.counters.size(); ++i) o << (i ? "," : "") << W.counters[i];
    o << "],\"tasks\":[";
    for (size_t i = 0; i < W.tasks.size(); ++i) {
        const tnc::PersistTask& t = W.tasks[i];
        o << (i ? "," : "") << "[" << t.type << "," << t.idx << "," << t.item << "," << t.z << "," << t.wait[0]
          << "," << t.wait[1] << "," << t.wait[2] << "," << t.signal << "," << t.signal2 << "," << W.level[i] << ","
          << t.net << "]";
    }
    o << "]}";
    const std::string js = o.str();
    if (js.size() + 1 > cap) return fail(TNC_E_INVALID, "json capacity too small: need " + std::to_string(js.size() + 1));
    std::memcpy(json, js.c_str(), js.size() + 1);
    return TNC_OK;
}

tnc_status tnc_arena_json(tnc_net_t net, int64_t batch, int mode, int reuse, char* json, size_t cap) {
    if (!net || !json) return fail(TNC_E_INVALID, "NULL argument");
    if (mode < TNC_FP32 || mode > TNC_SPLIT_FP16X2) return fail(TNC_E_INVALID, "unknown mode");
    if (batch < 1 || batch > 1024) return fail(TNC_E_INVALID, "batch must be in [1, 1024]");
    if (reuse != 0 && reuse != 1) return fail(TNC_E_INVALID, "reuse must be 0 or 1");
    tnc_status st = ensure_plan(net);
    if (st != TNC_OK) return st;
    std::vector<ArenaEvent> log;
    const Arena ar = plan_arena_log(net, batch, mode, reuse == 1, &log);
    std::ostringstream o;
    o << "{\"peak\":" << ar.peak << ",\"events\":[";
    for (size_t i = 0; i < log.size(); ++i) {
        const ArenaEvent& e = log[i];
        o << (i ? "," : "") << "[" << e.op << "," << e.kind << "," << e.id << "," << e.off << "," << e.len << ","
          << e.step << "]";
    }
    o << "]}";
    const std::string js = o.str();
    if (js.size() + 1 > cap) return fail(TNC_E_INVALID, "json capacity too small: need " + std::to_string(js.size() + 1));
    std::memcpy(json, js.c_str(), js.size() + 1);
    return TNC_OK;
}

tnc_status tnc_worklist_json(tnc_net_t net, int64_t batch, int mode, int deps, char* json, size_t cap) {
    if (!net) return fail(TNC_E_INVALID, "NULL network");
    return worklist_json(1, &net, batch, mode, deps, json, cap);
}

tnc_status tnc_worklist_many_json(int n, const tnc_net_t* nets, int64_t batch, int mode, int deps, char* json,
                                  size_t cap) {
    return worklist_json(n, nets, batch, mode, deps, json, cap);
}

void tnc_destroy(tnc_net_t net) {
    if (!net) return;
    many_forget(net->uid);
    delete net;
}

}  // extern "C"
