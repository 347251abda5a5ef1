// Host side of tnc_contract_many: many networks in merged level launches or
// one persistent launch per round, captured into a CUDA graph.
#include "host.hpp"

namespace tnc_host {

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
    }
    // persistent executor when every network has it on: forced, or the
    // automatic choice over the whole call
    bool pers = true, forced = true;
    for (tnc_net* net : mc.nets) {
        pers &= net->persistent != 0;
        forced &= net->persistent == 1;
    }
    if (pers && !forced) {
        double launches = 0, seconds = 0;
        for (int i = 0; i < n; ++i) level_cost(mc.nets[i], mc.mode, mc.nb[i], true, &launches, &seconds);
        pers = seconds < kPersistAutoSecondsPerLaunch * std::max(launches, 1.0);
    }
    for (int i = 0; i < n; ++i) {
        tnc_net* net = mc.nets[i];
        const int64_t nb = mc.nb[i];
        // a network whose tensors all fit at once (its own workspace of at most
        // the larger of 256 MiB and the reusing layout) takes per-entry
        // dependencies in the persistent lists
        Arena ar = plan_arena(net, nb, mc.mode);
        net->last_arena_bytes[0] = (size_t)ar.peak;
        net->last_arena_bytes[1] = 0;
        net->last_persist_deps = false;
        if (pers && net->persist_deps) {
            const Arena flat = plan_arena(net, nb, mc.mode, false);
            net->last_arena_bytes[1] = (size_t)flat.peak;
            const size_t cap = net->ws_user ? net->ws_user_bytes : std::max<size_t>(ar.peak, (size_t)256 << 20);
            bool fits = (size_t)flat.peak <= cap;
            if (fits && !net->ws_user && net->ws_own_bytes < (size_t)flat.peak) {
                void* p = nullptr;
                if (cudaMalloc(&p, (size_t)flat.peak) == cudaSuccess) {
                    if (net->ws_own) CUDA_TRY(cudaFree(net->ws_own));
                    net->ws_own = p;
                    net->ws_own_bytes = (size_t)flat.peak;
                    mc.wss[i] = (char*)p;
                } else {
                    (void)cudaGetLastError();
                    fits = false;
                }
            }
            if (fits) {
                ar = flat;
                net->last_persist_deps = true;
            }
        }
        net->inv_key.clear();
        mc.arenas[i] = ar;
        if ((st = ensure_groups(net, mc.arenas[i], mc.wss[i], mc.mode, nb, s)) != TNC_OK) return st;
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
    // persistent executor: per round one work list with every network's
    // tasks, levels interleaved; slice ids per network come from the round's
    // row of the device table d_rs0. A network it cannot run keeps the whole
    // call on the merged level launches.
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
    if (!pers) {
        mc.wls.clear();
        for (tnc_net* net : mc.nets) net->last_persist_deps = false;
    }
    return TNC_OK;
}


}  // namespace tnc_host

extern "C" {

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
            << net->tc_row_bytes << ":" << (uintptr_t)net->d_prof << ":" << net->persist_deps;
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

}  // extern "C"
