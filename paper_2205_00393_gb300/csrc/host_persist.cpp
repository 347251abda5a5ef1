// Host side of the persistent executor: work lists of one slice batch (or
// one round of many networks), their validation, upload and launch.
#include "host.hpp"

namespace tnc_host {

// ------------------------------------------------------ persistent executor
//
// A work list is the whole computation of one launch: every contraction of a
// slice batch (and, in the first batch of a call, the slice-invariant ones)
// broken into tasks, in level order so that every task only waits on tasks
// before it (see kernels.h). A stage of a contraction (operand splits, tiles,
// K-split sums) counts its tasks down on counters; a task waits on the
// counters of the stage before it and of the contractions producing its
// inputs. On an arena that reuses memory across levels, each stage has one
// counter and a level chain makes every task wait for the whole level before
// it (its inputs included). On an arena without reuse, each stage has one
// counter per batch entry and a task of entry z waits only on entry z of what
// it reads, so the levels of different entries overlap.

constexpr int kSplitBlocksPerTask = 16;

// Counters of a stage of per_z tasks per batch entry over nz entries: one per
// entry without the level chain, else one for the stage. of(c, z) names entry
// z's (a single counter serves every entry).
static std::vector<int> wl_stage(WorkList& W, int64_t per_z, int nz) {
    std::vector<int> c;
    if (W.chain) c.push_back(W.new_counter((int)(per_z * nz)));
    else
        for (int z = 0; z < nz; ++z) c.push_back(W.new_counter((int)per_z));
    return c;
}
static int of(const std::vector<int>& c, int z) { return c.size() == 1 ? c[0] : c[z]; }

// The counter a task of entry z waits on before reading tensor v: the last
// stage of v's contraction when this launch produces v and no level chain
// orders it; -1 otherwise (a leaf, a cached invariant, or the chain waits).
static int wl_input(const WorkList& W, const std::map<int, std::vector<int>>& ctr, int v, int z) {
    if (W.chain) return -1;
    auto it = ctr.find(v);
    return it == ctr.end() ? -1 : of(it->second, z);
}

// Tasks of one non-root contraction np for batch b into W; ctr maps a tensor
// produced in this launch to the counters of its last stage. False if the
// contraction needs row or K panels (not run by the persistent executor).
bool wl_node(tnc_net* net, const Arena& ar, char* ws, const NodePlan& np, int b, int mode, int netidx, WorkList& W,
             std::map<int, std::vector<int>>& ctr) {
    const Plan& P = net->plan;
    tnc::GemmParams g = gemm_params(net, ar, ws, np, b);
    g.C = reinterpret_cast<float2*>(ws + ar.off[np.v]);
    g.c_batch_stride = np.per_slice ? tensor_bytes(P, np.v) / 8 : 0;
    W.cmacs += std::ldexp(1.0, np.mb + np.nb + np.kb) * b;
    const int choice = shape_choice(net, mode, np.mb, np.nb, np.kb, np.is_root);
    if (!choice) {
        const int gi = (int)W.gemm.size();
        W.gemm.push_back(g);
        const int64_t tiles = tnc::gemm_f32_tiles(np.mb, np.nb);
        const std::vector<int> c = wl_stage(W, tiles, b);
        for (int z = 0; z < b; ++z)
            for (int64_t t = 0; t < tiles; ++t)
                W.task(tnc::PT_GEMM, gi, t, z, netidx, 0, wl_input(W, ctr, np.A, z), wl_input(W, ctr, np.B, z), -1,
                       of(c, z));
        ctr[np.v] = c;
        return true;
    }
    const TcCut cut = tc_cut(net, mode, g.mb, g.nb, g.kb, cut_batch(ar, np, b));
    if (cut.pA || cut.pB || cut.pK) return false;
    W.tc_cmacs += std::ldexp(1.0, np.mb + np.nb + np.kb) * b;
    const size_t i = np.v - net->n_leaves;
    char* pa = ws + ar.planes_a[i];
    char* pb = ws + ar.planes_b[i];
    // an operand with neither batch stride nor sliced indices is the same for
    // every entry (a leaf or a slice-invariant tensor): split once
    const bool a_shared = b > 1 && g.A.batch_stride == 0 && g.A.n_sl == 0;
    const bool b_shared = b > 1 && g.B.batch_stride == 0 && g.B.n_sl == 0;
    int8_t* sexp_a = nullptr;
    int8_t* sexp_b = nullptr;
    if (mode == TNC_SPLIT_FP16X2) {
        sexp_a = reinterpret_cast<int8_t*>(pa + plane_data_bytes(mode, g.mb, g.kb, b));
        sexp_b = reinterpret_cast<int8_t*>(pb + plane_data_bytes(mode, g.nb, g.kb, b));
    }
    auto split = [&](const tnc::Operand& src, int src_v, int rb, const int64_t* rs, const int64_t* ks, void* dst,
                     int8_t* sexp, int nz) {
        tnc::SplitParams sp{};
        sp.src = src;
        sp.rb = rb;
        sp.kb = g.kb;
        for (int j = 0; j < rb; ++j) sp.rs[j] = rs[j];
        for (int j = 0; j < g.kb; ++j) sp.ks[j] = ks[j];
        sp.dst = dst;
        sp.sexp = sexp;
        const int64_t blocks = tnc::tc_split_prepare(sp);
        if (blocks <= 0) return std::vector<int>();
        const int si = (int)W.split.size();
        W.split.push_back(sp);
        const int64_t per = (blocks + kSplitBlocksPerTask - 1) / kSplitBlocksPerTask;
        const std::vector<int> c = wl_stage(W, per, nz);
        for (int z = 0; z < nz; ++z)
            for (int64_t q = 0; q < blocks; q += kSplitBlocksPerTask)
                W.task(tnc::PT_SPLIT, si, q, z, netidx, (int)std::min<int64_t>(kSplitBlocksPerTask, blocks - q),
                       wl_input(W, ctr, src_v, z), -1, -1, of(c, z));
        return c;
    };
    const std::vector<int> ca = split(g.A, np.A, g.mb, g.am, g.ak, pa, sexp_a, a_shared ? 1 : b);
    const std::vector<int> cb = split(g.B, np.B, g.nb, g.bn, g.bk, pb, sexp_b, b_shared ? 1 : b);
    if (ca.empty() || cb.empty()) return false;
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
    const std::vector<int> ct = wl_stage(W, tiles, b);
    for (int z = 0; z < b; ++z)
        for (int64_t t = 0; t < tiles; ++t) W.task(tnc::PT_TC, ti, t, z, netidx, 0, of(ca, z), of(cb, z), -1, of(ct, z));
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
    const std::vector<int> ck = wl_stage(W, chunks, b);
    for (int z = 0; z < b; ++z)
        for (int64_t q = 0; q < chunks; ++q) W.task(tnc::PT_KRED, ki, q, z, netidx, 0, of(ct, z), -1, -1, of(ck, z));
    ctr[np.v] = ck;
    return true;
}

// Tasks of the final contraction of network netidx for batch b: FP64 chunk
// sums then their ordered sum into out (at most 64 outputs), or an FP32 root
// tensor then its FP64 slice sum. The sum waits for every entry.
bool wl_root(tnc_net* net, const Arena& ar, char* ws, const NodePlan& np, int b, int netidx, double* out, WorkList& W,
             std::map<int, std::vector<int>>& ctr) {
    const Plan& P = net->plan;
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
            for (int c = 0; c < np.chunks; ++c)
                W.task(tnc::PT_ROOT, ri, c, z, netidx, ai, wl_input(W, ctr, np.A, z), wl_input(W, ctr, np.B, z), -1,
                       cr);
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
        for (int64_t t = 0; t < tiles; ++t)
            W.task(tnc::PT_GEMM, gi, t, z, netidx, 0, wl_input(W, ctr, np.A, z), wl_input(W, ctr, np.B, z), -1, cg);
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

static void level_cost_uncached(tnc_net* net, int mode, int64_t b, bool with_inv, double* launches,
                                double* seconds);

// Launches and estimated seconds of one batch of b slices on the per-level
// executor (the slice-invariant levels included when with_inv), added to
// *launches and *seconds: one grouped launch per level for its FP32
// contractions, three per tensor-core contraction (two operand splits and the
// GEMM), two for the final contraction. A contraction's time is estimated as
// the larger of its flops at 300 TFLOP/s and its operand and result bytes,
// 8 (MK + KN + MN) per slice, at 6 TB/s. Cached by plan_key, since the
// automatic executor choice asks for it on every call.
void level_cost(tnc_net* net, int mode, int64_t b, bool with_inv, double* launches, double* seconds) {
    const std::string key = plan_key(net, mode, b) + (with_inv ? ":i" : ":p");
    auto it = net->cost_cache.find(key);
    if (it == net->cost_cache.end()) {
        if (net->cost_cache.size() >= 64) net->cost_cache.clear();
        double l = 0, sec = 0;
        level_cost_uncached(net, mode, b, with_inv, &l, &sec);
        it = net->cost_cache.emplace(key, std::make_pair(l, sec)).first;
    }
    *launches += it->second.first;
    *seconds += it->second.second;
}

static void level_cost_uncached(tnc_net* net, int mode, int64_t b, bool with_inv, double* launches,
                                double* seconds) {
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


// Tasks of one network for a batch b: the slice-invariant levels (if with_inv),
// the per-slice levels and the final contraction.
bool wl_network(tnc_net* net, const Arena& ar, char* ws, int b, int mode, bool with_inv, int netidx, double* out,
                WorkList& W) {
    std::map<int, std::vector<int>> ctr;
    const Plan& P = net->plan;
    W.chain = ar.reuse;
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
    D.tensor_tasks = !W.split.empty() || !W.tc.empty() || !W.kred.empty();
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
    // a list without tensor-core work runs on the FP32 variant: two 256-thread
    // CTAs per SM instead of one CTA holding the tensor-core pipeline
    return tnc::launch_persist(p, D.tensor_tasks ? mode : TNC_FP32, s);
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


}  // namespace tnc_host
