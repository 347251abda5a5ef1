#!/usr/bin/env python
"""Benchmark of the sliced tensor-network contraction on GB300.

Workload: the 30-qubit 5x6 grid random circuit (14 cycles of the
sqrt(X)/sqrt(Y)/sqrt(W) + fSim family, seed 2) with the last 6 qubits open
(64 amplitudes), greedy contraction tree, lifetime-based slicing to at most
2^27-element intermediates (Algorithms 1 and 2, seed 7). A step is one
tnc_contract call over a batch of consecutive slices: every pairwise
contraction of those slices plus the FP64 slice sum. Inputs (leaves) are
resident in HBM when the timed region starts; every step streams 1 GiB
intermediates, far larger than the 129 MB L2, so no flush is needed.

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
on the host cores instead (rank 0 only; other ranks exit without work).
"""

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sliced contraction complex TFLOPS & s/1024 slices, split-TC vs FP32 at rel err≤1e-4"
UNIT = "TFLOPS (complex, effective 8*M*N*K per node)"
WORKLOAD = dict(rows=5, cols=6, cycles=14, seed=2, n_open=6, target_log2=27, sa_seed=7)
MODES = {"fp32": 0, "tf32": 1, "bf16": 2, "bf16x2": 3, "fp16x2": 4}
# FP32 CUDA-core peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flop x 2.070 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# Tensor flops per complex multiply-accumulate of one node (four real
# products Ar Br, Ai Bi, Ar Bi, Ai Br, each summed over the part pairs): BF16
# 3 parts -> 6 pairs, TF32, BF16x2 and FP16x2 2 parts -> 3 pairs; 2 flops per
# real MAC.
TENSOR_FLOPS_PER_CMAC = {"bf16": 4 * 6 * 2, "tf32": 4 * 3 * 2, "bf16x2": 4 * 3 * 2, "fp16x2": 4 * 3 * 2}
# dense TF32 / BF16 nominal rate ratio (1.1 vs 2.25 PFLOP/s per GPU)
TF32_OVER_BF16 = 1.1 / 2.25
KIND_NAMES = {0: "k_gemm_f32", 1: "k_root_partials", 2: "k_gemm_f32+slice_sum", 3: "k_cgemm_tc",
              4: "k_split_operand", 7: "k_ksplit_reduce", 8: "k_stem_fused", 9: "k_persist", -1: "k_slice_sum_f32", -2: "k_leaf_env_accum"}


def workload_name():
    w = WORKLOAD
    return ("rqc-%dx%d-%dcyc-seed%d-open%d-t%d" %
            (w["rows"], w["cols"], w["cycles"], w["seed"], w["n_open"], w["target_log2"]))


def build_network():
    from tnc_inputs import circuit_to_network, grid_rqc
    w = WORKLOAD
    c = grid_rqc(w["rows"], w["cols"], w["cycles"], w["seed"], n_open=w["n_open"])
    return c, circuit_to_network(c).as_complex64()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def kernel_traffic(kind_name, mode, cmacs_per_launch):
    """DRAM bytes per launch from the committed ncu capture, scaled by the
    launch's complex multiply-accumulates; valid only for the captured mode and
    while the kernel's source files are unchanged (hash of their concatenation
    recorded beside the figure)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kind_name)
    except (OSError, ValueError):
        return None
    if rec and "mode" not in rec:  # one record per mode
        rec = rec.get(mode)
    if not rec or rec.get("mode") != mode:
        return None
    srcs = rec["source"] if isinstance(rec["source"], list) else [rec["source"]]
    try:
        blob = b"".join(open(os.path.join(ROOT, f), "rb").read() for f in srcs)
    except OSError:
        return None
    h = hashlib.sha256(blob).hexdigest()[:16]
    return rec["bytes_per_cmac"] * cmacs_per_launch if h == rec["source_sha"] else None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def node_flops(stats, batch):
    """Effective complex flops (8*M*N*K per node) of one tnc_contract call over `batch` slices."""
    tot = 0
    for mb, nb, kb, per_slice, kind in stats["nodes"]:
        tot += 8 * (1 << (mb + nb + kb)) * (batch if per_slice else 1)
    return tot


def run_oracle_sample(ref_net, path, S):
    """Time the FP64 oracle on one full slice (slice 0) of the workload."""
    from oracle import tn
    log = []
    t0 = time.perf_counter()
    ref = tn.contract_slice(ref_net, path, S, 0, log=log)
    dt = time.perf_counter() - t0
    return sum(log), dt, ref


def kernel_breakdown(recs):
    by_kind = {}
    for r in recs:
        d = by_kind.setdefault(r["kind"], {"ms": 0.0, "cmacs": 0.0, "launches": 0})
        d["ms"] += r["ms"]
        d["launches"] += 1
        if r["kind"] in (0, 1, 2, 3, 9):
            d["cmacs"] += r["cmacs"]
    return by_kind


def probe_peaks(iters_ffma=300, iters_mma=1 << 22):
    """Peak rates measured by the library's own probe kernels (tnc_peak_probe),
    each timed alone with CUDA events after one warm-up launch (about 0.3 s
    per probe): FP32 FMA on the CUDA cores and tcgen05 MMA in kind::tf32,
    kind::f16 with BF16 and with FP16 operands."""
    import torch
    from paper_2205_00393_gb300 import peak_probe
    stream = torch.cuda.current_stream()
    out = {}
    for name, kind, iters in (("ffma_tflops", 0, iters_ffma), ("tf32_tflops", 1, iters_mma),
                              ("bf16_tflops", 2, iters_mma), ("fp16_tflops", 3, iters_mma)):
        peak_probe(kind, max(1, iters // 16), stream)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        flops = peak_probe(kind, iters, stream)
        ev1.record(stream)
        ev1.synchronize()
        out[name] = flops / (ev0.elapsed_time(ev1) / 1e3) / 1e12
    return out


def roofline_of(by_kind, mode, peaks, peak_src, sustained, probed=None, persist_tc_cmacs=None):
    """Roofline entry of the kernel with the most time. Tensor-core kernels in
    BF16/FP16 take the measured cuBLAS BF16 peak (the FP16 dense rate equals
    BF16's); TF32 takes the library's own kind::tf32 probe when given (else
    the BF16 peak times the nominal 1.1/2.25 ratio); FP32 CUDA-core kernels
    take the FFMA probe (else the unit-count derivation). The persistent
    kernel (k_persist) in a split mode counts only its tensor-core
    contractions as work (persist_tc_cmacs, from the library's stats) against
    its whole time, which also holds the splits, the FP32 contractions and the
    reductions it runs."""
    dom = max(by_kind, key=lambda k: by_kind[k]["ms"])
    d = by_kind[dom]
    share = d["ms"] / sum(v["ms"] for v in by_kind.values())
    sec = d["ms"] / 1e3
    tc_cmacs = None
    if dom == 3:
        tc_cmacs = d["cmacs"]
    elif dom == 9 and mode != "fp32" and persist_tc_cmacs:
        tc_cmacs = persist_tc_cmacs
    if tc_cmacs is not None:
        achieved = tc_cmacs * TENSOR_FLOPS_PER_CMAC[mode] / sec / 1e12
        if mode == "tf32" and probed:
            peak = probed["tf32_tflops"]
            src = "tcgen05 kind::tf32 probe of this run (tnc_peak_probe, 128x256x8 MMAs, one CTA per SM)"
        else:
            bf16 = peaks["bf16_tflops_sustained" if sustained else "bf16_tflops"]
            peak = bf16 * (TF32_OVER_BF16 if mode == "tf32" else 1.0)
            src = "%s bf16 %s (MEASURED_PEAKS.json)%s" % (
                "sustained" if sustained else "burst", peak_src,
                " x nominal tf32/bf16 ratio 1.1/2.25" if mode == "tf32" else "")
        r = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
             "frac": achieved / peak, "peak_source": src,
             "algorithmic_flops": "%d*M*N*K tensor flops per node (4 real products, %s part pairs)" % (
                 TENSOR_FLOPS_PER_CMAC[mode], mode)}
        if dom == 9:
            r["algorithmic_flops"] += ("; tensor-core contractions of the persistent kernel only, over its "
                                       "whole time")
    else:
        achieved = d["cmacs"] * 8 / sec / 1e12
        peak = probed["ffma_tflops"] if probed else FP32_PEAK_TFLOPS
        r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
             "frac": achieved / peak,
             "peak_source": ("FP32 FMA probe of this run (tnc_peak_probe, 8 chains per thread, 2048 threads "
                             "per SM)") if probed else "derived: 152 SM x 128 FP32 lanes x 2 flop x 2070 MHz",
             "algorithmic_flops": "8*M*N*K FP32 flops per node (4 real FMAs per complex MAC)"}
    r.update({"traffic": kernel_traffic(KIND_NAMES[dom], mode, d["cmacs"] / max(d["launches"], 1)),
              "kernel": KIND_NAMES[dom],
              "launches": d["launches"], "share_of_timed_kernel_time": share})
    return r


def top_nodes(recs, stats, n=6):
    agg = {}
    for r in recs:
        key = (r["node"], r["kind"])
        agg[key] = agg.get(key, 0.0) + r["ms"]
    nodes = stats["nodes"]
    out = []
    for (node, kind), ms in sorted(agg.items(), key=lambda x: -x[1])[:n]:
        i = node - stats["n_leaves"]
        mnk = nodes[i][:3] if 0 <= i < len(nodes) and node >= 0 else "grouped level launches"
        out.append({"node": node, "kernel": KIND_NAMES.get(kind, str(kind)), "log2_mnk": mnk, "ms": ms})
    return out


def cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        n = max((i.get("num_threads", 1) for i in info), default=os.cpu_count())
        return int(n)
    except Exception:
        return os.cpu_count()


def oracle_c1_seconds(threads=None):
    """Seconds the FP64 oracle takes for every slice (16) of the 12-qubit 3x4
    circuit (8 cycles, seed 1, t = 8), in a fresh interpreter so that the BLAS
    and OpenMP thread counts can be set before NumPy loads (threads=None: the
    host's default, all cores). Part of the CPU-baseline leg."""
    code = (
        "import json, time\n"
        "from oracle import planner, tn\n"
        "from tnc_inputs import circuit_to_network, grid_rqc\n"
        "net = circuit_to_network(grid_rqc(3, 4, 8, 1)).as_complex64()\n"
        "path = planner.greedy_path(net.indices, net.dims)\n"
        "S = planner.find_slices(planner.Tree(net.indices, net.dims, net.open_ids, path), 8, 7)\n"
        "t0 = time.perf_counter()\n"
        "for s in range(1 << len(S)):\n"
        "    tn.contract_slice(net, path, S, s)\n"
        "print(json.dumps({'seconds': time.perf_counter() - t0, 'slices': 1 << len(S)}))\n")
    env = dict(os.environ)
    if threads is not None:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[k] = str(threads)
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True,
                           timeout=300)
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # a missing figure, not a failed bench
        return {"error": str(e)[:200]}


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    from oracle import planner
    c, ref_net = build_network()
    path = planner.greedy_path(ref_net.indices, ref_net.dims)
    tree = planner.Tree(ref_net.indices, ref_net.dims, ref_net.open_ids, path)
    S = planner.find_slices(tree, WORKLOAD["target_log2"], WORKLOAD["sa_seed"])
    from oracle import tn
    times, macs = [], 0
    for i in range(args.warmup + args.steps):
        log = []
        t0 = time.perf_counter()
        tn.contract_slice(ref_net, path, S, i % (1 << len(S)), log=log)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            macs += sum(log)
    T = sum(times)
    tflops = 8 * macs / T / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": tflops, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "s_per_1024_slices": T / args.steps * 1024,
        "config": {"workload": workload_name(), "n_slices": 1 << len(S), "sliced": len(S),
                   "eq3_overhead": round(float(tree.overhead(S)), 5)},
        "mode": "oracle-fp64", "slices_per_step": 1, "parallelism": "host CPU",
        "cpu_baseline": {"value": tflops, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                         "sample": "one full slice (all pairwise contractions) per step, NumPy complex128"},
        "e2e": {"value": tflops, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def apply_options(net, args):
    if args.tc_row_bytes:
        net.set_option("tc_row_bytes", args.tc_row_bytes)
    if args.tc_group_m:
        net.set_option("tc_group_m", args.tc_group_m)
    if args.persistent is not None:
        net.set_option("persistent", args.persistent)


PERSIST_TASK_NAMES = ["fp32_tile", "split_blocks", "tc_tile", "ksplit_reduce", "root_chunk", "root_acc",
                      "root_sum", "stall"]


def persist_profile_of(prof):
    """Per task type of the persistent kernel: CTA-milliseconds in tasks (sum
    over CTAs), task count, CTA-milliseconds in dependency waits, and share of
    the task time."""
    tot = sum(r[0] for r in prof) or 1
    return {PERSIST_TASK_NAMES[t]: {"cta_ms": r[0] / 1e6, "tasks": r[1], "wait_cta_ms": r[2] / 1e6,
                                    "share": r[0] / tot}
            for t, r in enumerate(prof) if r[1]}


def executor_of(by_kind):
    return "persistent (k_persist, one launch per slice batch)" if 9 in by_kind else "one launch per tree level"


def single_node(args):
    """One isolated contraction C[m,n] = sum_k A[m,k] B[k,n] (plus a small root
    that contracts n away), random complex64 data; prints the node's kernel
    times. Used for isolated-kernel rooflines and ncu captures."""
    import torch
    from tnc_inputs.network import TensorNetwork
    from paper_2205_00393_gb300 import Network
    mb, nb, kb = (int(x) for x in args.single_node.split(","))
    rng = np.random.default_rng(0)

    def rnd(n):
        return ((rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)) / np.sqrt(2)).astype(np.complex64)
    # indices: m (dim 2^mb), k (2^kb), n (2^nb), o (2)
    dims = np.array([1 << mb, 1 << kb, 1 << nb, 2], dtype=np.int64)
    tn_ = TensorNetwork([rnd(mb + kb), rnd(kb + nb), rnd(nb + 1)], [(0, 1), (1, 2), (2, 3)], dims,
                        (0, 3), [-1, -1, -1])
    net = Network.from_tn(tn_)
    net.set_path([(0, 1), (2, 3)])
    apply_options(net, args)
    mode = MODES[args.mode]
    torch.cuda.set_device(0)
    for _ in range(args.warmup):
        net.contract(0, 1, mode)
    torch.cuda.synchronize()
    net.set_timing(True)
    for _ in range(args.steps):
        net.contract(0, 1, mode)
    net.check_device()
    recs, n_launches = net.last_timings()
    net.set_timing(False)
    by_kind = kernel_breakdown([r for r in recs if r["node"] in (3, -1) and r["kind"] in (3, 4, 0)])
    peaks, peak_src = load_peaks()
    line = {"single_node": [mb, nb, kb], "mode": args.mode, "tc_row_bytes": args.tc_row_bytes, "tc_group_m": args.tc_group_m,
            "steps": args.steps,
            "kernel_ms_per_call": {KIND_NAMES[k]: v["ms"] / args.steps for k, v in by_kind.items()},
            "roofline": roofline_of(by_kind, args.mode, peaks, peak_src, sustained=False),
            "gpu_launches": n_launches}
    print(json.dumps(line))
    return 0


def batched_circuits(n=256, seed0=1000, t_cap=24, cost_cap=None):
    """Plan the batched uneven workload (tnc_inputs.circuits.batched_workload):
    target t = min(W - k, t_cap) for a greedy tree of width W (k sliced modes
    where the greedy tree allows it, more where W - k > t_cap: no
    intermediate above 2^t_cap elements). With cost_cap, circuits whose
    slices cost more than cost_cap complex MACs are left out (returned
    separately); by default every circuit is kept."""
    from tnc_inputs import circuit_to_network
    from tnc_inputs.circuits import batched_workload
    from paper_2205_00393_gb300 import Network
    kept, dropped = [], []
    for i, (circ, k) in enumerate(batched_workload(n, seed0)):
        tn_ = circuit_to_network(circ).as_complex64()
        net = Network.from_tn(tn_)
        path = net.greedy_path()
        net.set_path(path)
        W = net.stats()["max_log2_size"]
        n_open = len(circ.open_qubits)
        t = max(min(W - k, t_cap), n_open + 4)
        S = net.find_slices(t, 7)
        net.set_slices(S)
        st = net.stats()
        per_slice = int(st["eq3"]) >> len(net.sliced)
        entry = dict(index=i, qubits=circ.n_qubits, cycles=circ.cycles, n_open=n_open, t=t,
                     slices=net.n_slices, per_slice_cmacs=per_slice, net=net, tn=tn_, circuit=circ,
                     path=[tuple(p) for p in path], S=list(S))
        (kept if cost_cap is None or per_slice <= cost_cap else dropped).append(entry)
    return kept, dropped


def many_bench(args):
    """Batched uneven workload: every kept circuit contributes its first
    --slices-per-step slices to each step. Times separate tnc_contract calls,
    and tnc_contract_many with the persistent executor (one launch per round,
    eager and graph replay) and with the merged per-level launches (graph
    replay). The headline value is the faster graph replay."""
    import torch
    from paper_2205_00393_gb300 import contract_many
    torch.cuda.set_device(0)
    kept, dropped = batched_circuits()
    mode = MODES[args.mode]
    nets = [e["net"] for e in kept]
    ranges = [(0, min(e["slices"], args.slices_per_step)) for e in kept]
    cmacs = sum(e["per_slice_cmacs"] * (hi - lo) for e, (lo, hi) in zip(kept, ranges))
    n_sl = sum(hi - lo for lo, hi in ranges)
    stream = torch.cuda.Stream()
    res = {}
    def executor(p):
        for n in nets:
            n.set_option("persistent", p)

    with torch.cuda.stream(stream):
        outs = [torch.empty(n.n_out, dtype=torch.complex128, device="cuda") for n in nets]

        def timed(fn):
            for _ in range(args.warmup):
                fn()
            stream.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(args.steps):
                fn()
            ev1.record(stream)
            stream.synchronize()
            return ev0.elapsed_time(ev1) / 1e3 / args.steps

        def separate():
            for net, (lo, hi), o in zip(nets, ranges, outs):
                net.contract(lo, hi, mode, out=o, stream=stream)
        executor(0)
        res["separate_per_level"] = timed(separate)
        # kernel time by kernel of one round of per-level separate calls
        for n in nets:
            n.set_timing(True)
        separate()
        stream.synchronize()
        per_level_kernels = {}
        for n in nets:
            for k, v in kernel_breakdown(n.last_timings()[0]).items():
                per_level_kernels[KIND_NAMES.get(k, str(k))] = per_level_kernels.get(KIND_NAMES.get(k, str(k)), 0.0) + v["ms"]
            n.set_timing(False)
        res["many_graph_per_level"] = timed(lambda: contract_many(nets, ranges, mode, outs=outs, use_graph=True,
                                                                  stream=stream))
        executor(1)
        res["separate_persistent"] = timed(separate)
        res["many_no_graph_persistent"] = timed(lambda: contract_many(nets, ranges, mode, outs=outs,
                                                                      use_graph=False, stream=stream))
        res["many_graph_persistent"] = timed(lambda: contract_many(nets, ranges, mode, outs=outs, use_graph=True,
                                                                   stream=stream))
        # kernels per step of each graph replay, counted by the library on the first network
        launches = {}
        for p, key in ((1, "persistent"), (0, "per_level")):
            executor(p)
            nets[0].set_timing(True)
            contract_many(nets, ranges, mode, outs=outs, use_graph=True, stream=stream)
            stream.synchronize()
            launches[key] = nets[0].last_timings()[1]
            nets[0].set_timing(False)
        executor(1)
        # where the persistent kernel's CTA time goes (one profiled call)
        nets[0].set_option("persist_profile", 1)
        contract_many(nets, ranges, mode, outs=outs, use_graph=True, stream=stream)
        stream.synchronize()
        nets[0].set_timing(True)
        contract_many(nets, ranges, mode, outs=outs, use_graph=True, stream=stream)
        stream.synchronize()
        prof = persist_profile_of(nets[0].stats()["persist_profile"])
        nets[0].set_timing(False)
        nets[0].set_option("persist_profile", 0)
        # the launch-bound end of the mix: circuits whose slices cost at most
        # 2^26 complex MACs, both executors, graph replay
        small = [i for i, e in enumerate(kept) if e["per_slice_cmacs"] <= 2 ** 26]
        s_nets = [nets[i] for i in small]
        s_ranges = [ranges[i] for i in small]
        s_outs = [outs[i] for i in small]
        subset = {"circuits": len(small),
                  "cmacs_per_step": float(sum(kept[i]["per_slice_cmacs"] * (ranges[i][1] - ranges[i][0])
                                              for i in small))}
        for p, key in ((0, "per_level"), (1, "persistent")):
            executor(p)
            subset["ms_" + key] = 1e3 * timed(lambda: contract_many(s_nets, s_ranges, mode, outs=s_outs,
                                                                    use_graph=True, stream=stream))
        subset["speedup_persistent_vs_per_level"] = subset["ms_per_level"] / subset["ms_persistent"]
    best = min(("many_graph_persistent", "many_graph_per_level"), key=lambda k: res[k])
    T = res[best]
    line = {"metric": "batched uneven circuits: effective complex TFLOPS & s/1024 slices (graph replay)",
            "value": 8 * cmacs / T / 1e12, "unit": UNIT, "s_per_1024_slices": T / n_sl * 1024,
            "executor": best, "ms_per_step": {k: 1e3 * v for k, v in res.items()},
            "kernels_per_step": launches, "persistent_task_profile": prof,
            "per_level_separate_kernel_ms": per_level_kernels, "launch_bound_subset": subset,
            "speedup_vs_separate_calls": min(res["separate_per_level"], res["separate_persistent"]) / T,
            "speedup_persistent_vs_per_level": res["many_graph_per_level"] / res["many_graph_persistent"],
            "mode": args.mode, "steps": args.steps,
            "warmup": args.warmup,
            "config": {"workload": "256 seeded grid circuits (seeds 1000..1255), qubits 20-36, cycles 10-16, "
                                   "open 0-6, slicing depth k 4-12, target t = min(W - k, 24) for greedy width W",
                       "circuits_run": len(kept), "circuits_left_out": len(dropped),
                       "n_slices_log2_range": [min(int(np.log2(e["slices"])) for e in kept),
                                                       max(int(np.log2(e["slices"])) for e in kept)],
                       "per_slice_cmacs_log2_range": [float(np.log2(min(e["per_slice_cmacs"] for e in kept))),
                                                float(np.log2(max(e["per_slice_cmacs"] for e in kept)))],
                       "slices_per_step": n_sl, "slices_per_circuit_max": args.slices_per_step}}
    if not args.no_cpu_baseline:
        # the FP64 oracle on the cheapest circuits' slices of a step (about 15 s
        # of CPU work), compared with this step's results for those circuits
        from oracle import tn as oracle_tn
        got = {e["index"]: o.cpu().numpy() for e, o in zip(kept, outs)}
        t_cpu, macs, worst, done = 0.0, 0, 0.0, 0
        for e, (lo, hi) in sorted(zip(kept, ranges), key=lambda er: er[0]["per_slice_cmacs"]):
            if t_cpu > 15.0:
                break
            t0 = time.perf_counter()
            want = oracle_tn.contract(e["tn"], e["path"], e["S"], range(lo, hi))
            t_cpu += time.perf_counter() - t0
            macs += e["per_slice_cmacs"] * (hi - lo)
            done += 1
            g = got[e["index"]]
            rms = float(np.sqrt(np.mean(np.abs(want) ** 2)))
            floor = max(0.1 * rms, 1e-300)  # a circuit whose amplitudes all vanish compares absolutely
            worst = max(worst, float(np.max(np.abs(g - want) / np.maximum(np.abs(want), floor))))
        line["cpu_baseline"] = {"value": 8 * macs / t_cpu / 1e12, "unit": UNIT, "cores": cpu_threads(),
                                "kind": "oracle",
                                "sample": "the %d cheapest circuits' slices of one step (NumPy complex128 "
                                          "tensordot per node), %.1f s" % (done, t_cpu)}
        line["rel_err_vs_oracle_floor_0.1rms"] = {"circuits": done, "max": worst}
    print(json.dumps(line))
    return 0


def bitstrings_bench(args):
    """Correlated amplitudes (Sec. 1 and 6.2): B closed bitstrings of the
    30-qubit circuit (64 open amplitudes each). Path "stem" (default): the
    time-ordered stem path, whose projection vectors come last, unsliced (the
    2^30-element state before the projections is shared by every bitstring);
    path "greedy": the greedy path sliced to 2^27 elements, every bitstring
    over the first --slices-per-step slices. Times one tnc_contract_variants
    call over the B bitstrings (the shared part computed once) against
    ordinary contractions of single bitstrings (each recomputing it; timed on
    min(B, 4) bitstrings and scaled to B)."""
    import torch
    from tnc_inputs import bitstring_variants, random_bitstrings, stem_path
    from paper_2205_00393_gb300 import Network
    torch.cuda.set_device(0)
    B = args.bitstrings
    c, ref_net = build_network()
    net = Network.from_tn(ref_net)
    if args.bitstring_path == "stem":
        net.set_path(stem_path(ref_net, c))
        if args.stem_coalesce_bits is not None:
            net.set_option("stem_coalesce_bits", args.stem_coalesce_bits)
        if args.stem_cap_log2 is not None:
            net.set_option("stem_cap_log2", args.stem_cap_log2)
        S = []
        ns = 1
    else:
        net.set_path(net.greedy_path())
        S = net.find_slices(WORKLOAD["target_log2"], WORKLOAD["sa_seed"])
        ns = args.slices_per_step
    net.set_slices(S)
    mode = MODES[args.mode]
    bits = random_bitstrings(c, B, 11)
    leaves, data = bitstring_variants(c, bits)
    net.set_leaf_variants(leaves, data)
    sbits = len(S)
    stream = torch.cuda.current_stream()
    out = torch.empty((B, net.n_out), dtype=torch.complex128, device="cuda")
    if mode != 0 and not args.no_autotune:
        net.autotune(mode, 0)

    def shared():
        net.contract_variants(0, B, 0, ns, mode, out=out)

    n_un = min(B, 4)

    def unshared():
        for v in range(n_un):
            net.contract((v << sbits), (v << sbits) + ns, mode, out=out[v])

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / 1e3 / args.steps

    net.set_option("cache_invariants", 0)
    t_shared = timed(shared)
    t_unshared = timed(unshared) * B / n_un
    # work of one call: shared part once plus every bitstring's own part
    net.set_timing(True)
    shared()
    torch.cuda.synchronize()
    c_shared = sum(r["cmacs"] for r in net.last_timings()[0])
    net.set_timing(True)
    net.contract(0, ns, mode, out=out[0])
    torch.cuda.synchronize()
    c_one = sum(r["cmacs"] for r in net.last_timings()[0])
    net.set_timing(False)
    line = {"metric": "correlated amplitudes of B bitstrings: effective complex TFLOPS (every bitstring's full "
                      "contraction counted)",
            "value": 8 * B * c_one / t_shared / 1e12, "unit": UNIT, "bitstrings": B,
            "bitstring_slices_per_s": B * ns / t_shared,
            "ms_per_call_shared": 1e3 * t_shared, "ms_per_call_unshared": 1e3 * t_unshared,
            "speedup_shared_vs_unshared": t_unshared / t_shared,
            "cmacs_per_call_shared": c_shared, "cmacs_per_bitstring_unshared": c_one,
            "shared_fraction_of_one_bitstring": 1.0 - (c_shared - c_one) / ((B - 1) * c_one) if B > 1 else None,
            "unshared_timed_on_bitstrings": n_un,
            "mode": args.mode, "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": "rqc-5x6-14cyc-seed2-open6, %s path%s" % (
                           args.bitstring_path, "" if S else ", unsliced"),
                       "slices_per_bitstring": ns, "n_slices": net.n_slices, "sliced": len(S),
                       "bitstring_seed": 11, "open_amplitudes_per_bitstring": net.n_out}}
    print(json.dumps(line))
    return 0


def persist_demo(args):
    """The two executors on a mid-size network: the 24-qubit 4x6 grid circuit
    (12 cycles, seed 3, last 4 qubits open), greedy path sliced to 2^20
    elements, 8 slices per call in split BF16 (tensor-core and FP32
    contractions mixed). Times one persistent launch per call, with per-entry
    dependencies and with the level chain, against one launch per tree
    level."""
    import torch
    from tnc_inputs import circuit_to_network, grid_rqc
    from paper_2205_00393_gb300 import Network
    torch.cuda.set_device(0)
    c = grid_rqc(4, 6, 12, 3, n_open=4)
    net = Network.from_tn(circuit_to_network(c).as_complex64())
    net.set_path(net.greedy_path())
    net.set_slices(net.find_slices(20, 7))
    stats = net.stats()
    mode = MODES[args.mode]
    B = args.slices_per_step
    stream = torch.cuda.current_stream()
    out = torch.empty(net.n_out, dtype=torch.complex128, device="cuda")
    res = {}
    for name, p, deps in (("persistent", 1, 1), ("persistent_level_chain", 1, 0), ("per_level", 0, 1)):
        net.set_option("persistent", p)
        net.set_option("persist_deps", deps)
        for i in range(args.warmup):
            net.contract((i * B) % net.n_slices, (i * B) % net.n_slices + B, mode, out=out)
        torch.cuda.synchronize()
        net.set_timing(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for i in range(args.steps):
            lo = (i * B) % net.n_slices
            net.contract(lo, lo + B, mode, out=out)
        ev1.record(stream)
        torch.cuda.synchronize()
        T = ev0.elapsed_time(ev1) / 1e3 / args.steps
        recs, nl = net.last_timings()
        net.set_timing(False)
        res[name] = {"ms_per_call": 1e3 * T, "value": node_flops(stats, B) / T / 1e12,
                     "kernels_per_call": nl / args.steps,
                     "kernel_ms_per_call": {KIND_NAMES.get(k, str(k)): v["ms"] / args.steps
                                            for k, v in kernel_breakdown(recs).items()}}
    line = {"metric": "persistent vs per-level executor: effective complex TFLOPS", "unit": UNIT,
            "value": res["persistent"]["value"], "mode": args.mode, "steps": args.steps, "warmup": args.warmup,
            "speedup_persistent_vs_per_level": res["per_level"]["ms_per_call"] / res["persistent"]["ms_per_call"],
            "speedup_deps_vs_level_chain": (res["persistent_level_chain"]["ms_per_call"] /
                                            res["persistent"]["ms_per_call"]),
            "executors": res,
            "config": {"workload": "rqc-4x6-12cyc-seed3-open4-t20", "slices_per_step": B, "n_slices": net.n_slices}}
    print(json.dumps(line))
    return 0


def executor_sweep(args):
    """Both executors on grid circuits from 12 to 30 qubits (greedy paths
    sliced to 2^8 .. 2^27-element intermediates), FP32 and split FP16x2, 1, 4
    and 16 slices per call: ms per call of each (CUDA events over a run of
    calls after 3 warm-up calls) beside the library's estimate of the
    per-level work (the automatic choice's input: per-level launches and
    estimated seconds) and the executor the automatic choice runs. One JSON
    line per configuration."""
    import torch
    from tnc_inputs import circuit_to_network, grid_rqc
    from paper_2205_00393_gb300 import Network
    torch.cuda.set_device(0)
    specs = [(3, 4, 8, 1, 0, 8), (4, 4, 10, 2, 2, 12), (4, 5, 12, 3, 3, 16), (4, 6, 12, 3, 4, 20),
             (5, 5, 12, 4, 4, 20), (5, 6, 12, 5, 4, 22), (5, 6, 14, 2, 6, 24), (5, 6, 14, 2, 6, 27)]
    stream = torch.cuda.current_stream()
    for (r, c, cyc, seed, n_open, t) in specs:
        net = Network.from_tn(circuit_to_network(grid_rqc(r, c, cyc, seed, n_open=n_open)).as_complex64())
        net.set_path(net.greedy_path())
        net.set_slices(net.find_slices(t, 7))
        out = torch.empty(net.n_out, dtype=torch.complex128, device="cuda")
        for mode in (0, 4):
            for B in (1, 4, 16):
                if B > net.n_slices or (t >= 24 and B > 1) or (t >= 27 and mode == 0):
                    continue
                ms, deps = {}, None
                for name, p in (("persistent", 1), ("per_level", 0)):
                    net.set_option("persistent", p)
                    calls = 12 if t < 24 else 4
                    for _ in range(3):
                        net.contract(0, B, mode, out=out)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for i in range(calls):
                        lo = (i * B) % net.n_slices
                        net.contract(lo, lo + B, mode, out=out)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    net.check_device()
                    ms[name] = e0.elapsed_time(e1) / calls
                    if p == 1:
                        deps = net.stats()["last_persist_deps"]
                # what the automatic choice runs for this call
                net.set_option("persistent", 2)
                net.set_timing(True)
                net.contract(0, B, mode, out=out)
                torch.cuda.synchronize()
                auto = "persistent" if 9 in {r["kind"] for r in net.last_timings()[0]} else "per_level"
                net.set_timing(False)
                launches, est_s = net.stats()["level_cost"][str(mode)]
                print(json.dumps({"metric": "executor sweep: ms per call", "workload":
                                  "rqc-%dx%d-%dcyc-seed%d-open%d-t%d" % (r, c, cyc, seed, n_open, t),
                                  "mode": {v: k for k, v in MODES.items()}[mode], "slices_per_call": B,
                                  "per_level_launches": launches, "estimated_us_per_launch": 1e6 * est_s / max(launches, 1),
                                  "ms_persistent": ms["persistent"], "ms_per_level": ms["per_level"],
                                  "per_level_over_persistent": ms["per_level"] / ms["persistent"],
                                  "automatic_choice": auto, "automatic_choice_is_faster":
                                  ms[auto] <= min(ms.values()), "persist_deps": deps}), flush=True)
        del net
    return 0


def c53_bench(args):
    """53-qubit lattice (6x9 grid minus one site), 20 cycles (seed 3), one
    amplitude, sliced to 2^30-element intermediates: a fixed subset of slices
    [0, n) (1024 by default) in the split mode, timed with CUDA events, in
    batches of --slices-per-step; then the first two slices again in split
    precision and on the FP32 CUDA-core path, whose sums are compared (the
    oracle cannot run at this size)."""
    import torch
    from tnc_inputs import circuit_to_network, lattice_53q_rqc
    from paper_2205_00393_gb300 import Network, tune_table
    torch.cuda.set_device(0)
    c = lattice_53q_rqc(20, 3)
    net = Network.from_tn(circuit_to_network(c).as_complex64())
    net.set_path(net.greedy_path())
    net.set_slices(net.find_slices(30, 7))
    apply_options(net, args)
    mode = MODES[args.mode]
    B = args.slices_per_step
    n = args.c53_slices
    if not args.no_autotune:
        net.autotune(mode, 0)
    ws = torch.empty(net.workspace_bytes(B), dtype=torch.uint8, device="cuda")
    net.set_workspace(ws)
    stats = net.stats()
    out = torch.empty(net.n_out, dtype=torch.complex128, device="cuda")
    acc = torch.zeros(net.n_out, dtype=torch.complex128, device="cuda")
    net.contract(n, n + B, mode, out=out)  # warm-up on slices outside the timed subset
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        ev0.record(stream)
        for lo in range(0, n, B):
            net.contract(lo, min(lo + B, n), mode, out=out)
            acc += out
        ev1.record(stream)
        torch.cuda.synchronize()
    net.check_device()
    T = ev0.elapsed_time(ev1) / 1e3
    # per-launch breakdown on one more call (outside the timed subset)
    net.set_timing(True)
    net.contract(n, n + B, mode, out=out)
    torch.cuda.synchronize()
    recs, _ = net.last_timings()
    net.set_timing(False)
    by_kind = kernel_breakdown(recs)
    flops = node_flops(stats, n)
    split2 = net.contract(0, 2, mode, out=out).cpu().numpy()[0]
    t0 = time.perf_counter()
    fp32 = net.contract(0, 2, 0, out=out).cpu().numpy()[0]
    t_fp32 = time.perf_counter() - t0
    line = {"metric": "53-qubit lattice, 20 cycles: sliced contraction of a fixed slice subset",
            "mode": args.mode, "value": flops / T / 1e12, "unit": UNIT,
            "s_per_1024_slices": T / n * 1024, "slices": n, "seconds": T,
            "n_sliced": len(net.sliced), "eq3_overhead": stats["overhead"], "max_log2_size": stats["max_log2_size"],
            "workspace_gb": ws.numel() / 1e9, "partial_amplitude": [float(acc[0].real), float(acc[0].imag)],
            "rel_err_vs_fp32_path_2_slices": float(abs(split2 - fp32) / abs(fp32)),
            "fp32_path_s_per_slice": t_fp32 / 2, "clocks": clk.summary(),
            "kernel_time_ms_one_call": {KIND_NAMES.get(k, str(k)): v["ms"] for k, v in by_kind.items()},
            "top_nodes_one_call": top_nodes(recs, stats, 10),
            "tuned_shapes": [e for e in tune_table() if e[0] == mode]}
    print(json.dumps(line))
    return 0


def grad42_bench(args):
    """Gradient configuration: 42-qubit 6x7 grid, 12 cycles (seed 5), one
    amplitude, sliced to 2^30-element intermediates; d amp / d(theta, phi) of
    all fSim gates for the partial amplitude over slices [0, n) by the adjoint
    pass under an 80 GB budget (per-level checkpointing as needed), checked
    against central finite differences (h = 1e-3) on 16 parameters chosen by
    seed 6, and against the gate-perturbation witness (F(G + dG) - F(G - dG)) / 2,
    exact because the amplitude is linear in every gate matrix."""
    import torch
    from tnc_inputs import circuit_to_network, grid_rqc
    from paper_2205_00393_gb300.torch_fn import CircuitAmplitudes
    torch.cuda.set_device(0)
    c = grid_rqc(6, 7, 12, 5)
    tn_ = circuit_to_network(c)
    fsim = [li for li, g in enumerate(tn_.leaf_gate) if g >= 0 and c.gates[g].name == "fsim"]
    n_sl = args.slices_per_step
    mode = MODES[args.mode]  # FP32 by default: complex64 forward, FP32 adjoint
    amp = CircuitAmplitudes(tn_, fsim, target_log2=30, seed=7, lo=0, hi=n_sl, mode=mode,
                            budget_bytes=80 << 30)
    params = torch.tensor(np.array([g.params for g in c.gates if g.name == "fsim"], dtype=np.float64),
                          dtype=torch.float64, requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    a = amp(params)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    a.real.sum().backward()  # d Re(amp) / d params
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    amp.net.check_device()
    st = amp.net.stats()
    g = params.grad.numpy()
    rng = np.random.default_rng(6)
    flat = rng.choice(params.numel(), 16, replace=False)
    which = [(int(f) // 2, int(f) % 2) for f in flat]
    p0 = params.detach().numpy().copy()
    got = np.array([g[k, j] for (k, j) in which])

    def central_fd(h):
        fd = []
        for (k, j) in which:
            vals = []
            for sgn in (1, -1):
                p = p0.copy()
                p[k, j] += sgn * h
                with torch.no_grad():
                    vals.append(float(amp(torch.from_numpy(p)).real.sum()))
            fd.append((vals[0] - vals[1]) / (2 * h))
        amp.set_params(p0)  # the loop leaves the last parameter perturbed
        fd = np.array(fd)
        rms = float(np.sqrt(np.mean(fd ** 2)))
        return (float(np.max(np.abs(got - fd) / np.maximum(np.abs(fd), rms))),
                float(np.linalg.norm(got - fd) / np.linalg.norm(fd)))
    err, err_norm = central_fd(1e-3)
    # the witness's own noise: rounding of the forward divided by 2h falls as 1/h
    # until the truncation error (h^2 / 6 relative) takes over
    fd_by_h = {"%g" % h: dict(zip(("max_rel", "normwise"), central_fd(h))) for h in args.fd_extra_h}
    # second witness: the amplitude is linear in every gate matrix, so
    # (amp(G + dG) - amp(G - dG)) / 2 is the exact derivative along dG
    from tnc_inputs import gates as G
    lin = []
    for (k, j) in which:
        th, ph = p0[k]
        dG = G.dfsim_dtheta(th, ph) if j == 0 else G.dfsim_dphi(th, ph)
        vals = []
        for sgn in (1, -1):
            amp.net.set_tensor_data(fsim[k], (G.fsim(th, ph) + sgn * dG).reshape(2, 2, 2, 2))
            vals.append(float(amp.net.contract(0, n_sl, mode).real.sum()))
        amp.net.set_tensor_data(fsim[k], G.fsim(th, ph).reshape(2, 2, 2, 2))
        lin.append((vals[0] - vals[1]) / 2)
    lin = np.array(lin)
    rms_l = float(np.sqrt(np.mean(lin ** 2)))
    err_lin = float(np.max(np.abs(got - lin) / np.maximum(np.abs(lin), rms_l)))
    err_lin_norm = float(np.linalg.norm(got - lin) / np.linalg.norm(lin))
    line = {"metric": "adjoint gradient of a 42-qubit amplitude (partial over slices) vs central differences",
            "mode": args.mode, "params": int(params.numel()), "slices": n_sl,
            "n_sliced": len(amp.net.sliced), "forward_s": t1 - t0, "backward_s": t2 - t1,
            "max_rel_err_vs_fd_h1e-3": err, "normwise_rel_err_vs_fd_h1e-3": err_norm, "fd_params": 16,
            "max_rel_err_vs_gate_perturbation": err_lin, "normwise_rel_err_vs_gate_perturbation": err_lin_norm,
            "fd_other_h": fd_by_h,
            "backward_keep_every": st.get("backward_keep_every"),
            "backward_workspace_gb": st.get("backward_workspace", 0) / 1e9, "budget_gb": 80 * 1.073741824,
            "amplitude_partial": [float(a.detach().real.sum()), float(a.detach().imag.sum())]}
    print(json.dumps(line))
    return 0


def backward_bench(args):
    """Forward + adjoint pass over a batch of slices per step: environments of
    every fSim leaf for F = sum of the 64 amplitudes (FP32 environment
    contractions; forward in --mode)."""
    import torch
    from paper_2205_00393_gb300 import Network
    torch.cuda.set_device(0)
    c, ref_net = build_network()
    net = Network.from_tn(ref_net)
    net.set_path(net.greedy_path())
    S = net.find_slices(WORKLOAD["target_log2"], WORKLOAD["sa_seed"])
    net.set_slices(S)
    apply_options(net, args)
    mask = np.array([1 if g >= 0 and c.gates[g].name == "fsim" else 0 for g in ref_net.leaf_gate], dtype=np.uint8)
    seed = torch.ones(net.n_out, dtype=torch.complex128, device="cuda")
    B = args.slices_per_step
    mode = MODES[args.mode]
    for i in range(args.warmup):
        net.contract_backward(seed, (i * B) % net.n_slices, (i * B) % net.n_slices + B, mode, leaf_mask=mask)
    torch.cuda.synchronize()
    net.set_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for i in range(args.steps):
        lo = ((args.warmup + i) * B) % net.n_slices
        net.contract_backward(seed, lo, lo + B, mode, leaf_mask=mask)
    ev1.record()
    torch.cuda.synchronize()
    T = ev0.elapsed_time(ev1) / 1e3
    net.check_device()
    recs, n_launches = net.last_timings()
    net.set_timing(False)
    by_kind = kernel_breakdown(recs)
    cmacs = sum(v["cmacs"] for k, v in by_kind.items() if k in (0, 3))
    stats = net.stats()
    line = {"metric": "adjoint pass (forward + environments of all fSim leaves), effective complex TFLOPS",
            "value": 8 * cmacs / T / 1e12, "unit": UNIT, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * T / args.steps, "s_per_1024_slices": T / (args.steps * B) * 1024,
            "forward_mode": args.mode,
            "env_precision": "same arithmetic as the forward mode (split precision: FP32 accumulate)",
            "config": {"workload": workload_name(), "slices_per_step": B, "n_slices": net.n_slices,
                       "fsim_leaves": int(mask.sum())},
            "kernel_time_ms": {KIND_NAMES.get(k, str(k)): v["ms"] for k, v in by_kind.items()},
            "gpu_launches": n_launches, "backward_batch": stats.get("last_batch")}
    print(json.dumps(line))
    return 0


def stem_bench(args):
    """Fused stem groups (secondary slicing, Sec. 5.2) on a time-ordered stem
    path (every contraction a narrow step: a stem absorbing a gate): 28-qubit
    4x7 grid, 12 cycles (seed 4), last 4 qubits open (16 amplitudes), not
    sliced, so the stem reaches 2^28 complex elements (2 GiB, far above L2).
    The whole contraction is timed with fusion on (the default) and off."""
    import torch
    from tnc_inputs import circuit_to_network, grid_rqc, stem_path
    from paper_2205_00393_gb300 import Network
    torch.cuda.set_device(0)
    rows, cols = (int(x) for x in args.stem_grid.split("x"))
    c = grid_rqc(rows, cols, 12, 4, n_open=4)
    tn_ = circuit_to_network(c).as_complex64()
    net = Network.from_tn(tn_)
    net.set_path(stem_path(tn_, c))
    if args.stem_coalesce_bits is not None:
        net.set_option("stem_coalesce_bits", args.stem_coalesce_bits)
    if args.stem_cap_log2 is not None:
        net.set_option("stem_cap_log2", args.stem_cap_log2)
    cap = net.stats()["stem_cap_log2"]
    stats = net.stats()
    groups = stats["stem_groups"]
    flops = node_flops(stats, 1)
    stream = torch.cuda.current_stream()
    out = torch.empty(net.n_out, dtype=torch.complex128, device="cuda")
    res = {}
    # both on the per-level executor: the fused groups run there, and the
    # unfused baseline is the same contractions as separate per-level launches
    net.set_option("persistent", 0)
    for name, cap in (("fused", cap), ("unfused", 0)):
        if name == "unfused" and args.stem_no_unfused:
            continue
        net.set_option("stem_cap_log2", cap)
        ws = torch.empty(net.workspace_bytes(1), dtype=torch.uint8, device="cuda")
        net.set_workspace(ws)
        for _ in range(args.warmup):
            net.contract(0, 1, 0, out=out)
        torch.cuda.synchronize()
        net.set_timing(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            ev0.record(stream)
            for _ in range(args.steps):
                net.contract(0, 1, 0, out=out)
            ev1.record(stream)
            torch.cuda.synchronize()
        net.check_device()
        T = ev0.elapsed_time(ev1) / 1e3 / args.steps
        recs, n_launches = net.last_timings()
        net.set_timing(False)
        res[name] = {"s_per_call": T, "value": flops / T / 1e12, "launches_per_call": n_launches / args.steps,
                     "kernel_time_ms_per_call": {KIND_NAMES.get(k, str(k)): v["ms"] / args.steps
                                                 for k, v in kernel_breakdown(recs).items()},
                     "clocks": clk.summary(), "amplitudes": out.cpu().numpy()}
        del ws
    a = res["fused"].pop("amplitudes")
    b = res["unfused"].pop("amplitudes") if "unfused" in res else None
    # the fused kernel against HBM: per launch it reads its input stem and writes its output once
    st_ms = res["fused"]["kernel_time_ms_per_call"].get("k_stem_fused", 0.0)
    st_bytes = sum(8 * ((1 << g[5]) + (1 << g[6])) for g in groups)
    peaks, peak_src = load_peaks()
    gbs = st_bytes / (st_ms / 1e3) / 1e9 if st_ms else None
    line = {"metric": "fused stem groups (secondary slicing) on a stem path: effective complex TFLOPS",
            "value": res["fused"]["value"], "unit": UNIT, "steps": args.steps, "warmup": args.warmup,
            "speedup_vs_unfused": res["unfused"]["s_per_call"] / res["fused"]["s_per_call"] if b is not None else None,
            "fused_vs_unfused_max_rel_diff": float(np.max(np.abs(a - b)) / np.max(np.abs(b))) if b is not None else None,
            "groups": len(groups), "fused_steps": sum(g[1] for g in groups), "nodes": len(stats["nodes"]),
            "k_stem_fused": {"ms_per_call": st_ms, "algorithmic_bytes_per_call": st_bytes,
                             "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                          "frac": gbs / peaks["hbm_gbs"] if gbs else None,
                                          "peak_source": "hbm copy %s (MEASURED_PEAKS.json)" % peak_src}},
            "fused": res["fused"], "unfused": res.get("unfused"),
            "config": {"workload": "rqc-%s-12cyc-seed4-open4 time-ordered stem path, not sliced" % args.stem_grid,
                       "max_log2_size": stats["max_log2_size"], "mode": "fp32 (narrow steps run on CUDA cores)",
                       "stem_coalesce_bits": args.stem_coalesce_bits, "stem_cap_log2": cap}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=24)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tnc", choices=["tnc", "reference"])
    ap.add_argument("--mode", default=None, choices=sorted(MODES),
                    help="arithmetic of the contractions (default fp16x2; bf16 for the single-node, "
                         "backward and many-circuit modes; fp32 for --grad42)")
    ap.add_argument("--compare-modes", default="bf16,tf32",
                    help="comma-separated split modes also timed on the same slices in the default run "
                         "(reported under split_modes; empty to skip)")
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tc-row-bytes", type=int, default=None)
    ap.add_argument("--tc-group-m", type=int, default=None)
    ap.add_argument("--persistent", type=int, default=None, choices=[0, 1],
                    help="executor: 1 the persistent work-list kernel, 0 one launch per tree level "
                         "(default: the library's choice)")
    ap.add_argument("--c53", action="store_true",
                    help="53-qubit lattice, 20 cycles, t = 30: time a fixed subset of slices")
    ap.add_argument("--c53-slices", type=int, default=1024)
    ap.add_argument("--fd-extra-h", type=float, nargs="*", default=[],
                    help="--grad42: further central-difference steps to report besides h = 1e-3")
    ap.add_argument("--grad42", action="store_true",
                    help="42-qubit gradient configuration (adjoint vs finite differences) instead")
    ap.add_argument("--many", action="store_true",
                    help="time the batched uneven workload of many circuits instead")
    ap.add_argument("--executor-sweep", action="store_true",
                    help="time both executors on grid circuits of 12 to 30 qubits (calibrates the automatic choice)")
    ap.add_argument("--persist-demo", action="store_true",
                    help="time the persistent executor against per-level launches on a 24-qubit network instead")
    ap.add_argument("--bitstrings", type=int, default=0,
                    help="time B correlated bitstrings of the 30-qubit workload (leaf variants) instead")
    ap.add_argument("--bitstring-path", default="stem", choices=["stem", "greedy"],
                    help="--bitstrings: contraction path (stem: projections last, unsliced)")
    ap.add_argument("--stem", action="store_true",
                    help="time fused stem groups against separate launches on a 28-qubit stem path instead")
    ap.add_argument("--stem-grid", default="4x7", help="--stem: grid of the circuit (ROWSxCOLS)")
    ap.add_argument("--stem-cap-log2", type=int, default=None,
                    help="--stem, --bitstrings: the stem_cap_log2 option of the fused groups (default: the library's)")
    ap.add_argument("--stem-no-unfused", action="store_true",
                    help="--stem: skip the unfused baseline (for sweeps of the fusion options)")
    ap.add_argument("--stem-coalesce-bits", type=int, default=None,
                    help="--stem, --bitstrings: the stem_coalesce_bits option (default: the library's)")
    ap.add_argument("--backward", action="store_true",
                    help="time the adjoint pass (leaf environments of all fSim gates) instead")
    ap.add_argument("--single-node", default=None,
                    help="MB,NB,KB: time one isolated contraction node (log2 sizes) instead")
    ap.add_argument("--slices-per-step", type=int, default=None,
                    help="slices per tnc_contract call (default 4 for the 30-qubit line, 2 for the other modes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.slices_per_step is None:
        plain = not (args.grad42 or args.c53 or args.many or args.backward or args.single_node or args.stem or
                     args.persist_demo)
        args.slices_per_step = 4 if plain else (8 if args.persist_demo else 2)
    if args.mode is None:
        if args.grad42:
            args.mode = "fp32"
        elif args.single_node or args.backward or args.many or args.persist_demo or args.impl == "reference":
            args.mode = "bf16"
        else:
            args.mode = "fp16x2"

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.single_node:
        return single_node(args)
    if args.backward:
        return backward_bench(args)
    if args.stem:
        return stem_bench(args)
    if args.bitstrings:
        return bitstrings_bench(args)
    if args.persist_demo:
        return persist_demo(args)
    if args.executor_sweep:
        return executor_sweep(args)
    if args.many:
        return many_bench(args)
    if args.grad42:
        return grad42_bench(args)
    if args.c53:
        return c53_bench(args)

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_2205_00393_gb300 import Network, tune_table

    c, ref_net = build_network()
    net = Network.from_tn(ref_net)
    path = net.greedy_path()
    net.set_path(path)
    S = net.find_slices(WORKLOAD["target_log2"], WORKLOAD["sa_seed"])
    net.set_slices(S)
    apply_options(net, args)
    n_slices = net.n_slices
    B = args.slices_per_step
    mode = MODES[args.mode]
    if mode != 0 and not args.no_autotune:
        net.autotune(mode, 0)  # setup: kernel choice per contraction shape
    ws = torch.empty(net.workspace_bytes(B), dtype=torch.uint8, device="cuda")
    net.set_workspace(ws)
    stats = net.stats()
    stream = torch.cuda.current_stream()
    out = torch.empty(net.n_out, dtype=torch.complex128, device="cuda")

    from paper_2205_00393_gb300.shard import step_range

    def slice_range(step):  # disjoint slice blocks per rank (weak scaling, no data-path collective)
        return step_range(step, world, rank, B, n_slices)

    def barrier():
        if world > 1:
            dist.barrier()

    for i in range(args.warmup):
        lo, hi = slice_range(i)
        net.contract(lo, hi, mode, out=out)
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs
    net.set_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flops = 0
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for i in range(args.steps):
            lo, hi = slice_range(args.warmup + i)
            net.contract(lo, hi, mode, out=out)
            flops += node_flops(stats, hi - lo)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    T = ev0.elapsed_time(ev1) / 1e3
    recs, n_launches = net.last_timings()
    persist_tc = net.stats()["timed_persist_tc_cmacs"]
    net.set_timing(False)
    n_sl_done = sum(slice_range(args.warmup + i)[1] - slice_range(args.warmup + i)[0]
                    for i in range(args.steps))
    if world > 1:
        t = torch.tensor([T], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        T = float(t.item())
        f = torch.tensor([flops, n_sl_done], device="cuda", dtype=torch.float64)
        dist.all_reduce(f)
        flops, n_sl_tot = float(f[0].item()), int(f[1].item())
    else:
        n_sl_tot = n_sl_done
    value = flops / T / 1e12

    # ---- dominant kernel roofline (per-launch CUDA events over the timed region)
    by_kind = kernel_breakdown(recs)
    peaks, peak_src = load_peaks()
    probed = probe_peaks()
    roofline = roofline_of(by_kind, args.mode, peaks, peak_src, sustained=True, probed=probed,
                           persist_tc_cmacs=persist_tc)

    # ---- end to end through the public API with host buffers
    leaf_bytes = net.leaf_bytes()
    packed = np.concatenate([np.asarray(t, dtype=np.complex64).reshape(-1) for t in ref_net.tensors])
    host_in = torch.from_numpy(packed.view(np.float32).copy()).pin_memory()
    host_out = torch.empty(net.n_out, dtype=torch.complex128).pin_memory()
    e2e_steps = max(2, min(args.steps, 4))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        lo, hi = slice_range(i)
        net.upload_leaves(host_in.data_ptr(), stream)
        net.contract(lo, hi, mode, out=out)
        host_out.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
    Te = time.perf_counter() - t0
    e2e_flops = sum(node_flops(stats, slice_range(i)[1] - slice_range(i)[0]) for i in range(e2e_steps))
    if world > 1:
        t = torch.tensor([Te], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        Te = float(t.item())
        e2e_flops *= world
    e2e = {"value": e2e_flops / Te / 1e12, "unit": UNIT, "h2d_bytes_per_step": leaf_bytes,
           "d2h_bytes_per_step": net.n_out * 16}

    # ---- the sharded sum: slices [0, world * B) dealt to the ranks in blocks of B,
    # partial sums added by one all-reduce; rank 0 checks the total against its
    # own contraction of the same slices (untimed)
    from paper_2205_00393_gb300.shard import sharded_sum
    v_hi = min(world * B, n_slices)
    total = sharded_sum(lambda a, b: net.contract(a, b, mode, out=out).clone(), 0, v_hi, B, world, rank)
    shard_check = None
    if rank == 0:
        one = net.contract(0, v_hi, mode, out=out).cpu().numpy()
        shard_check = {"slices": [0, v_hi], "ranks": world,
                       "max_rel_diff_vs_one_rank": float(np.max(np.abs(total - one)) / np.max(np.abs(one)))}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16x3/f32", "tf32": "tf32x2/f32", "bf16x2": "bf16x2/f32",
                  "fp16x2": "f16x2/f32"}[args.mode],
        "arithmetic": {"fp32": "complex64 products and sums in FP32 on the CUDA cores",
                       "bf16": "complex64 operands split into 3 BF16 parts, 6 part pairs on the tensor cores, FP32 accumulation",
                       "tf32": "complex64 operands split into 2 TF32 parts, 3 part pairs on the tensor cores, FP32 accumulation",
                       "bf16x2": "complex64 operands split into 2 BF16 parts, 3 part pairs on the tensor cores, FP32 accumulation",
                       "fp16x2": "complex64 operands scaled by 2^e per row (column) and 256 of K, split into 2 FP16 parts, "
                                 "3 part pairs on the tensor cores, FP32 accumulation"}[args.mode],
        "data": "synthetic",
        "s_per_1024_slices": T / n_sl_tot * 1024,
        "gpu_s_per_1024_slices": T * world / n_sl_tot * 1024,
        "config": {"workload": workload_name(), "n_slices": n_slices, "sliced": len(S),
                   "eq3_overhead": round(float(stats["overhead"]), 5)},
        "mode": args.mode, "slices_per_step": B, "l2": "working set > L2 (1 GiB intermediates), no flush",
        "parallelism": "slices sharded over ranks" if world > 1 else "1 GPU",
        "roofline": roofline, "clocks": clk.summary(), "e2e": e2e, "gpu_launches": n_launches,
        "executor": executor_of(by_kind),
        "sharded_sum_check": shard_check, "peaks_probed": probed,
        "kernel_time_ms": {KIND_NAMES[k]: v["ms"] for k, v in by_kind.items()},
        "top_nodes": top_nodes(recs, stats),
        "tuned_shapes": [e for e in tune_table() if e[0] == mode],
    }
    if args.mode != "fp32" and not args.no_fp32_compare:
        # the plain FP32 CUDA-core path on the same slices, for the split-TC / FP32 ratio
        for i in range(2):
            lo, hi = slice_range(i)
            net.contract(lo, hi, MODES["fp32"], out=out)
        torch.cuda.synchronize()
        barrier()
        net.set_timing(True)
        ev0.record(stream)
        f32_flops = 0
        for i in range(args.steps):
            lo, hi = slice_range(args.warmup + i)
            net.contract(lo, hi, MODES["fp32"], out=out)
            f32_flops += node_flops(stats, hi - lo)
        ev1.record(stream)
        torch.cuda.synchronize()
        Tf = ev0.elapsed_time(ev1) / 1e3
        f_recs, _ = net.last_timings()
        net.set_timing(False)
        line["fp32_roofline"] = roofline_of(kernel_breakdown(f_recs), "fp32", peaks, peak_src, sustained=True,
                                            probed=probed)
        line["fp32_executor"] = executor_of(kernel_breakdown(f_recs))
        if world > 1:
            t = torch.tensor([Tf], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            Tf = float(t.item())
            f32_flops *= world
        line["fp32_value"] = f32_flops / Tf / 1e12
        line["speedup_vs_fp32"] = line["value"] / line["fp32_value"]
    others = [m for m in args.compare_modes.split(",") if m and m != args.mode and m != "fp32"]
    if others:
        # other split modes on the same slices: value, dominant-kernel roofline, error below
        line["split_modes"] = {}
        for m in others:
            mo = MODES[m]
            if not args.no_autotune:
                net.autotune(mo, 0)
            for i in range(args.warmup):
                lo, hi = slice_range(i)
                net.contract(lo, hi, mo, out=out)
            torch.cuda.synchronize()
            barrier()
            net.set_timing(True)
            ev0.record(stream)
            m_flops = 0
            for i in range(args.steps):
                lo, hi = slice_range(args.warmup + i)
                net.contract(lo, hi, mo, out=out)
                m_flops += node_flops(stats, hi - lo)
            ev1.record(stream)
            torch.cuda.synchronize()
            Tm = ev0.elapsed_time(ev1) / 1e3
            m_recs, _ = net.last_timings()
            m_tc = net.stats()["timed_persist_tc_cmacs"]
            net.set_timing(False)
            if world > 1:
                t = torch.tensor([Tm], device="cuda", dtype=torch.float64)
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                Tm = float(t.item())
                m_flops *= world
            line["split_modes"][m] = {
                "value": m_flops / Tm / 1e12, "ms_per_step": 1e3 * Tm / args.steps,
                "s_per_1024_slices": Tm / n_sl_tot * 1024,
                "roofline": roofline_of(kernel_breakdown(m_recs), m, peaks, peak_src, sustained=True,
                                        probed=probed, persist_tc_cmacs=m_tc),
                "executor": executor_of(kernel_breakdown(m_recs))}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        path_py = [tuple(p) for p in path]
        macs, dt, ref0 = run_oracle_sample(ref_net, path_py, S)
        line["cpu_baseline"] = {"value": 8 * macs / dt / 1e12, "unit": UNIT, "cores": cpu_threads(),
                                "kind": "oracle",
                                "sample": "one full slice (slice 0) of the workload, NumPy complex128 "
                                          "tensordot per node, %.1f s" % dt,
                                "c1_12q_all_16_slices": {"all_cores": oracle_c1_seconds(None),
                                                         "one_core": oracle_c1_seconds(1)}}
        rms = float(np.sqrt(np.mean(np.abs(ref0) ** 2)))

        def errs(mo):
            got = net.contract(0, 1, mo, out=out).cpu().numpy()
            d = np.abs(got - ref0)
            return (float(np.max(d / np.maximum(np.abs(ref0), rms))),
                    float(np.max(d / np.maximum(np.abs(ref0), 0.1 * rms))))
        line["rel_err_vs_oracle"], line["rel_err_vs_oracle_floor_0.1rms"] = errs(mode)
        for m in line.get("split_modes", {}):
            e1, e2 = errs(MODES[m])
            line["split_modes"][m]["rel_err_vs_oracle"] = e1
            line["split_modes"][m]["rel_err_vs_oracle_floor_0.1rms"] = e2
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
