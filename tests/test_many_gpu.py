"""tnc_contract_many: several circuits of uneven size in shared launches and
a replayed CUDA graph must give the same amplitudes as separate contractions
and as the FP64 oracle. Both executors: merged per-level launches, and the
persistent work-list kernel (one launch per round of slice batches, every
circuit's tasks in it, levels interleaved)."""

import numpy as np
import pytest

from tnc_inputs import circuit_to_network, grid_rqc
from oracle import tn

from ._util import floored_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _circuits():
    specs = [(3, 4, 8, 1, 0, 8), (2, 4, 6, 2, 2, 6), (3, 3, 7, 3, 1, 7), (4, 5, 10, 4, 3, 15),
             (2, 3, 5, 5, 0, None), (3, 5, 9, 6, 6, 11)]
    out = []
    from paper_2205_00393_gb300 import Network
    for (r, c, cyc, seed, n_open, t) in specs:
        circ = grid_rqc(r, c, cyc, seed, n_open=n_open)
        ref = circuit_to_network(circ).as_complex64()
        net = Network.from_tn(ref)
        path = net.greedy_path()
        net.set_path(path)
        S = net.find_slices(t, 7) if t is not None else []
        net.set_slices(S)
        out.append((circ, ref, net, path, S))
    return out


def _launches_of_replay(nets, ranges, mode, outs, stream):
    """Kernels one graph replay of the call launches (counted on nets[0])."""
    from paper_2205_00393_gb300 import contract_many
    nets[0].set_timing(True)
    contract_many(nets, ranges, mode, outs=outs, stream=stream)
    stream.synchronize()
    _, n = nets[0].last_timings()
    nets[0].set_timing(False)
    return n


@pytest.mark.parametrize("persistent,deps", [(0, 1), (1, 1), (1, 0)])
@pytest.mark.parametrize("mode", [0, 2, 4])
def test_many_matches_single_and_oracle(libtnc, mode, persistent, deps):
    """persistent 1 with deps 1: every circuit's tasks wait only on their own
    inputs per batch entry; deps 0: on the whole previous level of their
    circuit."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_00393_gb300 import contract_many
    cs = _circuits()
    nets = [c[2] for c in cs]
    for n in nets:
        n.set_option("persistent", persistent)
        n.set_option("persist_deps", deps)
    ranges = [(0, n.n_slices) for n in nets]
    ranges[3] = (1, nets[3].n_slices - 1)  # a partial range
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        outs = [torch.empty(n.n_out, dtype=torch.complex128, device="cuda") for n in nets]
        for call in range(3):  # eager, capture + replay, replay
            for o in outs:
                o.fill_(float("nan"))
            contract_many(nets, ranges, mode, outs=outs, stream=stream)
            stream.synchronize()
            if call == 0:
                assert [n.stats()["last_persist_deps"] for n in nets] == [persistent * deps] * len(nets)
            for (circ, ref, net, path, S), (lo, hi), o in zip(cs, ranges, outs):
                single = net.contract(lo, hi, mode, stream=stream).cpu().numpy()
                stream.synchronize()
                got = o.cpu().numpy()
                assert np.allclose(got, single, rtol=1e-9, atol=1e-15), call
                if call == 0:
                    want = tn.contract(ref, path, S, range(lo, hi))
                    assert floored_rel_err(got, want, circ.n_qubits) <= (1e-5 if mode == 0 else 1e-4)
        launches = _launches_of_replay(nets, ranges, mode, outs, stream)
        for n in nets:
            n.set_option("persistent", 1 - persistent)
        other = _launches_of_replay(nets, ranges, mode, outs, stream)
    # the persistent executor launches one kernel per round of slice batches
    assert (launches < other) if persistent else (launches > other)


def test_many_rejects_duplicates(libtnc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_00393_gb300 import contract_many, TNCError
    cs = _circuits()
    with pytest.raises(TNCError):
        contract_many([cs[0][2], cs[0][2]])


@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("mode", [0, 2])
def test_batched_uneven_workload_subset(libtnc, mode, persistent):
    """First 48 circuits of the seeded batched workload (those whose slices
    cost at most 2^32 complex MACs), two slices each: the merged launches
    (or the persistent kernel) with graph replay equal separate
    contractions."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from bench import batched_circuits
    from paper_2205_00393_gb300 import contract_many
    kept, dropped = batched_circuits(n=48, cost_cap=2 ** 32)
    assert len(kept) >= 20
    nets = [e["net"] for e in kept]
    for n in nets:
        n.set_option("persistent", persistent)
    ranges = [(0, min(2, e["slices"])) for e in kept]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        outs = [torch.empty(n.n_out, dtype=torch.complex128, device="cuda") for n in nets]
        for call in range(3):
            contract_many(nets, ranges, mode, outs=outs, stream=stream)
        stream.synchronize()
        for net, (lo, hi), o in zip(nets, ranges, outs):
            single = net.contract(lo, hi, mode, stream=stream).cpu().numpy()
            assert np.allclose(o.cpu().numpy(), single, rtol=1e-9, atol=1e-15)
