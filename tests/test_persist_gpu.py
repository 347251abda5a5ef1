"""The persistent executor: one launch per batch of slices in which one CTA
per SM takes tasks (FP32 tiles, operand splits, tensor-core tiles, K-split
reductions, final-contraction chunks and their ordered sums) from a device
work list, each waiting on counters of the contractions that produce its
inputs: per batch entry when every tensor of the batch has bytes of its own
("persist_deps", the default when that fits), else per stage behind a chain
of tree levels. Either way it runs the same arithmetic in the same order as
the separate launches, so results are bit-identical to them, and they match
the FP64 oracle. A dependency wait that runs out reports TNC_E_TIMEOUT without a
fault (no task ever signals the counter it waits on) and leaves the context
usable."""

import numpy as np
import pytest

from tnc_inputs import circuit_to_network, grid_rqc
from oracle import tn

from ._util import floored_rel_err
from .test_parity_tc_gpu import _three_leaf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(libtnc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return libtnc


def _run(net, lo, hi, mode, persistent, deps=1, expect=None):
    net.set_option("persistent", persistent)
    net.set_option("persist_deps", deps)
    net.set_timing(True)
    got = net.contract(lo, hi, mode).cpu().numpy()
    recs, n = net.last_timings()
    net.set_timing(False)
    net.check_device()
    kinds = [r["kind"] for r in recs]
    if 9 in kinds:
        assert net.stats()["last_persist_deps"] == (deps if expect is None else expect)
    return got, kinds


def _grid(rows, cols, cycles, seed, n_open, t):
    from paper_2205_00393_gb300 import Network
    c = grid_rqc(rows, cols, cycles, seed, n_open=n_open)
    ref_net = circuit_to_network(c).as_complex64()
    net = Network.from_tn(ref_net)
    path = net.greedy_path()
    net.set_path(path)
    S = net.find_slices(t, 7)
    net.set_slices(S)
    return ref_net, net, path, S


@pytest.mark.parametrize("deps", [1, 0])
@pytest.mark.parametrize("mode", [0, 2, 4])
def test_persistent_equals_launches_12q(lib, mode, deps):
    ref_net, net, path, S = _grid(3, 4, 8, 1, 0, 8)
    per, kinds = _run(net, 0, net.n_slices, mode, 1, deps)
    assert kinds == [9], kinds  # one launch per batch (all 16 slices in one batch)
    leg, kinds0 = _run(net, 0, net.n_slices, mode, 0)
    assert 9 not in kinds0
    assert np.array_equal(per, leg)
    ref = tn.contract(ref_net, path, S)
    assert floored_rel_err(per, ref, 12) <= (1e-5 if mode == 0 else 1e-4)


@pytest.mark.parametrize("deps", [1, 0])
@pytest.mark.parametrize("mode", [2, 4, 1, 0])
def test_persistent_equals_launches_24q_tensor_cores(lib, mode, deps):
    """24-qubit 4x6 grid, 12 cycles, 4 open qubits, t = 20: tensor-core
    contractions (splits, tiles) and small FP32 ones; slices [1, 5) in one
    batch, then [0, 3) and [3, 7) with invariants cached."""
    ref_net, net, path, S = _grid(4, 6, 12, 3, 4, 20)
    per, kinds = _run(net, 1, 5, mode, 1, deps)
    leg, _ = _run(net, 1, 5, mode, 0)
    assert kinds.count(9) >= 1 and set(kinds) == {9}, kinds
    assert np.array_equal(per, leg)
    ref = tn.contract(ref_net, path, S, slices=range(1, 5))
    assert floored_rel_err(per, ref, 24) <= (1e-5 if mode == 0 else 1e-4)
    net.set_option("cache_invariants", 1)
    a, _ = _run(net, 0, 3, mode, 1, deps)
    b, _ = _run(net, 3, 7, mode, 1, deps)
    net.set_option("cache_invariants", 0)
    c, _ = _run(net, 0, 7, mode, 0)
    assert float(np.max(np.abs(a + b - c)) / np.max(np.abs(c))) <= 1e-12


@pytest.mark.parametrize("deps", [1, 0])
@pytest.mark.parametrize("mode", [4, 2])
def test_persistent_k_splits(lib, mode, deps):
    """(2^7, 2^7, 2^16): few output tiles, K split over CTAs; the persistent
    executor runs the split tiles and the K-split reduction as tasks."""
    from paper_2205_00393_gb300 import Network
    net_ref = _three_leaf(401, 7, 7, 16, False)
    net = Network.from_tn(net_ref)
    net.set_path([(0, 1), (2, 3)])
    per, kinds = _run(net, 0, 1, mode, 1, deps)
    leg, kinds0 = _run(net, 0, 1, mode, 0)
    assert kinds == [9] and 7 in kinds0
    assert np.array_equal(per, leg)


def test_persistent_deps_need_flat_workspace(lib):
    """A caller workspace that holds the reusing layout of a batch but not
    every tensor of it at once: the persistent executor keeps the level
    chain; one that holds them all gives the per-entry dependencies. Both
    equal the per-level launches bit for bit."""
    ref_net, net, path, S = _grid(4, 6, 12, 3, 4, 20)
    leg, _ = _run(net, 0, 4, 4, 0)
    _run(net, 0, 4, 4, 1, 1)
    reuse, flat = net.stats()["last_workspace"]
    assert flat > reuse > 0
    for size, deps in ((reuse, 0), (flat, 1)):
        ws = torch.empty((size + 255) // 256 * 256, dtype=torch.uint8, device="cuda")
        net.set_workspace(ws)
        got, kinds = _run(net, 0, 4, 4, 1, 1, expect=deps)
        assert kinds == [9]
        assert np.array_equal(got, leg)
    net.set_workspace(None)


def test_persistent_wait_timeout(lib):
    """A test-only task waits on a counter that no task decrements: the wait
    gives up after 20 ms and reports TNC_E_TIMEOUT; the next contraction on
    the same network is correct."""
    from paper_2205_00393_gb300 import TNCError
    ref_net, net, path, S = _grid(3, 4, 8, 1, 0, 8)
    net.set_option("persist_wait_ms", 20)
    net.set_option("persist_test_stall", 1)
    net.contract(0, net.n_slices, 2)
    with pytest.raises(TNCError) as e:
        net.check_device()
    assert e.value.status == 4
    net.set_option("persist_test_stall", 0)
    net.set_option("persist_wait_ms", 0)
    got = net.contract(0, net.n_slices, 2).cpu().numpy()
    net.check_device()
    assert floored_rel_err(got, tn.contract(ref_net, path, S), 12) <= 1e-4


def test_automatic_executor_choice(lib):
    """Default ("persistent" = 2): the 12-qubit call (16 slices, contractions
    of at most a few thousand MACs) is launch-bound and runs as one
    persistent launch; four slices of the 24-qubit circuit (where the
    per-level launches are faster) and two slices of the 30-qubit workload
    (contractions of 2^38 MACs) run one launch per tree level."""
    _, net, _, _ = _grid(3, 4, 8, 1, 0, 8)
    net.set_timing(True)
    net.contract(0, net.n_slices, 2)
    assert [r["kind"] for r in net.last_timings()[0]] == [9]
    _, mid, _, _ = _grid(4, 6, 12, 3, 4, 20)
    mid.set_timing(True)
    mid.contract(0, 4, 4)
    assert 9 not in {r["kind"] for r in mid.last_timings()[0]}
    mid.set_timing(False)
    _, big, _, _ = _grid(5, 6, 14, 2, 6, 27)
    big.set_timing(True)
    big.contract(0, 2, 4)
    kinds = {r["kind"] for r in big.last_timings()[0]}
    big.set_timing(False)
    big.check_device()
    assert 9 not in kinds and 3 in kinds
