"""GPU parity: libtnc's CUDA path against the FP64 oracle, element by element.

All inputs are seeded synthetic circuits of the paper's gate family. The
oracle contracts the same complex64-rounded leaves in complex128. Tolerance:
FP32 path 1e-5 relative per amplitude (floored metric of tests/_util.py).
"""

import numpy as np
import pytest

from tnc_inputs import circuit_to_network, grid_rqc
from oracle import planner, statevector, tn

from ._util import floored_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def lib(libtnc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return libtnc


def _setup(rows, cols, cyc, seed, n_open, t, sa_seed=7):
    from paper_2205_00393_gb300 import Network
    c = grid_rqc(rows, cols, cyc, seed, n_open=n_open)
    ref_net = circuit_to_network(c).as_complex64()
    net = Network.from_tn(ref_net)
    path = net.greedy_path()
    net.set_path(path)
    S = net.find_slices(t, sa_seed) if t is not None else []
    net.set_slices(S)
    return c, ref_net, net, path, S


def _gpu(net, lo, hi, mode=0):
    out = net.contract(lo, hi, mode)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_c1_all_slices_vs_oracle_and_statevector(lib):
    c, ref_net, net, path, S = _setup(3, 4, 8, 1, 0, 8)
    assert len(S) == 4
    got = _gpu(net, 0, 16)
    ref = tn.contract(ref_net, path, S)
    assert floored_rel_err(got, ref, 12) <= TOL_FP32
    sv = statevector.amplitudes(c)
    assert floored_rel_err(got, sv, 12) <= TOL_FP32


@pytest.mark.parametrize("lo,hi", [(0, 1), (3, 11), (15, 16), (5, 5)])
def test_c1_slice_subranges(lib, lo, hi):
    c, ref_net, net, path, S = _setup(3, 4, 8, 1, 0, 8)
    got = _gpu(net, lo, hi)
    ref = tn.contract(ref_net, path, S, range(lo, hi))
    if hi == lo:
        assert np.all(got == 0)
    else:
        assert floored_rel_err(got, ref, 12) <= TOL_FP32


def test_open_outputs(lib):
    c, ref_net, net, path, S = _setup(3, 3, 6, 2, 3, 5)
    got = _gpu(net, 0, net.n_slices)
    ref = tn.contract(ref_net, path, S)
    assert got.shape == (8,)
    assert floored_rel_err(got, ref, 9) <= TOL_FP32


def test_all_open_normalised(lib):
    # 2^8 outputs: the root goes through the GEMM + FP64 slice-sum path; two
    # closed indices are sliced by hand (slicing is exact for any closed set)
    c, ref_net, net, path, S = _setup(2, 4, 5, 9, 8, None)
    closed = sorted(e for e in range(len(ref_net.dims)) if e not in ref_net.open_ids)
    S = [closed[len(closed) // 3], closed[2 * len(closed) // 3]]
    net.set_slices(S)
    assert net.n_slices == 4
    got = _gpu(net, 0, net.n_slices)
    ref = tn.contract(ref_net, path, S)
    assert floored_rel_err(got, ref, 8) <= TOL_FP32
    assert abs(np.sum(np.abs(got) ** 2) - 1) < 1e-5


def test_unsliced(lib):
    c, ref_net, net, path, S = _setup(3, 4, 8, 1, 2, None)
    assert net.n_slices == 1
    got = _gpu(net, 0, 1)
    ref = tn.contract(ref_net, path)
    assert floored_rel_err(got, ref, 12) <= TOL_FP32


def test_multi_tile_ragged(lib):
    # intermediates up to 2^20: GEMMs span many 64x64 tiles with ragged edges
    c, ref_net, net, path, S = _setup(4, 6, 12, 4, 3, 20)
    sl = list(range(0, net.n_slices, 37))
    ref = sum(tn.contract_slice(ref_net, path, S, s) for s in sl)
    got = sum(_gpu(net, s, s + 1) for s in sl)
    assert floored_rel_err(got, ref, 24) <= TOL_FP32


def test_batched_workspace_matches_unbatched(lib):
    c, ref_net, net, path, S = _setup(4, 5, 12, 7, 2, 16)
    n = net.n_slices
    one = net.workspace_bytes(1)
    ws1 = torch.empty(one, dtype=torch.uint8, device="cuda")
    net.set_workspace(ws1)
    a = _gpu(net, 0, n)
    big = net.workspace_bytes(n)
    wsn = torch.empty(big, dtype=torch.uint8, device="cuda")
    net.set_workspace(wsn)
    b = _gpu(net, 0, n)
    assert net.stats()["last_batch"] == n
    assert np.allclose(a, b, rtol=1e-12, atol=1e-15)
    ref = tn.contract(ref_net, path, S)
    assert floored_rel_err(b, ref, 20) <= TOL_FP32


def test_single_leaf_network(lib):
    from paper_2205_00393_gb300 import Network
    rng = np.random.default_rng(0)
    t = (rng.standard_normal((2, 2, 2)) + 1j * rng.standard_normal((2, 2, 2))).astype(np.complex64)
    net = Network([t], [(0, 1, 2)], [2, 2, 2], [2, 0, 1])
    net.set_path([])
    got = _gpu(net, 0, 1)
    assert np.allclose(got, np.transpose(t, (2, 0, 1)).reshape(-1), atol=1e-7)


def test_set_tensor_data_updates_result(lib):
    c, ref_net, net, path, S = _setup(3, 4, 8, 1, 0, 8)
    a = _gpu(net, 0, 16)
    i = next(k for k, g in enumerate(ref_net.leaf_gate) if g >= 0 and c.gates[g].name == "fsim")
    new = (ref_net.tensors[i] * np.complex64(0.5j)).astype(np.complex64)
    net.set_tensor_data(i, new)
    b = _gpu(net, 0, 16)
    assert floored_rel_err(b, a * 0.5j, 12) <= TOL_FP32


def test_invalid_range_and_mode(lib):
    from paper_2205_00393_gb300 import TNCError
    c, ref_net, net, path, S = _setup(3, 4, 8, 1, 0, 8)
    with pytest.raises(TNCError):
        net.contract(0, 17)
    with pytest.raises(TNCError):
        net.contract(3, 2)
    with pytest.raises(TNCError):
        net.contract(0, 1, mode=9)


@pytest.mark.parametrize("persistent", [0, 1])
def test_cached_invariants(lib, persistent):
    """cache_invariants: the second call reuses the slice-invariant tensors
    (fewer complex multiply-accumulates run) with identical results; changing
    a leaf recomputes them. Both executors: one launch per contraction level,
    and the persistent one."""
    c, ref_net, net, path, S = _setup(4, 5, 12, 7, 2, 16)
    net.set_option("persistent", persistent)
    n = net.n_slices
    base = _gpu(net, 0, n)
    net.set_option("cache_invariants", 1)
    net.set_timing(True)
    a = _gpu(net, 0, n)
    r1, l1 = net.last_timings()
    net.set_timing(True)
    b = _gpu(net, 0, n)
    r2, l2 = net.last_timings()
    net.set_timing(False)
    assert np.array_equal(a, base) and np.array_equal(b, base)
    assert sum(r["cmacs"] for r in r2) < sum(r["cmacs"] for r in r1)
    assert l2 <= l1
    # change a leaf that no sliced index touches: the cache must be refreshed
    tree = planner.Tree(ref_net.indices, ref_net.dims, ref_net.open_ids, path)
    i = next(v for v in range(ref_net.n_tensors)
             if len(ref_net.indices[v]) == 4 and not set(ref_net.indices[v]) & set(S))
    new = (ref_net.tensors[i] * np.complex64(-1j)).astype(np.complex64)
    net.set_tensor_data(i, new)
    got = _gpu(net, 0, n)
    ts = list(ref_net.tensors)
    ts[i] = new
    want = tn.contract(ref_net.with_tensors(ts), path, S)
    assert floored_rel_err(got, want, 20) <= TOL_FP32
