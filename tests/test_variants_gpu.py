"""Leaf variants on the GPU (correlated amplitudes, Sec. 1 and 6.2): B closed
bitstrings of one circuit in one tnc_contract_variants call. Each variant is
compared with the FP64 oracle on the network that carries that bitstring's
projection vectors (same path and slicing set), and with an ordinary
contraction of that network. The slice-invariant part is computed once for
all variants: the call runs fewer complex multiply-accumulates than B
single-variant calls."""

import json
import os

import numpy as np
import pytest

from oracle import tn
from tnc_inputs import bitstring_variants, circuit_to_network, grid_rqc, random_bitstrings

from ._util import floored_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 2: 1e-4, 4: 1e-4}
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rqc30_bitstrings.json")


@pytest.fixture(scope="module")
def lib(libtnc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return libtnc


def _net(c, bitstring=None, t=None):
    from paper_2205_00393_gb300 import Network
    ref = circuit_to_network(c, bitstring=bitstring).as_complex64()
    net = Network.from_tn(ref)
    path = net.greedy_path()
    net.set_path(path)
    S = net.find_slices(t, 7) if t is not None else []
    net.set_slices(S)
    return ref, net, [tuple(p) for p in path], S


@pytest.mark.parametrize("persistent", [1, 0])
@pytest.mark.parametrize("mode", [0, 2, 4])
@pytest.mark.parametrize("n_open", [0, 2])
def test_bitstring_batch_12q(lib, mode, n_open, persistent):
    """3x4 grid, 8 cycles, sliced to 2^8 elements; 32 bitstrings (seed 5)."""
    c = grid_rqc(3, 4, 8, 1, n_open=n_open)
    ref, net, path, S = _net(c, t=8)
    net.set_option("persistent", persistent)
    bits = random_bitstrings(c, 32, 5)
    leaves, data = bitstring_variants(c, bits)
    net.set_leaf_variants(leaves, data)
    net.set_timing(True)
    got = net.contract_variants(0, 32, 0, net.n_slices, mode).cpu().numpy()
    all_cmacs = sum(r["cmacs"] for r in net.last_timings()[0])
    # variant 5 alone through tnc_contract (slice ids 5 * 2^|S| + s), shared part included
    net.set_timing(True)
    ns = net.n_slices
    one = net.contract(5 * ns, 6 * ns, mode).cpu().numpy()
    one_cmacs = sum(r["cmacs"] for r in net.last_timings()[0])
    net.set_timing(False)
    net.check_device()
    assert got.shape == (32, 1 << n_open)
    assert np.array_equal(one, got[5])
    shared = (32 * one_cmacs - all_cmacs) / 31  # the part run once instead of 32 times
    assert shared > 0
    want = np.stack([tn.contract(circuit_to_network(c, bitstring=b).as_complex64(), path, S) for b in bits])
    err = floored_rel_err(got, want.reshape(got.shape), 12)
    print("mode %d open %d: 32 bitstrings, err %.3e, cmacs %.3g vs 32 x %.3g (shared %.3g)" % (
        mode, n_open, err, all_cmacs, one_cmacs, shared))
    assert err <= TOL[mode]
    for v in (0, 31):  # the ordinary contraction of that bitstring's network
        _, other, _, _ = _net(c, bitstring=bits[v], t=8)
        assert other.sliced == net.sliced
        single = other.contract(0, other.n_slices, mode).cpu().numpy()
        assert floored_rel_err(got[v], single, 12) <= 1e-6


@pytest.mark.parametrize("mode", [0, 2, 4])
def test_bitstring_batch_30q(lib, mode):
    """The 30-qubit 5x6 grid circuit (14 cycles, seed 2, 6 open qubits), sliced
    to 2^27 elements: 4 bitstrings (seed 11) over slices [0, 2), each with 64
    amplitudes, against the oracle amplitudes stored in
    tests/golden/rqc30_bitstrings.json (written by make_rqc30_bitstrings.py,
    which calls only the oracle)."""
    with open(GOLDEN) as f:
        rec = json.load(f)
    c = grid_rqc(5, 6, 14, 2, n_open=6)
    ref, net, path, S = _net(c, t=27)
    assert [int(e) for e in S] == rec["sliced"]
    bits = np.array(rec["bitstrings"], dtype=np.uint8)
    leaves, data = bitstring_variants(c, bits)
    net.set_leaf_variants(leaves, data)
    lo, hi = rec["slices"]
    got = net.contract_variants(0, len(bits), lo, hi, mode).cpu().numpy()
    net.check_device()
    want = np.array([[complex(re, im) for re, im in a] for a in rec["amplitudes"]])
    errs = [floored_rel_err(got[v], want[v], 30) for v in range(len(bits))]
    print("mode %d: 30-qubit bitstrings, errors %s" % (mode, ["%.2e" % e for e in errs]))
    assert max(errs) <= (1.5e-5 if mode == 0 else TOL[mode])


@pytest.mark.parametrize("mode", [0, 4])
def test_bitstring_batch_stem_path(lib, mode):
    """4x4 grid, 10 cycles, 2 open qubits, the time-ordered stem path (the
    projection vectors absorbed last), unsliced: the 2^16-element state is
    shared, each of 16 bitstrings (seed 9) only absorbs its projections, in
    fused stem groups whose branches are the variant leaves."""
    from paper_2205_00393_gb300 import Network
    from tnc_inputs import stem_path
    c = grid_rqc(4, 4, 10, 4, n_open=2)
    ref = circuit_to_network(c).as_complex64()
    net = Network.from_tn(ref)
    path = stem_path(ref, c)
    net.set_path(path)
    bits = random_bitstrings(c, 16, 9)
    leaves, data = bitstring_variants(c, bits)
    net.set_leaf_variants(leaves, data)
    st = net.stats()
    assert st["stem_groups"] and any(g[4] for g in st["stem_groups"])  # a per-variant fused group
    got = net.contract_variants(0, 16, 0, 1, mode).cpu().numpy()
    net.check_device()
    want = np.stack([tn.contract(circuit_to_network(c, bitstring=b).as_complex64(), path, []) for b in bits])
    err = floored_rel_err(got, want.reshape(got.shape), 16)
    print("mode %d stem path: 16 bitstrings, err %.3e" % (mode, err))
    assert err <= TOL[mode]
