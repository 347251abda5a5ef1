"""Fused stem groups on the GPU (secondary slicing, Sec. 5.2): a stem that
absorbs narrow branches keeps each sub-tensor in shared memory across the
steps of a group. Results are compared with the FP64 oracle along the same
path (FP32-path bound 1e-5, 0.1-rms floor) and with the same contraction
unfused (every step its own launch), which gives the same products summed in
the same order."""

import numpy as np
import pytest

from tnc_inputs import circuit_to_network, grid_rqc, stem_path
from oracle import tn

from ._util import floored_rel_err
from .test_stem_cpu import fig9_network

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(libtnc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return libtnc


def _kinds(net, lo, hi):
    net.set_timing(True)
    got = net.contract(lo, hi, 0).cpu().numpy()
    recs, _ = net.last_timings()
    net.set_timing(False)
    net.check_device()
    return got, [r["kind"] for r in recs]


def test_fig9_group_on_gpu(lib):
    from paper_2205_00393_gb300 import Network
    tn_, path = fig9_network()
    net = Network.from_tn(tn_)
    net.set_path(path)
    net.set_option("stem_cap_log2", 3)
    net.set_option("stem_min_outer_log2", 5)
    net.set_option("stem_coalesce_bits", 0)
    got, kinds = _kinds(net, 0, 1)
    assert kinds.count(8) == 1, kinds
    ref = tn.contract(tn_, path)
    assert floored_rel_err(got, ref, 0) <= 1e-5


@pytest.mark.parametrize("sliced", [False, True])
def test_stem_path_20_qubits(lib, sliced):
    """4x5 grid, 10 cycles, 4 open qubits (16 amplitudes), time-ordered stem
    path; sliced: two indices of the slicer's set, all 4 slices in one call
    (the groups then run on a batch of slices, branches fixed per slice)."""
    from paper_2205_00393_gb300 import Network
    c = grid_rqc(4, 5, 10, 11, n_open=4)
    tn_ = circuit_to_network(c).as_complex64()
    path = stem_path(tn_, c)
    net = Network.from_tn(tn_)
    net.set_path(path)
    S = []
    if sliced:
        S = [int(e) for e in net.find_slices(18, 7)[:2]]
        net.set_slices(S)
    hi = 1 << len(S)
    fused, kinds = _kinds(net, 0, hi)
    assert kinds.count(8) >= 10, kinds
    net.set_option("stem_cap_log2", 0)
    plain, kinds0 = _kinds(net, 0, hi)
    assert 8 not in kinds0
    ref = tn.contract(tn_, path, S)
    e_fused, e_plain = floored_rel_err(fused, ref, 20), floored_rel_err(plain, ref, 20)
    d = float(np.max(np.abs(fused - plain)) / np.max(np.abs(plain)))
    print("stem path, %d sliced: fused err %.3e, unfused err %.3e, fused vs unfused %.3e (identical: %s)" % (
        len(S), e_fused, e_plain, d, np.array_equal(fused, plain)))
    assert e_fused <= 1e-5 and e_plain <= 1e-5
    assert d <= 1e-6
