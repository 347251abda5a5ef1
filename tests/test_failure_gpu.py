"""Failure detection on the GPU without a fault: a bounded device-side wait is
made to run out (the tensor-core producer issues no loads, so the barrier the
MMA thread waits on is never completed). The kernel must record
TNC_E_TIMEOUT, release its tensor memory and return; the context must stay
usable, and the next contraction must be correct."""

import pytest

from oracle import tn

from .test_parity_tc_gpu import _three_leaf
from ._util import floored_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mb,nb", [(7, 7), (8, 7), (7, 8)])
def test_bounded_wait_timeout_reports_and_recovers(libtnc, mb, nb):
    """One to two 128x128 output tiles, each on one CTA: every CTA's MMA
    wait runs out and raises its abort flag."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_00393_gb300 import Network, TNCError
    net_ref = _three_leaf(7, mb, nb, 6, False)
    net = Network.from_tn(net_ref)
    path = [(0, 1), (2, 3)]
    net.set_path(path)
    net.set_option("tc_spin_limit", 1 << 14)
    net.set_option("tc_test_stall", 1)
    net.contract(0, 1, 2)
    with pytest.raises(TNCError) as e:
        net.check_device()
    assert e.value.status == 4  # TNC_E_TIMEOUT
    # the context is intact: a normal contraction on the same network is correct
    net.set_option("tc_test_stall", 0)
    net.set_option("tc_spin_limit", 0)
    got = net.contract(0, 1, 2)
    net.check_device()
    ref = tn.contract(net_ref, path)
    assert floored_rel_err(got.cpu().numpy(), ref, 0) <= 1e-4
