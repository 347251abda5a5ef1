"""tnc_autotune: timing FP32 vs tensor-core kernels per contraction shape
fills the process-wide table (choices 0 = FP32, 32 / 64 = tensor-core row
width); results after tuning still match the FP32 path."""

import pytest

from .test_parity_tc_gpu import _three_leaf
from ._util import floored_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autotune_table_and_results(libtnc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_00393_gb300 import Network, tune_table
    net_ref = _three_leaf(31, 10, 9, 9, True)
    net = Network.from_tn(net_ref)
    net.set_path([(0, 1), (2, 3)])
    ref = net.contract(0, 1, 0).cpu().numpy()
    net.autotune(2, 0)
    table = tune_table()
    entry = [e for e in table if e[0] == 2 and sorted(e[1:3]) == [9, 10] and e[3] == 9]
    assert len(entry) == 1 and entry[0][4] in (0, 32, 64)
    got = net.contract(0, 1, 2).cpu().numpy()
    net.check_device()
    assert floored_rel_err(got, ref, 0) <= 1e-4
