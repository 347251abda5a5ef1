"""Full-size parity: the 30-qubit 5x6 grid circuit (14 cycles, 6 open qubits,
sliced to 2^27-element intermediates), one slice against the FP64 oracle,
in the launch configuration the benchmark times."""

import pytest

from tnc_inputs import circuit_to_network, grid_rqc
from oracle import tn

from ._util import floored_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2(libtnc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_00393_gb300 import Network
    c = grid_rqc(5, 6, 14, 2, n_open=6)
    ref_net = circuit_to_network(c).as_complex64()
    net = Network.from_tn(ref_net)
    path = net.greedy_path()
    net.set_path(path)
    S = net.find_slices(27, 7)
    net.set_slices(S)
    return ref_net, net, path, S


def test_c2_one_slice_fp32(c2):
    ref_net, net, path, S = c2
    s = 5
    got = net.contract(s, s + 1, 0)
    torch.cuda.synchronize()
    ref = tn.contract_slice(ref_net, path, S, s)
    got = got.cpu().numpy()
    print("c2 slice %d: err(floor=0.1rms)=%.3e err(floor=rms)=%.3e" % (
        s, floored_rel_err(got, ref, 30), floored_rel_err(got, ref, 30, floor=1.0)))
    assert floored_rel_err(got, ref, 30) <= 1e-5
