"""53-qubit lattice (6x9 grid minus one site), 20 cycles, sliced to 2^30-
element intermediates: one slice in split BF16 and split TF32 on the tensor
cores against the GPU FP32 path (the FP64 oracle cannot run at this size:
2^44 complex multiply-accumulates and 8 GiB tensors per slice)."""

import pytest

from tnc_inputs import circuit_to_network, lattice_53q_rqc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_53q_one_slice_split_vs_fp32(libtnc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_00393_gb300 import Network
    c = lattice_53q_rqc(20, 3)
    net = Network.from_tn(circuit_to_network(c).as_complex64())
    net.set_path(net.greedy_path())
    net.set_slices(net.find_slices(30, 7))
    assert max(n[0] + n[1] for n in net.stats()["nodes"]) <= 30
    s = 3
    ref = net.contract(s, s + 1, 0).cpu().numpy()[0]
    for mode in (2, 1):
        got = net.contract(s, s + 1, mode).cpu().numpy()[0]
        net.check_device()
        assert abs(got - ref) <= 1e-4 * abs(ref), (mode, got, ref)
