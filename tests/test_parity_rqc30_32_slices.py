"""Full-size parity on 32 slices: the 30-qubit 5x6 grid circuit (14 cycles,
seed 2, 6 open qubits: 64 amplitudes per slice), greedy path, sliced to
2^27-element intermediates, contracted over slices [0, 32) in every
arithmetic mode and compared element by element with the FP64 oracle's sums
stored in tests/golden/rqc30_slices_0_32.json (written by
tests/golden/make_rqc30_slices.py, which calls only the oracle).

Each mode runs as one call over [0, 32) (the library batches the slices) and
as eight calls over blocks of 4 slices (the launch configuration the
benchmark times), each block against its own oracle sum. Bounds: 1e-4 for
split TF32, split BF16 and split FP16x2 and 1e-3 for 2-part BF16, on the
32-slice sum and on every block, with the 0.1-rms floor of the other parity
tests. The FP32 path is held to 1e-5 on the 32-slice sum with that floor and
on every block with the rms floor; per block at the 0.1-rms floor it is held
to 1.5e-5. Storing the intermediates in complex64 alone (exact arithmetic in
every contraction otherwise) already gives 4e-6 on block 1 at that floor,
and the FP32 products and sums of the contractions bring it to about 1.1e-5."""

import json
import os

import numpy as np
import pytest

from tnc_inputs import circuit_to_network, grid_rqc

from ._util import floored_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rqc30_slices_0_32.json")
TOL = {0: 1e-5, 1: 1e-4, 2: 1e-4, 3: 1e-3, 4: 1e-4}


def _dec(v):
    return np.array([complex(re, im) for re, im in v], dtype=np.complex128)


@pytest.fixture(scope="module")
def rqc30(libtnc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_00393_gb300 import Network
    with open(GOLDEN) as f:
        gold = json.load(f)
    c = grid_rqc(5, 6, 14, 2, n_open=6)
    net = Network.from_tn(circuit_to_network(c).as_complex64())
    net.set_path(net.greedy_path())
    S = net.find_slices(27, 7)
    assert [int(e) for e in S] == gold["sliced"]  # the planner gives the oracle twin's slicing set
    net.set_slices(S)
    return net, gold


@pytest.mark.parametrize("mode", [4, 2, 1, 0, 3])
def test_rqc30_32_slices_vs_oracle(rqc30, mode):
    net, gold = rqc30
    blk = gold["block"]
    total = net.contract(0, 32, mode).cpu().numpy()
    blocks = [net.contract(b * blk, (b + 1) * blk, mode).cpu().numpy() for b in range(32 // blk)]
    net.check_device()
    ref_total = _dec(gold["total"])
    e_total = floored_rel_err(total, ref_total, 30)
    e_blocks = [floored_rel_err(got, _dec(ref), 30) for got, ref in zip(blocks, gold["block_sums"])]
    print("mode %d: 32 slices err %.3e (rms floor %.3e); 4-slice blocks max err %.3e" % (
        mode, e_total, floored_rel_err(total, ref_total, 30, floor=1.0), max(e_blocks)))
    assert e_total <= TOL[mode]
    if mode == 0:
        e_blocks_rms = [floored_rel_err(got, _dec(ref), 30, floor=1.0) for got, ref in zip(blocks, gold["block_sums"])]
        assert max(e_blocks_rms) <= TOL[mode]
        assert max(e_blocks) <= 1.5e-5
    else:
        assert max(e_blocks) <= TOL[mode]
