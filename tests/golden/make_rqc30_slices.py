"""Write rqc30_slices_0_32.json: FP64 oracle sums of the 30-qubit workload.

Workload: the 5x6 grid random circuit (14 cycles, seed 2) with the last 6
qubits open (64 amplitudes), greedy contraction path, lifetime-based slicing
to 2^27-element intermediates (Algorithms 1 and 2, annealing seed 7). For
slices [0, 32) the script stores the oracle's complex128 sum over each block
of 4 consecutive slices (the batch one library call contracts) and the sum
over all 32. Every value comes from ``oracle`` (plain NumPy); the inputs come
from the seeded generators in ``tnc_inputs``.

Usage: python tests/golden/make_rqc30_slices.py   (about 15 CPU-minutes)
"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import planner, tn  # noqa: E402
from tnc_inputs import circuit_to_network, grid_rqc  # noqa: E402

BLOCK = 4
N_SLICES = 32


def main():
    c = grid_rqc(5, 6, 14, 2, n_open=6)
    net = circuit_to_network(c).as_complex64()
    path = planner.greedy_path(net.indices, net.dims)
    tree = planner.Tree(net.indices, net.dims, net.open_ids, path)
    S = planner.find_slices(tree, 27, 7)
    blocks = []
    t0 = time.time()
    for b in range(N_SLICES // BLOCK):
        acc = np.zeros(1 << len(net.open_ids), dtype=np.complex128)
        for s in range(b * BLOCK, (b + 1) * BLOCK):
            acc += tn.contract_slice(net, path, S, s)
        blocks.append(acc)
        print("block %d done (%.0f s)" % (b, time.time() - t0), flush=True)
    total = np.sum(blocks, axis=0)
    enc = lambda v: [[float(x.real), float(x.imag)] for x in v]  # noqa: E731
    rec = {
        "source": "FP64 oracle (oracle.tn.contract_slice) on the 30-qubit 5x6 grid circuit, 14 cycles, "
                  "seed 2, last 6 qubits open; greedy path (oracle.planner.greedy_path); slicing set of "
                  "Algorithms 1-2 (oracle.planner.find_slices, t = 27, seed 7); written by "
                  "tests/golden/make_rqc30_slices.py",
        "n_qubits": 30, "sliced": [int(e) for e in S], "path_len": len(path),
        "block": BLOCK, "slices": [0, N_SLICES],
        "block_sums": [enc(v) for v in blocks],
        "total": enc(total),
    }
    with open(os.path.join(HERE, "rqc30_slices_0_32.json"), "w") as f:
        json.dump(rec, f)
        f.write("\n")


if __name__ == "__main__":
    main()
