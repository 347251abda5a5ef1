"""Write rqc30_bitstrings.json: FP64 oracle amplitudes of a batch of closed
bitstrings of the 30-qubit workload (correlated samples, Sec. 1 and 6.2).

Workload: the 5x6 grid random circuit (14 cycles, seed 2) with the last 6
qubits open (64 amplitudes per bitstring), greedy contraction path,
lifetime-based slicing to 2^27-element intermediates (Algorithms 1 and 2,
annealing seed 7). Four bitstrings over the 24 closed qubits are drawn by
tnc_inputs.random_bitstrings (seed 11); for each, the network with that
bitstring's projection vectors is contracted by the oracle over slices
[0, 2) and the sum stored. Every value comes from ``oracle`` (plain NumPy);
the inputs come from the seeded generators in ``tnc_inputs``.

Usage: python tests/golden/make_rqc30_bitstrings.py   (about 4 CPU-minutes)
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
from tnc_inputs import circuit_to_network, grid_rqc, random_bitstrings  # noqa: E402

N_BITSTRINGS = 4
SLICES = (0, 2)
SEED = 11


def main():
    c = grid_rqc(5, 6, 14, 2, n_open=6)
    net = circuit_to_network(c).as_complex64()
    path = planner.greedy_path(net.indices, net.dims)
    tree = planner.Tree(net.indices, net.dims, net.open_ids, path)
    S = planner.find_slices(tree, 27, 7)
    bits = random_bitstrings(c, N_BITSTRINGS, SEED)
    amps = []
    t0 = time.time()
    for b in bits:
        nb = circuit_to_network(c, bitstring=b).as_complex64()
        acc = np.zeros(1 << len(nb.open_ids), dtype=np.complex128)
        for s in range(*SLICES):
            acc += tn.contract_slice(nb, path, S, s)
        amps.append(acc)
        print("bitstring done (%.0f s)" % (time.time() - t0), flush=True)
    enc = lambda v: [[float(x.real), float(x.imag)] for x in v]  # noqa: E731
    rec = {
        "source": "FP64 oracle (oracle.tn.contract_slice) on the 30-qubit 5x6 grid circuit, 14 cycles, "
                  "seed 2, last 6 qubits open, with the closed qubits projected on each bitstring; greedy "
                  "path (oracle.planner.greedy_path); slicing set of Algorithms 1-2 "
                  "(oracle.planner.find_slices, t = 27, seed 7); written by "
                  "tests/golden/make_rqc30_bitstrings.py",
        "n_qubits": 30, "sliced": [int(e) for e in S], "slices": list(SLICES),
        "bitstring_seed": SEED, "bitstrings": [[int(x) for x in b] for b in bits],
        "amplitudes": [enc(a) for a in amps],
    }
    with open(os.path.join(HERE, "rqc30_bitstrings.json"), "w") as f:
        json.dump(rec, f)


if __name__ == "__main__":
    main()
