"""Seeded random grid circuits of the paper's workload family.

The paper's workload (Sec. 6) is Google's Sycamore random quantum circuit; its
circuit files are not available, so circuits of the same gate family and 2D
nearest-neighbour structure are generated here:

* qubits sit on a rows x cols grid (minus optional removed sites), numbered in
  row-major order over the sites that exist;
* every cycle applies one single-qubit gate per qubit, drawn i.i.d. uniformly
  from {sqrt(X), sqrt(Y), sqrt(W)}, then fSim(theta, phi) on the couplers of
  pattern P[cycle mod 8] of the sequence A, B, C, D, C, D, A, B where
  A/B are horizontal pairs (r,c)-(r,c+1) with c even/odd and C/D vertical
  pairs (r,c)-(r+1,c) with r even/odd;
* theta ~ U[0, pi/2], phi ~ U[0, pi], one draw pair per fSim;
* there is no final single-qubit layer; all qubits start in |0>.

Random draws come from ``numpy.random.default_rng(seed)`` in a fixed order:
per cycle the single-qubit choices, then (theta, phi) per coupler in coupler
order; after the last cycle the bitstring. Open qubits are the last ``n_open``
qubits in row-major order.
"""

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

from . import gates as G

PATTERN_SEQUENCE = "ABCDCDAB"


@dataclass
class Gate:
    name: str
    qubits: Tuple[int, ...]
    matrix: np.ndarray
    params: Optional[Tuple[float, float]] = None  # (theta, phi) for fsim


@dataclass
class Circuit:
    n_qubits: int
    gates: List[Gate]
    bitstring: np.ndarray  # length n_qubits, values 0/1 (open qubits ignored)
    open_qubits: Tuple[int, ...] = ()
    sites: List[Tuple[int, int]] = field(default_factory=list)
    cycles: int = 0

    def fsim_gates(self):
        return [i for i, g in enumerate(self.gates) if g.name == "fsim"]


def coupler_layers(rows, cols, removed=()):
    """Return (sites, {pattern letter: [(qa, qb), ...]}) for a grid."""
    removed = set(removed)
    sites = [(r, c) for r in range(rows) for c in range(cols) if (r, c) not in removed]
    qid = {s: i for i, s in enumerate(sites)}
    layers = {k: [] for k in "ABCD"}
    for (r, c) in sites:
        if (r, c + 1) in qid:
            layers["A" if c % 2 == 0 else "B"].append((qid[(r, c)], qid[(r, c + 1)]))
        if (r + 1, c) in qid:
            layers["C" if r % 2 == 0 else "D"].append((qid[(r, c)], qid[(r + 1, c)]))
    return sites, layers


def grid_rqc(rows, cols, cycles, seed, n_open=0, removed=()):
    sites, layers = coupler_layers(rows, cols, removed)
    n = len(sites)
    if not 0 <= n_open <= n:
        raise ValueError("n_open out of range")
    rng = np.random.default_rng(seed)
    gates = []
    for cyc in range(cycles):
        choice = rng.integers(0, 3, size=n)
        for q in range(n):
            name = G.SINGLE_QUBIT_FAMILY[int(choice[q])]
            gates.append(Gate(name, (q,), G.single_qubit(name)))
        for (qa, qb) in layers[PATTERN_SEQUENCE[cyc % 8]]:
            theta = float(rng.uniform(0.0, np.pi / 2))
            phi = float(rng.uniform(0.0, np.pi))
            gates.append(Gate("fsim", (qa, qb), G.fsim(theta, phi), (theta, phi)))
    bits = rng.integers(0, 2, size=n).astype(np.int64)
    open_q = tuple(range(n - n_open, n))
    return Circuit(n, gates, bits, open_q, sites, cycles)


def lattice_53q_rqc(cycles, seed, n_open=0):
    """53-qubit 2D lattice: a 6x9 grid with site (0, 0) removed."""
    return grid_rqc(6, 9, cycles, seed, n_open=n_open, removed=((0, 0),))


def with_fsim_params(circuit, params):
    """Copy of ``circuit`` whose fSim gates take the (theta, phi) pairs in ``params``."""
    out = []
    k = 0
    for g in circuit.gates:
        if g.name == "fsim":
            th, ph = params[k]
            k += 1
            out.append(Gate("fsim", g.qubits, G.fsim(th, ph), (float(th), float(ph))))
        else:
            out.append(g)
    return Circuit(circuit.n_qubits, out, circuit.bitstring.copy(), circuit.open_qubits,
                   list(circuit.sites), circuit.cycles)


def batched_workload(n=256, seed0=1000):
    """The batched uneven workload: n seeded grid circuits with qubits
    U{20..36} (near-square grids, surplus sites removed from the last row),
    cycles U{10..16}, open qubits U{0..6} and a slicing depth k U{4..12}, drawn
    from default_rng(seed0) in that order per circuit; circuit i uses seed
    seed0 + i. Returns a list of (circuit, k)."""
    import math
    rng = np.random.default_rng(seed0)
    out = []
    for i in range(n):
        nq = int(rng.integers(20, 37))
        cyc = int(rng.integers(10, 17))
        n_open = int(rng.integers(0, 7))
        k = int(rng.integers(4, 13))
        r = int(math.floor(math.sqrt(nq)))
        c = int(math.ceil(nq / r))
        removed = [(r - 1, cc) for cc in range(c - (r * c - nq), c)]
        out.append((grid_rqc(r, c, cyc, seed0 + i, n_open=n_open, removed=removed), k))
    return out
