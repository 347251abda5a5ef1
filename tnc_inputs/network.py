"""Circuit -> tensor network (Sec. 2.1.1: tensors are vertices, indices are edges).

Every wire segment between two gates is one index of dimension 2. Leaves, in
order: the |0> vector of every qubit (qubit order), every gate in circuit
order, then the <x_q| projection vector of every closed qubit (qubit order).
A 1-qubit gate U is the rank-2 tensor T[out, in] = U[out, in]; a 2-qubit gate
on (a, b) is T[out_a, out_b, in_a, in_b] = U.reshape(2, 2, 2, 2). The final
wire index of each open qubit is an open index; the result tensor is ordered
by open qubit, ascending. Every index joins at most two tensors.
"""

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np


@dataclass
class TensorNetwork:
    tensors: List[np.ndarray]          # complex128, shape (dims of its indices)
    indices: List[Tuple[int, ...]]     # index ids per tensor, row-major order
    dims: np.ndarray                   # int64 dimension per index id
    open_ids: Tuple[int, ...]          # order of the result tensor
    leaf_gate: List[int]               # gate number per leaf (-1: boundary vector)

    @property
    def n_tensors(self):
        return len(self.tensors)

    @property
    def n_indices(self):
        return int(len(self.dims))

    def as_complex64(self):
        """Same network with every leaf rounded to complex64 (the library's input type)."""
        return TensorNetwork([t.astype(np.complex64) for t in self.tensors],
                             list(self.indices), self.dims.copy(), self.open_ids,
                             list(self.leaf_gate))

    def with_tensors(self, tensors):
        return TensorNetwork(list(tensors), list(self.indices), self.dims.copy(),
                             self.open_ids, list(self.leaf_gate))


def circuit_to_network(circuit, bitstring=None):
    n = circuit.n_qubits
    bits = circuit.bitstring if bitstring is None else np.asarray(bitstring)
    open_set = set(circuit.open_qubits)
    next_id = 0
    wire = []
    tensors, indices, leaf_gate = [], [], []
    for q in range(n):
        wire.append(next_id)
        tensors.append(np.array([1.0, 0.0], dtype=np.complex128))
        indices.append((next_id,))
        leaf_gate.append(-1)
        next_id += 1
    for gi, g in enumerate(circuit.gates):
        k = len(g.qubits)
        ins = [wire[q] for q in g.qubits]
        outs = list(range(next_id, next_id + k))
        next_id += k
        for q, o in zip(g.qubits, outs):
            wire[q] = o
        tensors.append(np.asarray(g.matrix, dtype=np.complex128).reshape((2,) * (2 * k)).copy())
        indices.append(tuple(outs + ins))
        leaf_gate.append(gi)
    for q in range(n):
        if q in open_set:
            continue
        v = np.zeros(2, dtype=np.complex128)
        v[int(bits[q])] = 1.0
        tensors.append(v)
        indices.append((wire[q],))
        leaf_gate.append(-1)
    open_ids = tuple(wire[q] for q in sorted(open_set))
    dims = np.full(next_id, 2, dtype=np.int64)
    return TensorNetwork(tensors, indices, dims, open_ids, leaf_gate)


def projection_leaves(circuit):
    """Leaf ids of the <x_q| projection vectors of ``circuit_to_network(circuit)``
    and their qubits, in qubit order (closed qubits only)."""
    open_set = set(circuit.open_qubits)
    first = circuit.n_qubits + len(circuit.gates)
    closed = [q for q in range(circuit.n_qubits) if q not in open_set]
    return [first + j for j in range(len(closed))], closed


def random_bitstrings(circuit, n, seed):
    """n seeded bitstrings (uint8, shape (n, n_qubits)) over the circuit's
    qubits; open qubits are 0 (they are summed over as outputs, not fixed)."""
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2, size=(n, circuit.n_qubits)).astype(np.uint8)
    bits[:, list(circuit.open_qubits)] = 0
    return bits


def bitstring_variants(circuit, bitstrings):
    """Variant data for the projection leaves: for each closed qubit q, an
    array of shape (n, 2) whose row v is the one-hot vector <b_v[q]|. Returns
    (leaf ids, list of arrays), the arguments of Network.set_leaf_variants."""
    leaves, closed = projection_leaves(circuit)
    bits = np.asarray(bitstrings, dtype=np.int64)
    data = []
    for q in closed:
        a = np.zeros((bits.shape[0], 2), dtype=np.complex64)
        a[np.arange(bits.shape[0]), bits[:, q]] = 1.0
        data.append(a)
    return leaves, data
