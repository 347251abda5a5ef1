"""Brute-force state-vector simulation (oracle; test infrastructure only).

The state of n qubits is a complex128 array of shape (2,)*n, qubit 0 on axis
0 (most significant bit of a bitstring index). A gate U on qubits (q_a, ...)
maps psi to sum_in U[out, in] psi[..., in, ...]. This is the textbook
definition of applying a circuit; it is the ground truth for the tensor
networks built from the same circuits (an amplitude <x|C|0...0> equals the full
contraction of the circuit's network, Sec. 2.1.1).
"""

import numpy as np


def apply_gate(psi, matrix, qubits):
    k = len(qubits)
    u = np.asarray(matrix, dtype=np.complex128).reshape((2,) * (2 * k))
    # contract U's input axes (k..2k-1) with the state's qubit axes
    out = np.tensordot(u, psi, axes=(list(range(k, 2 * k)), list(qubits)))
    # tensordot puts U's output axes first; move them back to the qubit positions
    return np.moveaxis(out, list(range(k)), list(qubits))


def simulate(circuit, gate_override=None):
    """Final state of ``circuit`` from |0...0>.

    ``gate_override`` maps gate number -> replacement matrix (used for exact
    derivatives: the state is linear in every gate matrix).
    """
    n = circuit.n_qubits
    psi = np.zeros((2,) * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    for gi, g in enumerate(circuit.gates):
        m = g.matrix if gate_override is None or gi not in gate_override else gate_override[gi]
        psi = apply_gate(psi, m, g.qubits)
    return psi


def amplitudes(circuit, bitstring=None, gate_override=None):
    """Amplitudes <x|C|0>: closed qubits fixed to ``bitstring``, open qubits
    (``circuit.open_qubits``) left as a tensor in ascending qubit order.
    Returns a complex128 array of length 2**n_open (a 1-element array if none)."""
    psi = simulate(circuit, gate_override)
    bits = circuit.bitstring if bitstring is None else np.asarray(bitstring)
    open_set = set(circuit.open_qubits)
    sel = tuple(slice(None) if q in open_set else int(bits[q]) for q in range(circuit.n_qubits))
    return np.asarray(psi[sel], dtype=np.complex128).reshape(-1)
