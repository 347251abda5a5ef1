"""Gate matrices of the random-circuit family (complex128).

Single-qubit gates act as ``new = U @ old`` on a 2-vector. Two-qubit gates are
4x4 in the basis |q_a q_b> with q_a the most significant bit.
"""

import numpy as np


def identity2():
    return np.eye(2, dtype=np.complex128)


def sqrt_x():
    """Principal square root of Pauli X: ((1+i) I + (1-i) X) / 2."""
    return 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128)


def sqrt_y():
    """Principal square root of Pauli Y: ((1+i) I + (1-i) Y) / 2."""
    return 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], dtype=np.complex128)


def sqrt_w():
    """Principal square root of W = (X + Y)/sqrt(2): ((1+i) I + (1-i) W) / 2.

    W squares to the identity, so its principal root has the same closed form
    as the roots of X and Y. Equals exp(-i pi/4 W) * exp(i pi/4).
    """
    r2 = np.sqrt(2.0)
    return 0.5 * np.array([[1 + 1j, -1j * r2], [r2, 1 + 1j]], dtype=np.complex128)


def fsim(theta, phi):
    """fSim(theta, phi): iSWAP-like rotation by theta plus a conditional phase phi."""
    c, s = np.cos(theta), np.sin(theta)
    return np.array(
        [
            [1, 0, 0, 0],
            [0, c, -1j * s, 0],
            [0, -1j * s, c, 0],
            [0, 0, 0, np.exp(-1j * phi)],
        ],
        dtype=np.complex128,
    )


def dfsim_dtheta(theta, phi):
    """Elementwise derivative of fsim with respect to theta."""
    c, s = np.cos(theta), np.sin(theta)
    return np.array(
        [[0, 0, 0, 0], [0, -s, -1j * c, 0], [0, -1j * c, -s, 0], [0, 0, 0, 0]],
        dtype=np.complex128,
    )


def dfsim_dphi(theta, phi):
    """Elementwise derivative of fsim with respect to phi."""
    out = np.zeros((4, 4), dtype=np.complex128)
    out[3, 3] = -1j * np.exp(-1j * phi)
    return out


def hadamard():
    return np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)


def s_gate():
    return np.array([[1, 0], [0, 1j]], dtype=np.complex128)


def cnot():
    """Control on the first (most significant) qubit."""
    m = np.eye(4, dtype=np.complex128)
    m[2:, 2:] = [[0, 1], [1, 0]]
    return m


def cz():
    return np.diag([1, 1, 1, -1]).astype(np.complex128)


SINGLE_QUBIT_FAMILY = ("sqrt_x", "sqrt_y", "sqrt_w")
_SQ = {"sqrt_x": sqrt_x, "sqrt_y": sqrt_y, "sqrt_w": sqrt_w}


def single_qubit(name):
    return _SQ[name]()
