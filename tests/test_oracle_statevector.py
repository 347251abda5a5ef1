"""Pins for the gate matrices and the state-vector oracle.

Nothing here re-types the oracle's own formulas: gates are checked through
algebraic identities, the simulator through a Kronecker-product construction
of the full unitary and through closed-form states (GHZ, identity, Clifford).
"""


import numpy as np
import pytest

from tnc_inputs import gates as G
from tnc_inputs.circuits import Circuit, Gate, grid_rqc
from oracle import statevector


X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)


def test_sqrt_gates_square_to_paulis():
    W = (X + Y) / np.sqrt(2)
    for root, full in ((G.sqrt_x(), X), (G.sqrt_y(), Y), (G.sqrt_w(), W)):
        assert np.allclose(root @ root, full, atol=1e-15)
        assert np.allclose(root.conj().T @ root, np.eye(2), atol=1e-15)
        # principal root: eigenvalues 1 and i (arguments in [0, pi/2])
        ev = np.linalg.eigvals(root)
        assert np.allclose(sorted(np.angle(ev)), [0, np.pi / 2], atol=1e-12)


def test_sqrt_w_matches_exponential_form():
    # sqrt(W) = exp(-i pi/4 W) exp(i pi/4), computed here by eigendecomposition
    W = (X + Y) / np.sqrt(2)
    w, v = np.linalg.eigh(W)
    expo = v @ np.diag(np.exp(-1j * np.pi / 4 * w)) @ v.conj().T * np.exp(1j * np.pi / 4)
    assert np.allclose(expo, G.sqrt_w(), atol=1e-15)


@pytest.mark.parametrize("theta,phi", [(0.0, 0.0), (0.3, 1.1), (np.pi / 2, np.pi / 6), (1.0, 3.0)])
def test_fsim_unitary_and_special_cases(theta, phi):
    f = G.fsim(theta, phi)
    assert np.allclose(f.conj().T @ f, np.eye(4), atol=1e-15)
    if theta == 0 and phi == 0:
        assert np.allclose(f, np.eye(4))
    # fSim conserves the Hamming weight of the 2-qubit basis state
    for i in range(4):
        for j in range(4):
            if bin(i).count("1") != bin(j).count("1"):
                assert f[i, j] == 0
    # the (theta, phi) generator: fSim(t,p) = exp(-i t (XX+YY)/2) * diag(1,1,1,e^{-ip})
    XX_YY = (np.kron(X, X) + np.kron(Y, Y)) / 2
    w, v = np.linalg.eigh(XX_YY)
    rot = v @ np.diag(np.exp(-1j * theta * w)) @ v.conj().T
    assert np.allclose(rot @ np.diag([1, 1, 1, np.exp(-1j * phi)]), f, atol=1e-14)


def test_fsim_derivatives_match_fd():
    th, ph, h = 0.7, 1.9, 1e-6
    d_t = (G.fsim(th + h, ph) - G.fsim(th - h, ph)) / (2 * h)
    d_p = (G.fsim(th, ph + h) - G.fsim(th, ph - h)) / (2 * h)
    assert np.allclose(d_t, G.dfsim_dtheta(th, ph), atol=1e-9)
    assert np.allclose(d_p, G.dfsim_dphi(th, ph), atol=1e-9)


def _kron_unitary(n, gate):
    """Full 2^n x 2^n matrix of a gate by Kronecker products and a basis
    permutation (qubit 0 = most significant bit) -- independent of tensordot."""
    k = len(gate.qubits)
    dim = 1 << n
    U = np.zeros((dim, dim), dtype=complex)
    others = [q for q in range(n) if q not in gate.qubits]
    for col in range(dim):
        bits = [(col >> (n - 1 - q)) & 1 for q in range(n)]
        sub_in = 0
        for q in gate.qubits:
            sub_in = (sub_in << 1) | bits[q]
        for sub_out in range(1 << k):
            amp = gate.matrix[sub_out, sub_in]
            if amp == 0:
                continue
            nb = list(bits)
            for j, q in enumerate(gate.qubits):
                nb[q] = (sub_out >> (k - 1 - j)) & 1
            row = 0
            for b in nb:
                row = (row << 1) | b
            U[row, col] += amp
    return U


def test_statevector_matches_full_unitary_product():
    c = grid_rqc(2, 3, 4, seed=11)
    n = c.n_qubits
    state = np.zeros(1 << n, dtype=complex)
    state[0] = 1
    for g in c.gates:
        state = _kron_unitary(n, g) @ state
    psi = statevector.simulate(c).reshape(-1)
    assert np.allclose(psi, state, atol=1e-13)


def _ghz(n):
    gates = [Gate("h", (0,), G.hadamard())]
    for q in range(n - 1):
        gates.append(Gate("cnot", (q, q + 1), G.cnot()))
    return Circuit(n, gates, np.zeros(n, dtype=np.int64), tuple(range(n)))


@pytest.mark.parametrize("n", [2, 5, 9])
def test_ghz_closed_form(n):
    amps = statevector.amplitudes(_ghz(n))
    expect = np.zeros(1 << n, dtype=complex)
    expect[0] = expect[-1] = 1 / np.sqrt(2)
    assert np.allclose(amps, expect, atol=1e-15)


def test_identity_circuit():
    n = 6
    gates = []
    for q in range(n):
        gates.append(Gate("sqrt_x", (q,), G.sqrt_x()))
    for q in range(0, n - 1, 2):
        gates.append(Gate("fsim", (q, q + 1), G.fsim(0.0, 0.0), (0.0, 0.0)))
    for q in range(n):  # inverse of sqrt(X)
        gates.append(Gate("inv", (q,), G.sqrt_x().conj().T))
    c = Circuit(n, gates, np.zeros(n, dtype=np.int64), tuple(range(n)))
    amps = statevector.amplitudes(c)
    expect = np.zeros(1 << n, dtype=complex)
    expect[0] = 1
    assert np.allclose(amps, expect, atol=1e-15)


def test_clifford_support_and_weights():
    rng = np.random.default_rng(3)
    n = 7
    pool = [("h", G.hadamard()), ("s", G.s_gate()), ("sx", G.sqrt_x())]
    gates = []
    for layer in range(6):
        for q in range(n):
            name, m = pool[rng.integers(0, 3)]
            gates.append(Gate(name, (q,), m))
        for q in range(layer % 2, n - 1, 2):
            gates.append(Gate("cz", (q, q + 1), G.cz()))
    c = Circuit(n, gates, np.zeros(n, dtype=np.int64), tuple(range(n)))
    p = np.abs(statevector.amplitudes(c)) ** 2
    nz = p[p > 1e-12]
    k = int(round(np.log2(len(nz))))
    assert len(nz) == 1 << k
    assert np.allclose(nz, 2.0 ** -k, atol=1e-12)
    assert abs(p.sum() - 1) < 1e-12


def test_random_circuit_normalised():
    c = grid_rqc(3, 3, 6, seed=5, n_open=9)
    p = np.abs(statevector.amplitudes(c)) ** 2
    assert abs(p.sum() - 1) < 1e-12


def test_generator_is_seeded_and_shaped():
    a = grid_rqc(3, 4, 8, seed=1)
    b = grid_rqc(3, 4, 8, seed=1)
    assert [g.name for g in a.gates] == [g.name for g in b.gates]
    assert np.array_equal(a.bitstring, b.bitstring)
    n_fsim = sum(g.name == "fsim" for g in a.gates)
    # 3x4 grid: A=B=... per-pattern coupler counts, 8 cycles of ABCDCDAB
    from tnc_inputs.circuits import coupler_layers
    _, L = coupler_layers(3, 4)
    assert n_fsim == sum(len(L[p]) for p in "ABCDCDAB")
    assert sum(g.name != "fsim" for g in a.gates) == 12 * 8
    thetas = [g.params[0] for g in a.gates if g.name == "fsim"]
    phis = [g.params[1] for g in a.gates if g.name == "fsim"]
    assert min(thetas) >= 0 and max(thetas) <= np.pi / 2
    assert min(phis) >= 0 and max(phis) <= np.pi
