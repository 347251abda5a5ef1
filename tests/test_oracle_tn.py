"""Pins for the FP64 tensor-network contraction oracle.

* amplitudes equal brute-force state-vector amplitudes (Sec. 2.1.1: the
  amplitude is the full contraction of the circuit's network);
* the sum over all slices equals the unsliced contraction (Sec. 2.1.1);
* the result does not depend on the contraction path;
* normalisation with every qubit open;
* GHZ closed form through the network;
* the per-node multiply-add counts logged by the contraction equal the Eq. 1
  terms and their sum times 2^|S| equals Eq. 3.
"""

import numpy as np
import pytest

from tnc_inputs import circuit_to_network, grid_rqc
from tnc_inputs import gates as G
from tnc_inputs.circuits import Circuit, Gate
from oracle import planner, statevector, tn


def _setup(rows, cols, cycles, seed, n_open=0):
    c = grid_rqc(rows, cols, cycles, seed, n_open=n_open)
    net = circuit_to_network(c)
    path = planner.greedy_path(net.indices, net.dims)
    return c, net, path


def test_c1_amplitude_matches_statevector():
    c, net, path = _setup(3, 4, 8, 1)
    amp = tn.contract(net, path)
    ref = statevector.amplitudes(c)
    assert amp.shape == (1,)
    assert abs(amp[0] - ref[0]) <= 1e-12 * abs(ref[0])


@pytest.mark.parametrize("seed,n_open", [(2, 3), (4, 5)])
def test_open_outputs_match_statevector(seed, n_open):
    c, net, path = _setup(3, 3, 6, seed, n_open)
    amp = tn.contract(net, path)
    ref = statevector.amplitudes(c)
    assert np.allclose(amp, ref, rtol=0, atol=1e-13)


def test_all_open_normalised():
    c, net, path = _setup(2, 4, 5, 9, n_open=8)
    amp = tn.contract(net, path)
    assert abs(np.sum(np.abs(amp) ** 2) - 1) < 1e-12


def test_path_independence():
    c, net, path = _setup(2, 3, 5, 7, n_open=2)
    a = tn.contract(net, path)
    b = tn.contract_all_at_once(net)
    assert np.allclose(a, b, atol=1e-14)


def test_slices_sum_to_unsliced():
    c, net, path = _setup(3, 4, 8, 1)
    tree = planner.Tree(net.indices, net.dims, net.open_ids, path)
    rng = np.random.default_rng(0)
    closed = [e for e in tree.all_indices() if e not in tree.open]
    S = sorted(rng.choice(closed, size=5, replace=False).tolist())
    full = tn.contract(net, path)
    sl = tn.contract(net, path, S)
    assert abs(sl[0] - full[0]) <= 1e-12 * abs(full[0])
    # a slice differs from the total (slicing really splits the work)
    one = tn.contract_slice(net, path, S, 3)
    assert abs(one[0] - full[0]) > 1e-6 * abs(full[0])


def test_slice_bit_order():
    assign = tn.slice_assignment([40, 7, 19], 0b110)
    assert assign == {7: 0, 19: 1, 40: 1}


def test_ghz_through_network():
    n = 5
    gates = [Gate("h", (0,), G.hadamard())]
    for q in range(n - 1):
        gates.append(Gate("cnot", (q, q + 1), G.cnot()))
    c = Circuit(n, gates, np.zeros(n, dtype=np.int64), tuple(range(n)))
    net = circuit_to_network(c)
    path = planner.greedy_path(net.indices, net.dims)
    amp = tn.contract(net, path)
    expect = np.zeros(1 << n, dtype=complex)
    expect[0] = expect[-1] = 1 / np.sqrt(2)
    assert np.allclose(amp, expect, atol=1e-15)


def test_mac_log_matches_eq1_and_eq3():
    c, net, path = _setup(3, 4, 8, 1)
    tree = planner.Tree(net.indices, net.dims, net.open_ids, path)
    log = []
    tn.contract_slice(net, path, (), 0, log=log)
    assert log == [tree.node_cost(i) for i in range(len(path))]
    assert sum(log) == tree.eq1()
    S = planner.find_slices(tree, 8, seed=3)
    log = []
    tn.contract_slice(net, path, S, 0, log=log)
    assert sum(log) * (1 << len(S)) == tree.eq3(S)


def test_complex64_input_rounding_is_small():
    c, net, path = _setup(3, 4, 8, 1)
    a = tn.contract(net, path)[0]
    b = tn.contract(net.as_complex64(), path)[0]
    assert abs(a - b) < 1e-6 * abs(a)
