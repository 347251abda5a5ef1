"""Pins for the gradient oracle: the exact (multilinear) derivative through
the state vector, through the tensor network, and central finite differences
in FP64 agree."""

import numpy as np

from tnc_inputs import circuit_to_network, grid_rqc
from oracle import gradient, planner


def test_exact_derivative_matches_central_fd():
    c = grid_rqc(2, 3, 4, seed=21, n_open=1)
    g = gradient.exact_statevector(c)
    params = gradient.circuit_params(c)
    which = [(k, j) for k in range(len(params)) for j in range(2)]
    fd = gradient.central_fd(gradient.statevector_amp_fn(c), params, which, 1e-6)
    got = np.array([g[k, j] for (k, j) in which])
    assert np.max(np.abs(got - fd)) < 1e-8


def test_network_derivative_matches_statevector():
    c = grid_rqc(2, 3, 4, seed=22)
    net = circuit_to_network(c)
    path = planner.greedy_path(net.indices, net.dims)
    tree = planner.Tree(net.indices, net.dims, net.open_ids, path)
    S = planner.find_slices(tree, max(tree.size_log(v) for v in range(tree.n_tensors)) - 1, 1)
    a = gradient.exact_network(c, net, path, S)
    b = gradient.exact_statevector(c)
    assert np.allclose(a, b, atol=1e-13)


def test_leaf_environments_euler_identity():
    """F is linear in every leaf, so sum_i L[i] dF/dL[i] = F for each leaf."""
    c = grid_rqc(2, 2, 3, seed=31, n_open=1)
    net = circuit_to_network(c)
    path = planner.greedy_path(net.indices, net.dims)
    seed = np.array([0.3 - 0.7j, 1.1 + 0.2j])
    F = np.dot(seed, tn_contract(net, path))
    envs = gradient.leaf_environments(net, path, (), seed)
    for L, E in zip(net.tensors, envs):
        assert abs(np.sum(np.asarray(L) * E) - F) < 1e-13


def test_leaf_environments_match_gate_derivatives():
    c = grid_rqc(2, 2, 3, seed=32)
    net = circuit_to_network(c)
    path = planner.greedy_path(net.indices, net.dims)
    envs = gradient.leaf_environments(net, path)
    exact = gradient.exact_statevector(c)
    from tnc_inputs import gates as G
    k = 0
    for li, g in enumerate(net.leaf_gate):
        if g >= 0 and c.gates[g].name == "fsim":
            th, ph = c.gates[g].params
            dth = np.sum(envs[li] * G.dfsim_dtheta(th, ph).reshape(2, 2, 2, 2))
            assert abs(dth - exact[k, 0, 0]) < 1e-13
            k += 1


def tn_contract(net, path):
    from oracle import tn
    return tn.contract(net, path)
