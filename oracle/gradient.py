"""Derivatives of amplitudes with respect to fSim parameters (oracle).

Test infrastructure only. An amplitude <x|G_L ... G_1|0> is linear in every
gate matrix, so d amp / d theta_g is the same amplitude with gate g replaced by
its elementwise derivative dG_g/dtheta (likewise for phi). Two witnesses:

* ``exact_statevector``: that replacement in the state-vector simulator;
* ``exact_network``: that replacement in the network's leaf tensor, contracted
  with the FP64 tensor-network oracle along a given path and slicing set;

and ``central_fd`` (central finite differences of any amplitude function).
"""

import numpy as np

from tnc_inputs import gates as G
from tnc_inputs.circuits import with_fsim_params

from . import statevector, tn


def _fsim_derivs(circuit):
    out = []
    for gi, g in enumerate(circuit.gates):
        if g.name == "fsim":
            th, ph = g.params
            out.append((gi, G.dfsim_dtheta(th, ph), G.dfsim_dphi(th, ph)))
    return out


def exact_statevector(circuit):
    """Array [n_fsim, 2, n_amp]: d amp / d(theta, phi) for every fSim gate."""
    res = []
    for gi, dth, dph in _fsim_derivs(circuit):
        a = statevector.amplitudes(circuit, gate_override={gi: dth})
        b = statevector.amplitudes(circuit, gate_override={gi: dph})
        res.append(np.stack([a, b]))
    return np.array(res)


def exact_network(circuit, network, path, sliced_ids=()):
    """Same as ``exact_statevector`` through the tensor-network oracle."""
    leaf_of_gate = {g: i for i, g in enumerate(network.leaf_gate) if g >= 0}
    res = []
    for gi, dth, dph in _fsim_derivs(circuit):
        li = leaf_of_gate[gi]
        pair = []
        for d in (dth, dph):
            ts = list(network.tensors)
            ts[li] = d.reshape((2,) * 4)
            pair.append(tn.contract(network.with_tensors(ts), path, sliced_ids))
        res.append(np.stack(pair))
    return np.array(res)


def central_fd(amp_fn, params, which, h):
    """Central differences of ``amp_fn(params)`` w.r.t. params[k][j] for (k, j) in ``which``."""
    out = []
    for (k, j) in which:
        p = np.array(params, dtype=np.float64)
        p[k, j] += h
        fp = amp_fn(p)
        p[k, j] -= 2 * h
        fm = amp_fn(p)
        out.append((fp - fm) / (2 * h))
    return np.array(out)


def circuit_params(circuit):
    return np.array([g.params for g in circuit.gates if g.name == "fsim"], dtype=np.float64)


def statevector_amp_fn(circuit):
    def f(params):
        return statevector.amplitudes(with_fsim_params(circuit, params))
    return f


def leaf_environments(network, path, sliced_ids=(), seed=None, slices=None):
    """Holomorphic environments dF/dL of every leaf L, F = sum_o seed_o O_o
    with O the (sliced) contraction. F is linear in every leaf, so
    dF/dL[i] = F evaluated with L replaced by the unit tensor e_i.
    Returns a list of complex128 arrays shaped like the leaves."""
    n_out = int(np.prod([network.dims[e] for e in network.open_ids])) if network.open_ids else 1
    seed = np.ones(n_out, dtype=np.complex128) if seed is None else np.asarray(seed, dtype=np.complex128)
    envs = []
    for li, t in enumerate(network.tensors):
        t = np.asarray(t)
        env = np.zeros(t.size, dtype=np.complex128)
        for i in range(t.size):
            unit = np.zeros(t.size, dtype=np.complex128)
            unit[i] = 1.0
            ts = list(network.tensors)
            ts[li] = unit.reshape(t.shape)
            out = tn.contract(network.with_tensors(ts), path, sliced_ids, slices)
            env[i] = np.dot(seed, out)
        envs.append(env.reshape(t.shape))
    return envs
