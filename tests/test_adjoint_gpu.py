"""GPU parity of the adjoint pass (tnc_contract_backward, tnc_param_grads)
and of the torch.autograd wrapper.

Witnesses: the oracle's leaf environments (dF/dL[i] = F with L replaced by a
unit tensor, FP64), exact state-vector derivatives of amplitudes with respect
to fSim (theta, phi), and central finite differences (h = 1e-3) of the GPU
forward. Tolerance: gradients within 1e-4 relative (floored at the rms of
the checked set) of the FP64 witnesses, and within 1e-3 of finite
differences.
"""

import numpy as np
import pytest

from tnc_inputs import circuit_to_network, grid_rqc
from tnc_inputs import gates as G
from oracle import gradient, planner

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(libtnc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return libtnc


def _rel(a, b):
    a, b = np.asarray(a).reshape(-1), np.asarray(b).reshape(-1)
    rms = float(np.sqrt(np.mean(np.abs(b) ** 2)))
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), rms)))


def _unpack(net, packed):
    p = packed.cpu().numpy()
    return [p[o:o + n] for (o, n) in net.leaf_slices()]


@pytest.mark.parametrize("mode", [0, 2])
def test_leaf_environments_vs_oracle(lib, mode):
    from paper_2205_00393_gb300 import Network
    c = grid_rqc(2, 2, 4, seed=41, n_open=2)
    tn_ = circuit_to_network(c).as_complex64()
    net = Network.from_tn(tn_)
    path = net.greedy_path()
    net.set_path(path)
    tree = planner.Tree(tn_.indices, tn_.dims, tn_.open_ids, path)
    W = max(tree.size_log(v) for v in range(tree.n_tensors))
    S = net.find_slices(W - 1, 3)
    net.set_slices(S)
    assert net.n_slices >= 4
    rng = np.random.default_rng(5)
    seed = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    env = net.contract_backward(torch.from_numpy(seed), 0, net.n_slices, mode)
    net.check_device()
    got = _unpack(net, env)
    ref = gradient.leaf_environments(tn_, path, S, seed)
    for g, r in zip(got, ref):
        assert _rel(g, r.reshape(-1)) <= 1e-4


def test_partial_slice_range_environments(lib):
    from paper_2205_00393_gb300 import Network
    c = grid_rqc(2, 2, 3, seed=41, n_open=1)
    tn_ = circuit_to_network(c).as_complex64()
    net = Network.from_tn(tn_)
    path = net.greedy_path()
    net.set_path(path)
    tree = planner.Tree(tn_.indices, tn_.dims, tn_.open_ids, path)
    W = max(tree.size_log(v) for v in range(tree.n_tensors))
    S = net.find_slices(W - 1, 3)
    net.set_slices(S)
    lo, hi = 1, max(2, net.n_slices - 1)
    env = net.contract_backward(torch.tensor([1.0, -0.5j], dtype=torch.complex128), lo, hi, 0)
    got = _unpack(net, env)
    ref = gradient.leaf_environments(tn_, path, S, np.array([1.0, -0.5j]), slices=range(lo, hi))
    for g, r in zip(got, ref):
        assert _rel(g, r.reshape(-1)) <= 1e-4


def _c1_amplitudes(mode=0):
    from paper_2205_00393_gb300.torch_fn import CircuitAmplitudes
    c = grid_rqc(3, 4, 8, 1)
    tn_ = circuit_to_network(c)
    fsim_leaves = [li for li, g in enumerate(tn_.leaf_gate) if g >= 0 and c.gates[g].name == "fsim"]
    amp = CircuitAmplitudes(tn_, fsim_leaves, target_log2=8, seed=7, mode=mode)
    params = torch.tensor(gradient.circuit_params(c), dtype=torch.float64, requires_grad=True)
    return c, amp, params


@pytest.mark.parametrize("mode", [0, 2])
def test_param_gradients_vs_statevector(lib, mode):
    c, amp, params = _c1_amplitudes(mode)
    assert amp.net.n_slices == 16
    a = amp(params)
    # L = Re(conj(w) amp) has dL/dtheta = Re(conj(w) d amp/dtheta)
    w = complex(0.6, -0.8)
    L = (torch.conj(torch.tensor(w, dtype=torch.complex128, device="cuda")) * a).real.sum()
    L.backward()
    got = params.grad.numpy()
    ex = gradient.exact_statevector(c)[:, :, 0]  # d amp / d(theta, phi)
    ref = (np.conj(w) * ex).real
    assert _rel(got, ref) <= 1e-4


def test_autograd_vs_finite_differences(lib):
    c, amp, params = _c1_amplitudes(0)
    a = amp(params)
    (a.abs() ** 2).sum().backward()
    g = params.grad.numpy()
    rng = np.random.default_rng(6)
    which = [(int(k), int(j)) for k, j in zip(rng.integers(0, params.shape[0], 16), rng.integers(0, 2, 16))]
    h = 1e-3
    fd = []
    p0 = params.detach().numpy().copy()
    for (k, j) in which:
        vals = []
        for sgn in (+1, -1):
            p = p0.copy()
            p[k, j] += sgn * h
            with torch.no_grad():
                vals.append(float((amp(torch.from_numpy(p)).abs() ** 2).sum()))
        fd.append((vals[0] - vals[1]) / (2 * h))
    fd = np.array(fd)
    got = np.array([g[k, j] for (k, j) in which])
    rms = float(np.sqrt(np.mean(fd ** 2)))
    assert np.max(np.abs(got - fd) / np.maximum(np.abs(fd), rms)) <= 1e-3


def test_backward_budget_too_small(lib):
    from paper_2205_00393_gb300 import TNCError
    c, amp, params = _c1_amplitudes(0)
    with pytest.raises(TNCError) as e:
        amp.net.contract_backward(torch.ones(1, dtype=torch.complex128), 0, 16, 0, budget_bytes=1024)
    assert e.value.status == 2


@pytest.mark.parametrize("mode", [2, 1, 4])
def test_tensor_core_environments(lib, mode):
    """Environment contractions large enough for the tensor cores: split
    precision must agree with the FP32 environments, and F is linear in every
    leaf, so sum_i L[i] dF/dL[i] = F (the forward result) for each leaf."""
    from paper_2205_00393_gb300 import Network
    from .test_parity_tc_gpu import _three_leaf
    net_ref = _three_leaf(11, 8, 8, 7, True)
    net = Network.from_tn(net_ref)
    net.set_path([(0, 1), (2, 3)])
    n_out = net.n_out
    rng = np.random.default_rng(3)
    seed = torch.from_numpy(rng.standard_normal(n_out) + 1j * rng.standard_normal(n_out))
    F = complex(np.dot(seed.numpy(), net.contract(0, 1, 0).cpu().numpy()))
    e32 = _unpack(net, net.contract_backward(seed, 0, 1, 0))
    etc = _unpack(net, net.contract_backward(seed, 0, 1, mode))
    net.check_device()
    for (a, b, L) in zip(etc, e32, net_ref.tensors):
        assert _rel(a, b) <= 1e-4
        assert abs(np.sum(np.asarray(L).reshape(-1).astype(np.complex128) * a) - F) <= 1e-4 * abs(F)


def test_checkpointing_recompute(lib):
    """30-qubit workload, one slice: keeping only every 4th level of
    per-slice intermediates (recomputing the rest in the reverse walk) gives
    bit-identical environments; a budget below the smallest possible
    workspace is refused. (On this tree the peak is the working set of the
    largest node, so spacing the checkpoints does not lower it.)"""
    from paper_2205_00393_gb300 import Network, TNCError
    c = grid_rqc(5, 6, 14, 2, n_open=6)
    tn_ = circuit_to_network(c).as_complex64()
    net = Network.from_tn(tn_)
    net.set_path(net.greedy_path())
    net.set_slices(net.find_slices(27, 7))
    mask = np.array([1 if g >= 0 and c.gates[g].name == "fsim" else 0 for g in tn_.leaf_gate], dtype=np.uint8)
    seed = torch.ones(net.n_out, dtype=torch.complex128)
    full = net.contract_backward(seed, 3, 4, 2, leaf_mask=mask).cpu().numpy()
    st = net.stats()
    assert st["backward_keep_every"] == 1
    need = st["backward_workspace"]
    net.set_option("backward_keep_every", 4)
    ck = net.contract_backward(seed, 3, 4, 2, leaf_mask=mask).cpu().numpy()
    net.check_device()
    st2 = net.stats()
    assert st2["backward_keep_every"] == 4
    assert np.array_equal(full, ck)
    assert st2["backward_workspace"] > 0 and need > 0
    net.set_option("backward_keep_every", 0)
    with pytest.raises(TNCError) as e:
        net.contract_backward(seed, 3, 4, 2, leaf_mask=mask, budget_bytes=1 << 20)
    assert e.value.status == 2


@pytest.mark.parametrize("mode", [0, 2])
def test_30q_gradients_vs_gate_perturbation(lib, mode):
    """30-qubit 5x6 grid (14 cycles), one amplitude, one slice of the t = 27
    slicing: the amplitude is linear in every gate matrix G, so
    (F(G + dG) - F(G - dG)) / 2 is the exact derivative along dG = dG/dtheta
    (or dG/dphi) up to the forward's rounding. The adjoint gradient of
    Re(F) on 16 seeded parameters matches it within 1e-4 (floored at the rms
    of the checked set)."""
    from paper_2205_00393_gb300.torch_fn import CircuitAmplitudes
    c = grid_rqc(5, 6, 14, 2)
    tn_ = circuit_to_network(c)
    fsim = [li for li, g in enumerate(tn_.leaf_gate) if g >= 0 and c.gates[g].name == "fsim"]
    amp = CircuitAmplitudes(tn_, fsim, target_log2=27, seed=7, lo=3, hi=4, mode=mode)
    p0 = gradient.circuit_params(c)
    params = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    amp(params).real.sum().backward()
    amp.net.check_device()
    g = params.grad.numpy()
    rng = np.random.default_rng(6)
    which = [(int(f) // 2, int(f) % 2) for f in rng.choice(p0.size, 16, replace=False)]
    lin = []
    for (k, j) in which:
        th, ph = p0[k]
        dG = G.dfsim_dtheta(th, ph) if j == 0 else G.dfsim_dphi(th, ph)
        vals = []
        for sgn in (1, -1):
            amp.net.set_tensor_data(fsim[k], (G.fsim(th, ph) + sgn * dG).reshape(2, 2, 2, 2))
            vals.append(complex(amp.net.contract(3, 4, mode).sum()))
        amp.net.set_tensor_data(fsim[k], G.fsim(th, ph).reshape(2, 2, 2, 2))
        lin.append(((vals[0] - vals[1]) / 2).real)
    got = np.array([g[k, j] for (k, j) in which])
    err = _rel(got, np.array(lin))
    print("30q mode %d adjoint vs gate perturbation %.3e" % (mode, err))
    assert err <= 1e-4
