"""Differentiable circuit amplitudes: a torch.autograd.Function around
tnc_contract / tnc_contract_backward / tnc_param_grads.

The forward contracts the circuit's network in libtnc; the backward runs the
library's adjoint pass (leaf environments) and its chain-rule kernel. Gate
matrices for given (theta, phi) and their elementwise derivatives are inputs
prepared on the host; every contraction runs in the library.

Convention: PyTorch passes grad = dL/dRe(amp) + i dL/dIm(amp) for a complex
output; with F = sum_o conj(grad_o) amp_o the library returns dF/dleaf and
dL/dtheta = Re(dF/dtheta).
"""

import numpy as np
import torch

from ._lib import FP32, Network


def _fsim(theta, phi):
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[1, 0, 0, 0], [0, c, -1j * s, 0], [0, -1j * s, c, 0], [0, 0, 0, np.exp(-1j * phi)]])


def _dfsim(theta, phi):
    c, s = np.cos(theta), np.sin(theta)
    dt = np.array([[0, 0, 0, 0], [0, -s, -1j * c, 0], [0, -1j * c, -s, 0], [0, 0, 0, 0]])
    dp = np.zeros((4, 4), dtype=complex)
    dp[3, 3] = -1j * np.exp(-1j * phi)
    return dt, dp


class CircuitAmplitudes:
    """Amplitudes of a circuit network as a function of its fSim (theta, phi).

    network: a tensor network (leaf tensors, index lists, dims, open ids)
    whose leaves listed in ``fsim_leaves`` are fSim gates T[o_a, o_b, i_a, i_b]
    = fSim(theta, phi)[(o_a o_b), (i_a i_b)], in parameter order."""

    def __init__(self, network, fsim_leaves, path=None, target_log2=None, seed=7, lo=0, hi=None, mode=FP32,
                 budget_bytes=0):
        self.net = Network.from_tn(network)
        self.net.set_path(path if path is not None else self.net.greedy_path())
        if target_log2 is not None:
            self.net.set_slices(self.net.find_slices(target_log2, seed))
        self.fsim_leaves = list(fsim_leaves)
        self.lo = lo
        self.hi = self.net.n_slices if hi is None else hi
        self.mode = mode
        self.budget = budget_bytes
        self.mask = np.zeros(self.net.n_tensors, dtype=np.uint8)
        self.mask[self.fsim_leaves] = 1

    def set_params(self, params):
        p = np.asarray(params, dtype=np.float64).reshape(-1, 2)
        for leaf, (th, ph) in zip(self.fsim_leaves, p):
            self.net.set_tensor_data(leaf, _fsim(th, ph).reshape(2, 2, 2, 2))

    def __call__(self, params):
        return _AmplitudeFn.apply(params, self)


class _AmplitudeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, obj):
        obj.set_params(params.detach().cpu().numpy())
        out = obj.net.contract(obj.lo, obj.hi, obj.mode)
        ctx.obj = obj
        ctx.save_for_backward(params)
        return out

    @staticmethod
    def backward(ctx, grad):
        obj = ctx.obj
        (params,) = ctx.saved_tensors
        p = params.detach().cpu().numpy().reshape(-1, 2)
        env = obj.net.contract_backward(torch.conj(grad), obj.lo, obj.hi, obj.mode, leaf_mask=obj.mask,
                                        budget_bytes=obj.budget)
        ids, d = [], []
        for leaf, (th, ph) in zip(obj.fsim_leaves, p):
            dt, dp = _dfsim(th, ph)
            ids += [leaf, leaf]
            d += [dt.reshape(-1), dp.reshape(-1)]
        dleaf = torch.from_numpy(np.concatenate(d).astype(np.complex64))
        g = obj.net.param_grads(ids, dleaf, env)
        out = g.real.reshape(params.shape).to(params.device, params.dtype)
        return out, None
