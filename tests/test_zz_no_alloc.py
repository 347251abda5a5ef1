"""The allocation-free entry point against the regular contraction and an
FP64 NumPy product of the same matrices.

tnc_reduce_pair_noalloc serves callers that may not allocate device memory
(their device memory belongs to another allocator, or a cudaMalloc would stall
a latency-critical path); it keeps its FP64 partial sums in a static device
array instead of a workspace. This file is collected last so that a failure
here never hides the other tests. It must pass alone in a fresh process (the
first call on the device looks up the array's address) and after the rest of
the suite.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5  # the FP32-path tolerance used by the other parity tests


def _pair(seed, m_log2, n_log2, k_log2):
    rng = np.random.default_rng(seed)
    M, N, K = 1 << m_log2, 1 << n_log2, 1 << k_log2
    a = ((rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))) / np.sqrt(K)).astype(np.complex64)
    b = (rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))).astype(np.complex64)
    assert a.dtype == b.dtype == np.complex64
    return a, b


@pytest.mark.parametrize("m_log2,n_log2,k_log2", [(2, 3, 16), (0, 0, 5), (3, 3, 20)])
def test_noalloc_matches_contract(libtnc, m_log2, n_log2, k_log2):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_00393_gb300 import Network
    a, b = _pair(1234 + k_log2, m_log2, n_log2, k_log2)
    M, N, K = a.shape[0], b.shape[1], a.shape[1]
    # the same contraction through tnc_contract: indices m (dim M), k (K), n (N)
    net = Network([a, b], [(0, 1), (1, 2)], [M, K, N], [0, 2])
    net.set_path([(0, 1)])
    ref = net.contract(0, 1).cpu().numpy()

    fn = libtnc.tnc_reduce_pair_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    da = torch.from_numpy(a.view(np.float32).reshape(-1).copy()).cuda()
    db = torch.from_numpy(b.view(np.float32).reshape(-1).copy()).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # an independent reference: the same product in FP64 by NumPy, no library kernel involved
    exact = (a.astype(np.complex128) @ b.astype(np.complex128)).reshape(-1)

    def err(got, want):
        rms = float(np.sqrt(np.mean(np.abs(want) ** 2)))
        return float(np.max(np.abs(got - want) / np.maximum(np.abs(want), 0.1 * rms)))
    assert err(ref, exact) <= TOL
    for call in range(2):  # two calls in a row share the static scratch
        out = torch.full((M * N,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        st = fn(ctypes.c_void_p(da.data_ptr()), ctypes.c_void_p(db.data_ptr()), m_log2, n_log2, k_log2,
                ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0, libtnc.tnc_last_error()
        got = out.cpu().numpy()
        assert err(got, ref) <= TOL, (call, err(got, ref))
        assert err(got, exact) <= TOL, (call, err(got, exact))


def test_noalloc_rejects_oversize(libtnc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fn = libtnc.tnc_reduce_pair_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert fn(p, p, 4, 3, 10, p, None) == 1  # 128 outputs > 64
    assert b"64" in libtnc.tnc_last_error()
    assert fn(p, p, 0, 0, 32, p, None) == 1  # K > 2^31
