"""ctypes binding of libtnc (include/tnc.h). Argument marshalling only.

Every contraction step runs in the library's CUDA kernels; this module only
converts Python/NumPy/PyTorch objects to the C ABI's plain pointers and sizes.
The library is loaded from this package directory (built in-tree by
``paper_2205_00393_gb300/build.py``); a missing library is an error.
"""

import ctypes
import json
import os

import numpy as np

FP32, SPLIT_TF32, SPLIT_BF16, SPLIT_BF16X2, SPLIT_FP16X2 = 0, 1, 2, 3, 4

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


class TNCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libtnc status %d: %s" % (status, msg))
        self.status = status


def lib_path():
    return os.path.join(_HERE, "libtnc.so")


def load_library():
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError("libtnc.so is not built (run __graft_entry__.build() or "
                          "python -m paper_2205_00393_gb300.build)")
    try:  # share the CUDA runtime already loaded by PyTorch, if any
        import torch  # noqa: F401
    except ImportError:
        pass
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    c_i64p = P(ctypes.c_int64)
    sigs = {
        "tnc_create_network": [ctypes.c_int, P(ctypes.c_int), P(c_i64p), ctypes.c_int64, c_i64p,
                               P(P(ctypes.c_float)), ctypes.c_int, c_i64p, P(ctypes.c_void_p)],
        "tnc_set_tensor_data": [ctypes.c_void_p, ctypes.c_int, P(ctypes.c_float)],
        "tnc_set_leaf_variants": [ctypes.c_void_p, ctypes.c_int, P(ctypes.c_int), ctypes.c_int64,
                                  P(P(ctypes.c_float))],
        "tnc_contract_variants": [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
        "tnc_leaf_bytes": [ctypes.c_void_p, P(ctypes.c_size_t)],
        "tnc_upload_leaves": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
        "tnc_greedy_path": [ctypes.c_void_p, P(ctypes.c_int)],
        "tnc_set_path": [ctypes.c_void_p, ctypes.c_int, P(ctypes.c_int)],
        "tnc_find_slices": [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double,
                            ctypes.c_double, ctypes.c_double, c_i64p, P(ctypes.c_int), ctypes.c_int],
        "tnc_set_slices": [ctypes.c_void_p, ctypes.c_int, c_i64p],
        "tnc_workspace_bytes": [ctypes.c_void_p, ctypes.c_int64, P(ctypes.c_size_t)],
        "tnc_set_workspace": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t],
        "tnc_contract": [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                         ctypes.c_void_p, ctypes.c_void_p],
        "tnc_stats": [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t],
        "tnc_arena_json": [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_char_p,
                           ctypes.c_size_t],
        "tnc_worklist_json": [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_char_p,
                              ctypes.c_size_t],
        "tnc_worklist_many_json": [ctypes.c_int, P(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_char_p, ctypes.c_size_t],
        "tnc_set_timing": [ctypes.c_void_p, ctypes.c_int],
        "tnc_check_device": [ctypes.c_void_p, ctypes.c_void_p],
        "tnc_autotune": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p],
        "tnc_tune_table": [ctypes.c_char_p, ctypes.c_size_t],
        "tnc_set_option": [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int64],
        "tnc_contract_backward": [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p],
        "tnc_contract_many": [ctypes.c_int, P(ctypes.c_void_p), c_i64p, c_i64p, ctypes.c_int,
                              P(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p],
        "tnc_param_grads": [ctypes.c_void_p, ctypes.c_int, P(ctypes.c_int), ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_void_p],
        "tnc_peak_probe": [ctypes.c_int, ctypes.c_int64, P(ctypes.c_double), ctypes.c_void_p],
        "tnc_last_timings": [ctypes.c_void_p, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int),
                             P(ctypes.c_double), P(ctypes.c_float), ctypes.c_int, P(ctypes.c_int), c_i64p],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.tnc_last_error.argtypes = []
    lib.tnc_last_error.restype = ctypes.c_char_p
    lib.tnc_destroy.argtypes = [ctypes.c_void_p]
    lib.tnc_destroy.restype = None
    _LIB = lib
    return lib


def _check(lib, st):
    if st != 0:
        raise TNCError(st, lib.tnc_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def tune_table():
    """The process-wide tuning table: list of [mode, log2 M, log2 N, log2 K, choice]."""
    lib = load_library()
    buf = ctypes.create_string_buffer(1 << 20)
    _check(lib, lib.tnc_tune_table(buf, 1 << 20))
    return json.loads(buf.value.decode())


def peak_probe(kind, iters, stream=None):
    """Launch one peak-rate probe kernel (tnc_peak_probe) on `stream`; returns
    the floating-point operations it performs (the caller times it)."""
    lib = load_library()
    flops = ctypes.c_double(0.0)
    _check(lib, lib.tnc_peak_probe(int(kind), int(iters), ctypes.byref(flops), _stream_ptr(stream)))
    return flops.value


def worklist_many(networks, batch, mode=FP32, deps=1):
    """The merged persistent work list of several networks, one batch each
    (tnc_worklist_many_json)."""
    lib = load_library()
    handles = (ctypes.c_void_p * len(networks))(*[n._h.value for n in networks])
    cap = 1 << 27
    buf = ctypes.create_string_buffer(cap)
    _check(lib, lib.tnc_worklist_many_json(len(networks), handles, int(batch), int(mode), int(deps), buf, cap))
    return json.loads(buf.value.decode())


def contract_many(networks, ranges=None, mode=FP32, outs=None, use_graph=True, stream=None):
    """Contract several networks together (tnc_contract_many): shared grouped
    launches across networks, replayed through a CUDA graph on repeat calls.
    Returns one complex128 CUDA tensor per network."""
    import torch
    lib = load_library()
    n = len(networks)
    if ranges is None:
        ranges = [(0, net.n_slices) for net in networks]
    if outs is None:
        outs = [torch.empty(net.n_out, dtype=torch.complex128, device="cuda") for net in networks]
    hs = (ctypes.c_void_p * n)(*[net._h.value for net in networks])
    lo = (ctypes.c_int64 * n)(*[int(r[0]) for r in ranges])
    hi = (ctypes.c_int64 * n)(*[int(r[1]) for r in ranges])
    op = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib, lib.tnc_contract_many(n, hs, lo, hi, int(mode), op, 1 if use_graph else 0, _stream_ptr(stream)))
    return outs


class Network:
    """A tensor network held by libtnc (Sec. 2.1.1: tensors = vertices,
    indices = edges). ``tensors`` are complex arrays (rounded to complex64),
    ``indices`` the index ids per tensor, ``dims`` the dimension per id and
    ``open_ids`` the order of the result tensor."""

    def __init__(self, tensors, indices, dims, open_ids):
        self._lib = load_library()
        self.n_tensors = len(tensors)
        self.dims = np.asarray(dims, dtype=np.int64)
        self.open_ids = tuple(int(e) for e in open_ids)
        self._keep = []
        ranks = (ctypes.c_int * self.n_tensors)(*[len(ix) for ix in indices])
        idx_arrays = [np.ascontiguousarray(np.asarray(ix, dtype=np.int64)) for ix in indices]
        data = [np.ascontiguousarray(np.asarray(t, dtype=np.complex64)) for t in tensors]
        I64P = ctypes.POINTER(ctypes.c_int64)
        FP = ctypes.POINTER(ctypes.c_float)
        idx_ptrs = (I64P * self.n_tensors)(*[a.ctypes.data_as(I64P) for a in idx_arrays])
        data_ptrs = (FP * self.n_tensors)(*[d.ctypes.data_as(FP) for d in data])
        op = np.asarray(self.open_ids, dtype=np.int64)
        h = ctypes.c_void_p()
        st = self._lib.tnc_create_network(self.n_tensors, ranks, idx_ptrs, len(self.dims),
                                          self.dims.ctypes.data_as(I64P), data_ptrs, len(op),
                                          op.ctypes.data_as(I64P) if len(op) else None,
                                          ctypes.byref(h))
        _check(self._lib, st)
        self._h = h
        self.n_out = int(np.prod([self.dims[e] for e in self.open_ids])) if self.open_ids else 1
        self.sliced = []
        self._ws = None
        self._sizes = [int(np.prod([self.dims[e] for e in ix])) if len(ix) else 1 for ix in indices]

    @classmethod
    def from_tn(cls, tn):
        return cls(tn.tensors, tn.indices, tn.dims, tn.open_ids)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.tnc_destroy(h)
            self._h = None

    def greedy_path(self):
        n = max(self.n_tensors - 1, 0)
        buf = (ctypes.c_int * max(2 * n, 1))()
        _check(self._lib, self._lib.tnc_greedy_path(self._h, buf))
        return [(buf[2 * i], buf[2 * i + 1]) for i in range(n)]

    def set_path(self, pairs):
        flat = np.asarray(pairs, dtype=np.int32).reshape(-1)
        arr = (ctypes.c_int * max(len(flat), 1))(*flat.tolist())
        _check(self._lib, self._lib.tnc_set_path(self._h, len(flat) // 2, arr))
        self.sliced = []

    def find_slices(self, target_log2, seed, T0=1.0, Tf=1e-4, alpha=0.9, cap=4096):
        out = (ctypes.c_int64 * cap)()
        n = ctypes.c_int()
        _check(self._lib, self._lib.tnc_find_slices(self._h, int(target_log2), int(seed) & (2**64 - 1),
                                                    T0, Tf, alpha, out, ctypes.byref(n), cap))
        return [int(out[i]) for i in range(n.value)]

    def set_slices(self, ids):
        ids = [int(e) for e in ids]
        arr = (ctypes.c_int64 * max(len(ids), 1))(*ids)
        _check(self._lib, self._lib.tnc_set_slices(self._h, len(ids), arr))
        self.sliced = ids

    @property
    def n_slices(self):
        """Addressable slices: 2^min(|S|, 62) (slice ids are int64)."""
        return 1 << min(len(self.sliced), 62)

    def set_tensor_data(self, i, data):
        d = np.ascontiguousarray(np.asarray(data, dtype=np.complex64))
        _check(self._lib, self._lib.tnc_set_tensor_data(self._h, int(i),
                                                         d.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def leaf_bytes(self):
        n = ctypes.c_size_t()
        _check(self._lib, self._lib.tnc_leaf_bytes(self._h, ctypes.byref(n)))
        return n.value

    def upload_leaves(self, packed_host_ptr, stream=None):
        _check(self._lib, self._lib.tnc_upload_leaves(self._h, ctypes.c_void_p(packed_host_ptr),
                                                       _stream_ptr(stream)))

    def workspace_bytes(self, batch=1):
        n = ctypes.c_size_t()
        _check(self._lib, self._lib.tnc_workspace_bytes(self._h, int(batch), ctypes.byref(n)))
        return n.value

    def set_workspace(self, tensor):
        """Hand a caller-owned (PyTorch) device buffer to the library as workspace."""
        if tensor is None:
            _check(self._lib, self._lib.tnc_set_workspace(self._h, None, 0))
        else:
            _check(self._lib, self._lib.tnc_set_workspace(self._h, ctypes.c_void_p(tensor.data_ptr()),
                                                           tensor.numel() * tensor.element_size()))
        self._ws = tensor

    def contract(self, lo=0, hi=None, mode=FP32, out=None, stream=None):
        """Sum over slices [lo, hi) of the sliced contraction, as a complex128
        CUDA tensor of 2^n_open elements in open_ids order."""
        import torch
        if hi is None:
            hi = self.n_slices
        if out is None:
            out = torch.empty(self.n_out, dtype=torch.complex128, device="cuda")
        st = self._lib.tnc_contract(self._h, int(lo), int(hi), int(mode), ctypes.c_void_p(out.data_ptr()),
                                    _stream_ptr(stream))
        _check(self._lib, st)
        return out

    def set_leaf_variants(self, leaf_ids, data):
        """Leaf variants (tnc_set_leaf_variants): data[i] is an array of shape
        (n_variants, *leaf_shape) for leaf leaf_ids[i]; [] removes them."""
        n = len(leaf_ids)
        if n == 0:
            _check(self._lib, self._lib.tnc_set_leaf_variants(self._h, 0, None, 0, None))
            return
        arrs = [np.ascontiguousarray(np.asarray(d, dtype=np.complex64)) for d in data]
        nv = arrs[0].shape[0]
        if any(a.shape[0] != nv for a in arrs):
            raise ValueError("every variant leaf needs the same number of copies")
        ids = (ctypes.c_int * n)(*[int(i) for i in leaf_ids])
        ptrs = (ctypes.POINTER(ctypes.c_float) * n)(*[a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) for a in arrs])
        _check(self._lib, self._lib.tnc_set_leaf_variants(self._h, n, ids, int(nv), ptrs))

    def contract_variants(self, v_lo, v_hi, lo=0, hi=None, mode=FP32, out=None, stream=None):
        """Variants [v_lo, v_hi), each summed over its slices [lo, hi): a
        complex128 CUDA tensor of shape (v_hi - v_lo, 2^n_open)."""
        import torch
        if hi is None:
            hi = self.n_slices
        if out is None:
            out = torch.empty((v_hi - v_lo, self.n_out), dtype=torch.complex128, device="cuda")
        st = self._lib.tnc_contract_variants(self._h, int(v_lo), int(v_hi), int(lo), int(hi), int(mode),
                                             ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream))
        _check(self._lib, st)
        return out

    def set_option(self, key, value):
        """Tensor-core tuning option (see tnc_set_option in include/tnc.h)."""
        _check(self._lib, self._lib.tnc_set_option(self._h, key.encode(), int(value)))

    def autotune(self, mode, slice=0, stream=None):
        """Time FP32 vs tensor-core kernels per contraction shape (tnc_autotune)."""
        _check(self._lib, self._lib.tnc_autotune(self._h, int(mode), int(slice), _stream_ptr(stream)))

    def check_device(self, stream=None):
        """Wait for the stream; raise TNCError if a device-side wait gave up."""
        _check(self._lib, self._lib.tnc_check_device(self._h, _stream_ptr(stream)))

    def set_timing(self, enable):
        _check(self._lib, self._lib.tnc_set_timing(self._h, 1 if enable else 0))

    def last_timings(self, cap=1 << 16):
        """Per-launch records since set_timing(True): list of dicts with node
        (-1 for a grouped launch), kind, batch, cmacs (complex multiply-
        accumulates) and ms; plus the number of kernels launched."""
        node = (ctypes.c_int * cap)()
        kind = (ctypes.c_int * cap)()
        batch = (ctypes.c_int * cap)()
        mnk = (ctypes.c_double * cap)()
        ms = (ctypes.c_float * cap)()
        n = ctypes.c_int()
        nl = ctypes.c_int64()
        _check(self._lib, self._lib.tnc_last_timings(self._h, node, kind, batch, mnk, ms, cap,
                                                      ctypes.byref(n), ctypes.byref(nl)))
        recs = [dict(node=node[i], kind=kind[i], batch=batch[i], cmacs=mnk[i], ms=ms[i])
                for i in range(n.value)]
        return recs, nl.value

    def contract_backward(self, grad_out, lo=0, hi=None, mode=FP32, leaf_mask=None, budget_bytes=0,
                          stream=None):
        """Holomorphic leaf environments dF/dL, F = sum_o grad_out[o] O[o], as a
        packed complex64 CUDA tensor (leaves back to back, leaf order)."""
        import torch
        if hi is None:
            hi = self.n_slices
        # materialise lazy conjugate / negative views: the C ABI reads raw memory
        g = grad_out.to(device="cuda", dtype=torch.complex128).resolve_conj().resolve_neg().contiguous()
        out = torch.empty(self.leaf_bytes() // 8, dtype=torch.complex64, device="cuda")
        mask = None
        if leaf_mask is not None:
            m = np.ascontiguousarray(np.asarray(leaf_mask, dtype=np.uint8))
            mask = m.ctypes.data_as(ctypes.c_void_p)
        st = self._lib.tnc_contract_backward(self._h, int(lo), int(hi), int(mode), ctypes.c_void_p(g.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()), mask, int(budget_bytes),
                                             _stream_ptr(stream))
        _check(self._lib, st)
        return out

    def param_grads(self, leaf_ids, dleaf_packed, env_packed, stream=None):
        """sum_e env[leaf][e] * dleaf[e] per parameter, FP64, as a complex128 CUDA tensor."""
        import torch
        ids = (ctypes.c_int * max(len(leaf_ids), 1))(*[int(x) for x in leaf_ids])
        out = torch.empty(len(leaf_ids), dtype=torch.complex128, device="cuda")
        d = dleaf_packed.to(device="cuda", dtype=torch.complex64).resolve_conj().resolve_neg().contiguous()
        env_packed = env_packed.resolve_conj().resolve_neg().contiguous()
        st = self._lib.tnc_param_grads(self._h, len(leaf_ids), ids, ctypes.c_void_p(d.data_ptr()),
                                       ctypes.c_void_p(env_packed.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                       _stream_ptr(stream))
        _check(self._lib, st)
        return out

    def leaf_slices(self):
        """(offset, size) in elements of every leaf in the packed layout."""
        out, off = [], 0
        for t in self._sizes:
            out.append((off, t))
            off += t
        return out

    def stats(self):
        cap = 1 << 22
        buf = ctypes.create_string_buffer(cap)
        _check(self._lib, self._lib.tnc_stats(self._h, buf, cap))
        return json.loads(buf.value.decode())

    def arena(self, batch, mode=FP32, reuse=1):
        """The workspace plan of one batch (tnc_arena_json)."""
        cap = 1 << 26
        buf = ctypes.create_string_buffer(cap)
        _check(self._lib, self._lib.tnc_arena_json(self._h, int(batch), int(mode), int(reuse), buf, cap))
        return json.loads(buf.value.decode())

    def worklist(self, batch, mode=FP32, deps=1):
        """The persistent executor's work list for one batch (tnc_worklist_json)."""
        cap = 1 << 26
        buf = ctypes.create_string_buffer(cap)
        _check(self._lib, self._lib.tnc_worklist_json(self._h, int(batch), int(mode), int(deps), buf, cap))
        return json.loads(buf.value.decode())
