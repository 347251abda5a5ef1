"""Sliced tensor-network contraction along a contraction tree (oracle).

Test infrastructure only: product code must not import this module.

Definitions followed (Sec. 2.1.1):

* A pairwise contraction of tensors v0 and v1 removes the indices they share
  and keeps the rest; the new tensor carries v0's kept indices (in v0's order)
  followed by v1's kept indices (in v1's order).
* A contraction path in SSA form: leaves are 0..n-1 and step i contracts the
  two listed tensors into tensor n+i. The last step produces the result.
* Slicing (Sec. 2.1.1, Fig. 2): every sliced index e (w(e) = 2) is fixed to
  0 or 1, giving 2^|S| independent subtasks whose results are summed.
  Slice id s in [0, 2^|S|) assigns bit j of s to the j-th sliced index in
  ascending id order.

Each node is one ``numpy.tensordot`` in complex128 with the shared axes named
explicitly. Per node the multiply-add count M*N*K of the underlying matrix
product is logged (it equals the product of the dimensions of all indices the
node touches, the term of Eq. 1).
"""

import numpy as np


def _contract_pair(ta, ia, tb, ib):
    shared = [e for e in ia if e in ib]
    ax_a = [ia.index(e) for e in shared]
    ax_b = [ib.index(e) for e in shared]
    out = np.tensordot(ta, tb, axes=(ax_a, ax_b))
    keep_a = [e for e in ia if e not in shared]
    keep_b = [e for e in ib if e not in shared]
    m = int(np.prod([ta.shape[ia.index(e)] for e in keep_a], dtype=object)) if keep_a else 1
    n = int(np.prod([tb.shape[ib.index(e)] for e in keep_b], dtype=object)) if keep_b else 1
    k = int(np.prod([ta.shape[ia.index(e)] for e in shared], dtype=object)) if shared else 1
    return out, tuple(keep_a + keep_b), m * n * k


def slice_assignment(sliced_ids, s):
    """Slice id -> {index id: value}; bit j of s goes to the j-th smallest sliced id."""
    ids = sorted(int(e) for e in sliced_ids)
    return {e: (int(s) >> j) & 1 for j, e in enumerate(ids)}


def _fix_indices(tensor, idx, assign):
    sel = []
    kept = []
    for e in idx:
        if e in assign:
            sel.append(assign[e])
        else:
            sel.append(slice(None))
            kept.append(e)
    return np.asarray(tensor[tuple(sel)]), tuple(kept)


def contract_slice(network, path, sliced_ids=(), s=0, log=None):
    """Contract one slice of ``network`` along the SSA ``path``.

    Returns the result as a complex128 array in ``network.open_ids`` order,
    flattened (length 2**n_open; one element if there is no open index).
    ``log`` (a list), if given, receives the per-node multiply-add counts.
    """
    assign = slice_assignment(sliced_ids, s)
    live = {}
    for i, (t, idx) in enumerate(zip(network.tensors, network.indices)):
        live[i] = _fix_indices(np.asarray(t, dtype=np.complex128), tuple(idx), assign)
    nxt = network.n_tensors
    for (a, b) in path:
        ta, ia = live.pop(int(a))
        tb, ib = live.pop(int(b))
        out, io, mnk = _contract_pair(ta, ia, tb, ib)
        if log is not None:
            log.append(mnk)
        live[nxt] = (out, io)
        nxt += 1
    if len(live) != 1:
        raise ValueError("path does not contract the network to a single tensor")
    (t, idx), = live.values()
    order = [idx.index(e) for e in network.open_ids]
    if len(order) != len(idx):
        raise ValueError("result carries indices that are not open")
    return np.transpose(t, order).reshape(-1).astype(np.complex128)


def contract(network, path, sliced_ids=(), slices=None):
    """Sum of ``contract_slice`` over ``slices`` (default: all 2^|S| slices),
    accumulated in complex128 in ascending slice order."""
    if slices is None:
        slices = range(1 << len(sliced_ids))
    acc = None
    for s in slices:
        r = contract_slice(network, path, sliced_ids, s)
        acc = r if acc is None else acc + r
    if acc is None:
        acc = np.zeros(1 << len(network.open_ids), dtype=np.complex128)
    return acc


def contract_all_at_once(network):
    """Full contraction with no path structure: sequentially absorb leaves in
    leaf order into one running tensor (a different order than any planner
    path, used to check that the result does not depend on the path)."""
    t, idx = np.asarray(network.tensors[0], dtype=np.complex128), tuple(network.indices[0])
    for i in range(1, network.n_tensors):
        t, idx, _ = _contract_pair(t, idx, np.asarray(network.tensors[i], dtype=np.complex128),
                                   tuple(network.indices[i]))
    order = [idx.index(e) for e in network.open_ids]
    return np.transpose(t, order).reshape(-1)
