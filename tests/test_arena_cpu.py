"""The workspace plan (tnc_arena_json), checked on the host without a GPU
against the contraction tree: the first-fit simulation that places every
stored intermediate, split-plane pair and final-contraction scratch of a
batch. For every network, mode, batch and reuse setting checked:

* no two live allocations share a byte, and the peak is the highest end;
* every release matches a live allocation; without reuse nothing is
  released;
* a stored intermediate is allocated at a later level than each stored
  child, and a child is released exactly at its parent's level, after the
  parent's output is placed, or, if slice-invariant and read by per-slice
  contractions, or read by the final contraction, never;
* split planes live only during their contraction's level.

A plan that let a live tensor's bytes be reused would corrupt results on the
GPU; these checks cover many more trees than the GPU parity tests run."""

import pytest

from tnc_inputs import circuit_to_network, grid_rqc

TENSOR, PLANES_A, PLANES_B, SCRATCH = range(4)


def _net(r, c, cyc, seed, n_open, t, stem_cap=None):
    from paper_2205_00393_gb300 import Network
    net = Network.from_tn(circuit_to_network(grid_rqc(r, c, cyc, seed, n_open=n_open)).as_complex64())
    path = net.greedy_path()
    net.set_path(path)
    net.set_slices(net.find_slices(t, 7))
    if stem_cap is not None:
        net.set_option("stem_cap_log2", stem_cap)
    return net, path


def _check(net, path, batch, mode, reuse):
    a = net.arena(batch, mode, reuse)
    n_leaves = len(path) + 1
    children = {n_leaves + i: tuple(p) for i, p in enumerate(path)}
    root = n_leaves + len(path) - 1
    live, alloc_step, free_step, top = {}, {}, {}, 0
    alloc_at, free_at = {}, {}  # event positions
    for pos, (op, kind, ident, off, ln, step) in enumerate(a["events"]):
        key = (kind, ident)
        if op == 0:
            assert key not in live, key
            for o2, l2, _ in live.values():
                assert off + ln <= o2 or o2 + l2 <= off, (key, off, ln, o2, l2)
            live[key] = (off, ln, step)
            top = max(top, off + ln)
            if kind == TENSOR:
                alloc_step[ident] = step
                alloc_at[ident] = pos
        else:
            assert reuse, "released without reuse"
            assert key in live and live[key][:2] == (off, ln), key
            a_step = live.pop(key)[2]
            if kind in (PLANES_A, PLANES_B):
                assert a_step == step, key  # planes live only during their level
            if kind == TENSOR:
                free_step[ident] = step
                free_at[ident] = pos
    assert top == a["peak"]
    scratch = [s for op, kind, _, _, _, s in a["events"] if op == 0 and kind == SCRATCH]
    assert len(scratch) == 1
    for v, kids in children.items():
        for c in kids:
            if c < n_leaves or c not in alloc_step:
                continue  # a leaf, or an intermediate kept on chip inside a fused stem group
            if v == root:
                assert c not in free_step and alloc_step[c] < scratch[0]
                continue
            if v not in alloc_step:
                continue  # inside a fused group: its group output is checked against the group's input
            assert alloc_step[c] < alloc_step[v], (c, v)
            if c in free_step:
                # released at the parent's level, after the parent's output is
                # placed (so the output never takes the input's bytes)
                assert free_step[c] == alloc_step[v], (c, v, free_step[c], alloc_step[v])
                assert free_at[c] > alloc_at[v], (c, v)
    return a


@pytest.mark.parametrize("reuse", [1, 0])
@pytest.mark.parametrize("mode", [0, 2, 4])
@pytest.mark.parametrize("spec", [(3, 4, 8, 1, 0, 8), (4, 5, 12, 3, 3, 16), (4, 6, 12, 3, 4, 20),
                                  (5, 6, 14, 2, 6, 27)])
def test_arena_plan(libtnc, spec, mode, reuse):
    for stem_cap in (0, None):  # without fused stem groups, and with the default
        net, path = _net(*spec, stem_cap=stem_cap)
        for batch in (1, 4):
            _check(net, path, batch, mode, reuse)


def test_arena_reuse_saves_bytes(libtnc):
    """On the 30-qubit workload (4 slices) the reusing plan never needs more
    than one that keeps every tensor, and in the split modes, whose operand
    planes are dead after their level, clearly less (13.8 against 19.3 GB in
    FP16x2); tnc_workspace_bytes, the largest reusing plan over the modes,
    covers each mode's."""
    net, path = _net(5, 6, 14, 2, 6, 27, stem_cap=0)
    ws = net.workspace_bytes(4)
    for mode in (0, 2, 4):
        r, f = net.arena(4, mode, 1)["peak"], net.arena(4, mode, 0)["peak"]
        assert r <= f and r <= ws
        if mode:
            assert r < 0.8 * f


def test_arena_errors(libtnc):
    from paper_2205_00393_gb300 import TNCError
    net, _ = _net(3, 4, 8, 1, 0, 8)
    for args in ((0, 0, 1), (2000, 0, 1), (4, 9, 1), (4, 0, 2)):
        with pytest.raises(TNCError) as e:
            net.arena(*args)
        assert e.value.status == 1
