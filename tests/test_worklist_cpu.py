"""The persistent executor's work lists (tnc_worklist_json), checked on the
host without a GPU for the properties its correctness rests on, in both
dependency modes:

* progress: tasks are taken in list order, so every counter a task waits on
  must be signalled only by tasks before it (then the first unfinished task
  can always run, whatever the number of CTAs);
* accounting: a counter starts at the number of tasks that signal it, so it
  reaches zero exactly when they are all done;
* ordering of data: the final sum comes after every other task; a tile of a
  contraction above the first per-slice level comes after a tile of the
  level below of its own batch entry; with per-entry dependencies
  (deps = 1) no per-slice predecessor belongs to another batch entry (a
  slice-invariant producer serves every entry), and with the level chain
  (deps = 0) every task comes after the whole previous level.

FP32 mode only: its lists need no tensor maps, so no CUDA driver."""

import collections

import pytest

from tnc_inputs import circuit_to_network, grid_rqc

GEMM, SPLIT, TC, KRED, ROOT, ACC, SUM = range(7)


def _net(r, c, cyc, seed, n_open, t):
    from paper_2205_00393_gb300 import Network
    net = Network.from_tn(circuit_to_network(grid_rqc(r, c, cyc, seed, n_open=n_open)).as_complex64())
    net.set_path(net.greedy_path())
    net.set_slices(net.find_slices(t, 7))
    net.set_option("stem_cap_log2", 0)  # no fused stem groups: the whole tree runs in the list
    return net


def _signallers(tasks):
    by = collections.defaultdict(list)
    for i, t in enumerate(tasks):
        by[t[7]].append(i)
        if t[8] >= 0:
            by[t[8]].append(i)
    return by


def _closure(tasks, by, i):
    """Every task that task i waits on, directly or through the tasks it waits on."""
    seen, stack = set(), [i]
    while stack:
        for c in tasks[stack.pop()][4:7]:
            if c < 0:
                continue
            for j in by[c]:
                if j not in seen:
                    seen.add(j)
                    stack.append(j)
    return seen


@pytest.mark.parametrize("deps", [1, 0])
@pytest.mark.parametrize("spec,batch", [((3, 4, 8, 1, 0, 8), 4), ((4, 5, 12, 3, 3, 16), 2)])
def test_worklist_invariants(libtnc, spec, batch, deps):
    net = _net(*spec)
    wl = net.worklist(batch, 0, deps)
    tasks, counters = wl["tasks"], wl["counters"]
    assert wl["chain"] == 1 - deps
    assert tasks and all(t[0] in (GEMM, ROOT, ACC, SUM) for t in tasks)
    by = _signallers(tasks)
    # accounting
    for c, init in enumerate(counters):
        assert init == len(by[c]), (c, init, len(by[c]))
    # progress: waits name earlier tasks only
    for i, t in enumerate(tasks):
        for c in t[4:7]:
            if c >= 0:
                assert by[c] and max(by[c]) < i, (i, c)
    # the chain mode: a task also counts down its level, and every task past
    # the first level waits on the previous one; per-entry mode: no level counters
    if deps:
        assert all(t[8] == -1 for t in tasks)
    else:
        assert all(t[8] >= 0 for t in tasks)
        first_level = min(t[9] for t in tasks)
        for t in tasks:
            if t[9] > first_level:
                assert any(c >= 0 and all(tasks[j][9] == t[9] - 1 for j in by[c]) for c in t[4:7])
    # ordering of data. Every task feeds the result, so the final sum's
    # predecessors (direct or through other tasks) are all other tasks.
    final = [i for i, t in enumerate(tasks) if t[0] in (ACC, SUM)]
    assert len(final) == 1
    assert _closure(tasks, by, final[0]) == set(range(len(tasks))) - set(final)
    # A parameter entry with tasks of several batch entries is per-slice, one
    # with entry 0 only is slice-invariant (batch >= 2 here).
    zs = collections.defaultdict(set)
    for t in tasks:
        zs[(t[0], t[1])].add(t[3])
    per_slice = {k for k, v in zs.items() if len(v) > 1}
    tiles = [i for i, t in enumerate(tasks) if t[0] == GEMM and (t[0], t[1]) in per_slice]
    first = min(tasks[i][9] for i in tiles)
    for i in tiles:
        t, pred = tasks[i], _closure(tasks, by, i)
        if deps:
            # per entry: no per-slice predecessor of another batch entry
            assert all(tasks[j][3] == t[3] for j in pred if (tasks[j][0], tasks[j][1]) in per_slice), i
        else:
            # the chain: every task of the previous level
            assert all(j in pred for j, u in enumerate(tasks) if u[9] == t[9] - 1), i
        if t[9] > first:
            # a contraction above the first per-slice level reads one from
            # the level below, of its own entry
            assert any(tasks[j][9] == t[9] - 1 and tasks[j][3] == t[3] and (tasks[j][0], tasks[j][1]) in per_slice
                       for j in pred), i


def test_worklist_deps_wait_less(libtnc):
    """The same tasks with per-entry dependencies have strictly fewer
    transitive predecessors in total than with the level chain: the levels of
    different batch entries are no longer serialised."""
    net = _net(3, 4, 8, 1, 0, 8)
    a, b = net.worklist(8, 0, 1), net.worklist(8, 0, 0)
    assert len(a["tasks"]) == len(b["tasks"])
    ca = sum(len(_closure(a["tasks"], _signallers(a["tasks"]), i)) for i in range(len(a["tasks"])))
    cb = sum(len(_closure(b["tasks"], _signallers(b["tasks"]), i)) for i in range(len(b["tasks"])))
    assert ca < cb


def test_worklist_errors(libtnc):
    from paper_2205_00393_gb300 import TNCError
    net = _net(3, 4, 8, 1, 0, 8)
    for args in ((0, 0, 1), (2000, 0, 1), (4, 9, 1), (4, 0, 2)):
        with pytest.raises(TNCError) as e:
            net.worklist(*args)
        assert e.value.status == 1
