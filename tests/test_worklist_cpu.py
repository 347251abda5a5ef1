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


def _preds(tasks, by):
    """Per task, the bitset of every task it waits on, directly or through the
    tasks it waits on. List order is a topological order once the progress
    check has passed, so each counter's set is built from finished ones."""
    pred, per_counter = [0] * len(tasks), {}
    for i, t in enumerate(tasks):
        p = 0
        for c in t[4:7]:
            if c < 0:
                continue
            if c not in per_counter:
                m = 0
                for j in by[c]:
                    m |= pred[j] | (1 << j)
                per_counter[c] = m
            p |= per_counter[c]
        pred[i] = p
    return pred


def _mask(indices):
    m = 0
    for i in indices:
        m |= 1 << i
    return m


def _check(wl, deps):
    tasks, counters = wl["tasks"], wl["counters"]
    n = len(tasks)
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
    pred = _preds(tasks, by)
    level = collections.defaultdict(list)
    for i, t in enumerate(tasks):
        level[t[9]].append(i)
    level = {L: _mask(v) for L, v in level.items()}
    # the chain mode: a task also counts down its level, and every task past
    # the first level follows the whole previous one; per-entry mode: no
    # level counters
    if deps:
        assert all(t[8] == -1 for t in tasks)
    else:
        assert all(t[8] >= 0 for t in tasks)
        first_level = min(level)
        for i, t in enumerate(tasks):
            if t[9] > first_level:
                assert level[t[9] - 1] & ~pred[i] == 0, i
    # ordering of data. Every task feeds the result, so the final sum follows
    # all other tasks.
    final = [i for i, t in enumerate(tasks) if t[0] in (ACC, SUM)]
    assert len(final) == 1
    assert pred[final[0]] == ((1 << n) - 1) & ~(1 << final[0])
    # A parameter entry with tasks of several batch entries is per-slice, one
    # with entry 0 only is slice-invariant (batch >= 2 here).
    zs = collections.defaultdict(set)
    for t in tasks:
        zs[(t[0], t[1])].add(t[3])
    per_slice = {k for k, v in zs.items() if len(v) > 1}
    ps_mask = _mask(i for i, t in enumerate(tasks) if (t[0], t[1]) in per_slice)
    entry = collections.defaultdict(list)
    for i, t in enumerate(tasks):
        entry[t[3]].append(i)
    entry = {z: _mask(v) for z, v in entry.items()}
    tiles = [i for i, t in enumerate(tasks) if t[0] == GEMM and (t[0], t[1]) in per_slice]
    first = min((tasks[i][9] for i in tiles), default=0)
    for i in tiles:
        t = tasks[i]
        if deps:
            # per entry: no per-slice predecessor of another batch entry
            assert pred[i] & ps_mask & ~entry[t[3]] == 0, i
        if t[9] > first:
            # a contraction above the first per-slice level reads one from
            # the level below, of its own entry
            assert pred[i] & level[t[9] - 1] & entry[t[3]] & ps_mask, i


@pytest.mark.parametrize("deps", [1, 0])
@pytest.mark.parametrize("spec,batch", [((3, 4, 8, 1, 0, 8), 4), ((4, 5, 12, 3, 3, 16), 2)])
def test_worklist_invariants(libtnc, spec, batch, deps):
    _check(_net(*spec).worklist(batch, 0, deps), deps)


@pytest.mark.parametrize("deps", [1, 0])
def test_worklist_invariants_batched_workload(libtnc, deps):
    """The first 24 circuits of the seeded batched workload (20-36 qubits,
    uneven trees), planned as the batched benchmark plans them, 2 slices;
    those whose list holds at most 2^14 tasks."""
    from paper_2205_00393_gb300 import Network
    from tnc_inputs.circuits import batched_workload
    checked = 0
    for circ, k in batched_workload(24, 1000):
        net = Network.from_tn(circuit_to_network(circ).as_complex64())
        net.set_path(net.greedy_path())
        W = net.stats()["max_log2_size"]
        t = max(min(W - k, 24), len(circ.open_qubits) + 4)
        net.set_slices(net.find_slices(t, 7))
        net.set_option("stem_cap_log2", 0)
        if net.n_slices < 2:
            continue
        wl = net.worklist(2, 0, deps)
        if len(wl["tasks"]) > 16384:  # bitsets of every task's predecessors stay small
            continue
        _check(wl, deps)
        checked += 1
    assert checked >= 12


def test_worklist_deps_wait_less(libtnc):
    """The same tasks with per-entry dependencies have strictly fewer
    transitive predecessors in total than with the level chain: the levels of
    different batch entries are no longer serialised."""
    net = _net(3, 4, 8, 1, 0, 8)
    a, b = net.worklist(8, 0, 1)["tasks"], net.worklist(8, 0, 0)["tasks"]
    assert len(a) == len(b)
    ca = sum(bin(p).count("1") for p in _preds(a, _signallers(a)))
    cb = sum(bin(p).count("1") for p in _preds(b, _signallers(b)))
    assert ca < cb


def test_worklist_errors(libtnc):
    from paper_2205_00393_gb300 import TNCError
    net = _net(3, 4, 8, 1, 0, 8)
    for args in ((0, 0, 1), (2000, 0, 1), (4, 9, 1), (4, 0, 2)):
        with pytest.raises(TNCError) as e:
            net.worklist(*args)
        assert e.value.status == 1


@pytest.mark.parametrize("deps", [1, 0])
def test_worklist_many_merged(libtnc, deps):
    """tnc_contract_many's merged list of four networks of different sizes:
    the merge keeps each network's list intact (its tasks, counters and
    initial values, offset), tasks are ordered by level across networks, no
    task waits on another network's counters, and progress and accounting
    hold for the merged list."""
    from paper_2205_00393_gb300 import worklist_many
    nets = [_net(3, 4, 8, 1, 0, 8), _net(4, 5, 12, 3, 3, 16), _net(3, 3, 7, 3, 1, 7), _net(4, 4, 10, 2, 2, 12)]
    merged = worklist_many(nets, 2, 0, deps)
    tasks, counters = merged["tasks"], merged["counters"]
    by = _signallers(tasks)
    for c, init in enumerate(counters):
        assert init == len(by[c])
    for i, t in enumerate(tasks):
        for c in t[4:7]:
            if c >= 0:
                assert by[c] and max(by[c]) < i
                assert all(tasks[j][10] == t[10] for j in by[c]), (i, c)
    assert [t[9] for t in tasks] == sorted(t[9] for t in tasks)
    # each network's share equals its own list, up to the offsets
    for k, net in enumerate(nets):
        own = net.worklist(2, 0, deps)
        mine = [t for t in tasks if t[10] == k]
        assert len(mine) == len(own["tasks"])
        assert sorted((t[0], t[2], t[3]) for t in mine) == sorted((t[0], t[2], t[3]) for t in own["tasks"])
        used = sorted({c for t in mine for c in (t[4], t[5], t[6], t[7], t[8]) if c >= 0})
        assert sorted(counters[c] for c in used) == sorted(own["counters"])
        # the network's own invariants on its share (counters renumbered)
        ren = {c: r for r, c in enumerate(used)}
        sub = [t[:4] + [ren.get(c, -1) for c in t[4:9]] + t[9:] for t in mine]
        _check({"chain": merged["chain"], "counters": [counters[c] for c in used], "tasks": sub}, deps)
