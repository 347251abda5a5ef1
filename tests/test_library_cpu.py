"""CPU-side tests of libtnc: the library loads and exports every entry point
of include/tnc.h, validates its inputs, and its host planner matches the
oracle's planning twin bit for bit (greedy paths, slicing sets in insertion
order, Eq. 1/Eq. 3 costs). No GPU call is made here."""

import os
import re

import numpy as np
import pytest

from tnc_inputs import circuit_to_network, grid_rqc, lattice_53q_rqc
from oracle import planner

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:tnc_status|const char\*|void)\s+(tnc_\w+)\s*\(", txt, re.M))
    return names


def test_exports_every_declared_symbol(libtnc):
    names = _declared()
    assert {"tnc_create_network", "tnc_set_path", "tnc_set_slices", "tnc_contract"} <= names
    for n in sorted(names):
        assert hasattr(libtnc, n), n


def _net(c):
    from paper_2205_00393_gb300 import Network
    tn = circuit_to_network(c)
    return tn, Network.from_tn(tn)


def test_validation_errors(libtnc):
    from paper_2205_00393_gb300 import Network, TNCError
    t = np.ones((2, 2), dtype=np.complex64)
    # index on three tensors
    with pytest.raises(TNCError):
        Network([t, t, t], [(0, 1), (0, 2), (0, 3)], [2, 2, 2, 2], [1, 2, 3])
    # non power of two
    with pytest.raises(TNCError):
        Network([np.ones((3,), np.complex64)], [(0,)], [3], [0])
    # dangling index not declared open
    with pytest.raises(TNCError):
        Network([t], [(0, 1)], [2, 2], [0])
    # repeated index within a tensor
    with pytest.raises(TNCError):
        Network([t], [(0, 0)], [2], [])
    n = Network([t, t], [(0, 1), (1, 2)], [2, 2, 2], [0, 2])
    with pytest.raises(TNCError) as e:
        n.set_slices([1])
    assert e.value.status == 5  # TNC_E_STATE before a path
    with pytest.raises(TNCError):
        n.set_path([(0, 0)])
    n.set_path([(0, 1)])
    with pytest.raises(TNCError):
        n.set_slices([0])  # open
    n.set_slices([1])
    assert n.n_slices == 2


CASES = [(3, 4, 8, 1, 0), (3, 3, 6, 2, 3), (2, 4, 8, 2, 0), (5, 6, 14, 2, 6), (4, 5, 12, 7, 2)]


@pytest.mark.parametrize("rows,cols,cyc,seed,n_open", CASES)
def test_greedy_path_twin(libtnc, rows, cols, cyc, seed, n_open):
    c = grid_rqc(rows, cols, cyc, seed, n_open=n_open)
    tn, net = _net(c)
    assert net.greedy_path() == planner.greedy_path(tn.indices, tn.dims)


def test_greedy_path_twin_53q(libtnc):
    c = lattice_53q_rqc(12, 3)
    tn, net = _net(c)
    assert net.greedy_path() == planner.greedy_path(tn.indices, tn.dims)


@pytest.mark.parametrize("rows,cols,cyc,seed,n_open,t,sa_seed", [
    (3, 4, 8, 1, 0, 8, 7), (3, 4, 8, 1, 0, 6, 3), (3, 3, 6, 2, 3, 5, 1),
    (5, 6, 14, 2, 6, 27, 7), (5, 6, 14, 2, 6, 24, 99), (4, 5, 12, 7, 2, 16, 5),
])
def test_slicer_twin(libtnc, rows, cols, cyc, seed, n_open, t, sa_seed):
    c = grid_rqc(rows, cols, cyc, seed, n_open=n_open)
    tn, net = _net(c)
    path = planner.greedy_path(tn.indices, tn.dims)
    net.set_path(path)
    tree = planner.Tree(tn.indices, tn.dims, tn.open_ids, path)
    S_py = planner.find_slices(tree, t, sa_seed)
    S_c = net.find_slices(t, sa_seed)
    assert S_c == S_py
    net.set_slices(S_c)
    st = net.stats()
    assert int(st["eq1"]) == tree.eq1()
    assert int(st["eq3"]) == tree.eq3(S_py)
    assert st["max_log2_size"] <= max(tree.size_log(v) for v in range(tree.n_tensors))


def test_slicer_twin_random_small_trees(libtnc):
    rng = np.random.default_rng(123)
    for trial in range(30):
        rows, cols = int(rng.integers(2, 4)), int(rng.integers(2, 5))
        c = grid_rqc(rows, cols, int(rng.integers(4, 10)), int(rng.integers(0, 10**6)),
                     n_open=int(rng.integers(0, 3)))
        tn, net = _net(c)
        path = planner.greedy_path(tn.indices, tn.dims)
        net.set_path(path)
        tree = planner.Tree(tn.indices, tn.dims, tn.open_ids, path)
        W = max(tree.size_log(v) for v in range(tree.n_tensors))
        t = max(W - int(rng.integers(1, 4)), 4 + len(tn.open_ids))
        seed = int(rng.integers(0, 2**63))
        try:
            S_py = planner.find_slices(tree, t, seed)
        except planner.Infeasible:
            from paper_2205_00393_gb300 import TNCError
            with pytest.raises(TNCError):
                net.find_slices(t, seed)
            continue
        assert net.find_slices(t, seed) == S_py


def test_eq3_wide_costs(libtnc):
    """53-qubit tree: Eq. 1 and Eq. 3 exceed 2^90; the exact wide-integer cost matches Python."""
    c = lattice_53q_rqc(20, 3)
    tn, net = _net(c)
    path = planner.greedy_path(tn.indices, tn.dims)
    net.set_path(path)
    tree = planner.Tree(tn.indices, tn.dims, tn.open_ids, path)
    S1 = planner.slice_finder(tree, 30)[:60]  # at most 62 sliced indices are accepted
    net.set_slices(S1)
    st = net.stats()
    assert int(st["eq3"]) == tree.eq3(S1) and tree.eq3(S1) > 2 ** 100
    assert int(st["eq1"]) == tree.eq1()


def test_tensor_core_cuts_on_the_53_qubit_plan():
    """tnc_stats reports how every tensor-core-eligible contraction is cut up
    (host logic, no GPU): K panels only for K-dominant contractions whose
    planes exceed the cap, each row or K panel within the cap unless it is
    already a single 128-row tile (or 64 of K), and K splits only while the
    output tiles fill fewer than four waves of 152 SMs, keeping at least 4096
    of K per split. On the 53-qubit lattice both K-dominant nodes run in K
    panels, and the one with few output tiles also splits K."""
    from tnc_inputs import circuit_to_network, lattice_53q_rqc
    from paper_2205_00393_gb300 import Network
    net = Network.from_tn(circuit_to_network(lattice_53q_rqc(20, 3)).as_complex64())
    net.set_path(net.greedy_path())
    net.set_slices(net.find_slices(30, 7))
    st = net.stats()
    b = st["tc_cut_batch"]
    cap = 1 << 32
    # (planes, bytes per element): the parts of Re and of Im
    planes = {"1": (4, 4), "2": (6, 2), "3": (4, 2), "4": (4, 2)}

    def align(x):
        return (x + 255) // 256 * 256
    seen = {}
    for mode, cuts in st["tc_cuts"].items():
        n_pl, elem = planes[mode]
        for i, pA, pB, pK, ks in cuts:
            mb, nb, kb = st["nodes"][i][:3]
            per = st["nodes"][i][3]
            bb = b if per else 1

            def fits(rb, k):  # split FP16x2 adds one scale byte per row and 256-wide K chunk
                scales = align(bb * (1 << max(k - 8, 0)) << rb) if mode == "4" else 0
                return align(bb * n_pl * elem * (1 << (rb + k))) + scales <= cap
            if pK:
                assert kb > max(mb, nb)
                assert fits(mb, kb - pK) and fits(nb, kb - pK) or kb - pK == 6
                assert not (fits(mb, kb - pK + 1) and fits(nb, kb - pK + 1))
            assert fits(mb - pA, kb - pK) or mb - pA == 7
            assert fits(nb - pB, kb - pK) or nb - pB == 7
            tiles = bb << ((mb - pA - 7) + (nb - pB - 7))
            if ks:
                assert (tiles << (ks - 1)) < 4 * 152 and kb - pK - ks >= 12
            else:
                assert tiles >= 4 * 152 or kb - pK <= 12
            seen[(mode, mb, nb, kb)] = (pA, pB, pK, ks)
    for mode in ("1", "2", "4"):
        assert seen[(mode, 12, 12, 18)][2] > 0
        assert seen[(mode, 11, 10, 19)][2] > 0 and seen[(mode, 11, 10, 19)][3] > 0


def test_option_validation():
    """tnc_set_option accepts each documented key within its range and
    rejects unknown keys and out-of-range values with TNC_E_INVALID (host
    logic, no GPU)."""
    from paper_2205_00393_gb300 import Network, TNCError
    t = np.ones((2, 2), dtype=np.complex64)
    net = Network([t, t], [(0, 1), (1, 2)], [2, 2, 2], [0, 2])
    good = {"tc_row_bytes": [32, 64], "tc_group_m": [1, 64],
            "tc_plane_cap_log2": [16, 40], "backward_keep_every": [0, 64], "cache_invariants": [0, 1],
            "tc_spin_limit": [0, 1 << 20], "tc_test_stall": [0], "stem_cap_log2": [0, 2, 13],
            "persistent": [0, 1, 2], "persist_deps": [0, 1]}
    bad = {"tc_row_bytes": [16, 128], "tc_group_m": [0, 65], "tc_pair": [0, 1], "tc_multicast": [0, 1],
           "tc_plane_cap_log2": [15, 41], "backward_keep_every": [-1, 65], "tc_spin_limit": [-1], "no_such_key": [1],
           "stem_cap_log2": [1, 14], "persistent": [-1, 3], "persist_deps": [-1, 2]}
    for k, vals in good.items():
        for v in vals:
            net.set_option(k, v)
    for k, vals in bad.items():
        for v in vals:
            with pytest.raises(TNCError) as e:
                net.set_option(k, v)
            assert e.value.status == 1, (k, v)


def test_executor_choice_inputs_in_stats():
    """tnc_stats carries what the automatic executor choice reads (host logic,
    no GPU): per mode, the per-level launches of a batch and their estimated
    seconds; the 12-qubit grid circuit's estimate is far below the 0.1 us
    per launch under which calls run persistent, the 30-qubit workload's far
    above. The dependency option is reported, and no contraction has run yet
    (no workspace sizes)."""
    from paper_2205_00393_gb300 import Network
    from tnc_inputs import circuit_to_network, grid_rqc

    def planned(r, c, cyc, seed, n_open, t):
        net = Network.from_tn(circuit_to_network(grid_rqc(r, c, cyc, seed, n_open=n_open)).as_complex64())
        net.set_path(net.greedy_path())
        net.set_slices(net.find_slices(t, 7))
        return net.stats()

    small, big = planned(3, 4, 8, 1, 0, 8), planned(5, 6, 14, 2, 6, 27)
    for st in (small, big):
        assert sorted(st["level_cost"]) == ["0", "1", "2", "3", "4"]
        for launches, seconds in st["level_cost"].values():
            assert launches >= 1 and seconds > 0
        assert st["persist_deps"] == 1 and st["last_persist_deps"] == 0 and st["last_workspace"] == [0, 0]
    per_launch = lambda st, m: st["level_cost"][m][1] / st["level_cost"][m][0]
    assert per_launch(small, "4") < 0.1e-6 < per_launch(big, "4")
    # a tensor-core mode launches the operand splits too
    assert big["level_cost"]["4"][0] > big["level_cost"]["0"][0]
