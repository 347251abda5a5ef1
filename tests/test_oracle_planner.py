"""Pins for the planning twin: lifetimes, Eq. 1/2/3, stem, Algorithms 1-4,
the greedy path and the PRNG.

Pins used: the paper's worked lifetime example (Sec. 3.1) and the
superposition multipliers (Sec. 3.2, Supplementary S2) under tests/golden/,
the Linearity theorem (Supplementary S1) as a property, brute force over all
slicing sets on small trees (Algorithm 1 size, Theorem 1, the Eq. 3 optimum
bound of Algorithm 2), the constraint of Sec. 4.1 after every refiner move,
a hand-derived greedy path and splitmix64's published first output.
"""

import itertools
import json
import os

import numpy as np
import pytest

from tnc_inputs import circuit_to_network, grid_rqc
from oracle import planner

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_lifetime_worked_example():
    g = _load("lifetime_fig4.json")
    names = g["index_names"]
    nid = {n: i for i, n in enumerate(names)}
    leaves = [tuple(nid[x] for x in leaf) for leaf in g["leaves"]]
    dims = np.full(len(names), 2)
    tree = planner.Tree(leaves, dims, [nid[x] for x in g["open"]], [tuple(p) for p in g["path"]])
    got = [set(tree.idx[v]) for v in range(len(leaves), tree.n_tensors)]
    assert got == [set(nid[x] for x in t) for t in g["intermediates"]]
    lf = [set(tree.idx[v]) for v in tree.lifetime(nid["e"])]
    assert sorted(map(sorted, lf)) == sorted(sorted(nid[x] for x in t) for t in g["lifetime_e"])
    assert len(tree.correlated_contractions(nid["e"])) == g["n_correlated_contractions_e"]


def _chain(spans):
    """Chain tree X0 -> X5 absorbing Y1..Y5; index ``name`` lies in the node
    index sets of parts spans[name][0]..spans[name][1]."""
    names = ["o0", "o5"] + ["c%d" % i for i in range(1, 6)] + sorted(spans)
    nid = {n: i for i, n in enumerate(names)}
    X0 = ["o0", "c1"]
    Y = {p: ["c%d" % p] + (["c%d" % (p + 1)] if p < 5 else ["o5"]) for p in range(1, 6)}
    for name, (p, q) in sorted(spans.items()):
        (X0 if p == 1 else Y[p]).append(name)
        Y[q].append(name)
    leaves = [tuple(nid[x] for x in X0)] + [tuple(nid[x] for x in Y[p]) for p in range(1, 6)]
    path = [(0, 1)] + [(6 + i, i + 2) for i in range(4)]
    tree = planner.Tree(leaves, np.full(len(names), 2), [nid["o0"], nid["o5"]], path)
    return tree, nid


def test_overhead_superposition_multipliers():
    g = _load("overhead_superposition.json")
    for case in g["cases"]:
        tree, nid = _chain({k: tuple(v) for k, v in case["spans"].items()})
        S = frozenset(nid[x] for x in case["sliced"])
        mult = [(tree.node_cost(i, S) << len(S)) // tree.node_cost(i) for i in range(5)]
        assert mult == case["multipliers"]
        # Eq. 3 is the multiplier-weighted sum of the Eq. 1 terms
        assert tree.eq3(S) == sum(m * tree.node_cost(i) for i, m in enumerate(mult))


def _c1_tree():
    c = grid_rqc(3, 4, 8, 1)
    net = circuit_to_network(c)
    path = planner.greedy_path(net.indices, net.dims)
    return planner.Tree(net.indices, net.dims, net.open_ids, path)


def test_linearity_of_lifetimes():
    """Supplementary S1: each index's lifetime lies on one tree path, from
    leaf to leaf (closed) or leaf to root (open); correlated contractions are
    exactly the nodes on that path."""
    c = grid_rqc(3, 3, 5, 4, n_open=2)
    net = circuit_to_network(c)
    tree = planner.Tree(net.indices, net.dims, net.open_ids,
                        planner.greedy_path(net.indices, net.dims))
    for e in tree.all_indices():
        lf = set(tree.lifetime(e))
        leaves = [v for v in lf if v < tree.n_leaves]
        tops = [v for v in lf if tree.parent[v] == -1 or tree.parent[v] not in lf]
        if e in tree.open:
            assert len(leaves) == 1 and tops == [tree.root]
        else:
            assert len(leaves) == 2 and len(tops) == 2
            assert tree.parent[tops[0]] == tree.parent[tops[1]]
        # every lifetime tensor except the tops has its parent in the lifetime
        for v in lf:
            if v not in tops:
                assert tree.parent[v] in lf
        cc = set(tree.correlated_contractions(e))
        assert cc == {tree.parent[v] for v in lf if tree.parent[v] != -1}


def test_stem_follows_costliest_child():
    tree = _c1_tree()
    cost = tree.subtree_cost()
    stem = tree.stem()
    assert stem[-1] == tree.root and stem[0] < tree.n_leaves
    for lo, hi in zip(stem[:-1], stem[1:]):
        a, b = tree.children[hi - tree.n_leaves]
        other = b if lo == a else a
        assert lo in (a, b)
        assert cost[lo] >= cost[other]


def _small_trees():
    for (r, c_, cyc, seed) in [(2, 3, 8, 1), (2, 4, 8, 2), (3, 3, 8, 5), (3, 4, 8, 1)]:
        circ = grid_rqc(r, c_, cyc, seed)
        net = circuit_to_network(circ)
        yield planner.Tree(net.indices, net.dims, net.open_ids,
                           planner.greedy_path(net.indices, net.dims))


def _universe(tree, t):
    """Closed indices of the tensors larger than 2^t: every index a slicing
    set needs, and every index Algorithms 1, 2 and 4 can pick, lies here."""
    big = [v for v in range(tree.n_tensors) if tree.size_log(v) > t]
    return sorted({e for v in big for e in tree.idx[v] if e not in tree.open}), big


def _valid_sets(tree, t, size, universe, big):
    for S in itertools.combinations(universe, size):
        Sset = frozenset(S)
        if all(tree.dim(v, Sset) <= t for v in big):
            yield S


def test_slice_finder_against_brute_force():
    for tree in _small_trees():
        W = max(tree.size_log(v) for v in range(tree.n_tensors))
        for t in range(max(W - 3, 4), W):
            closed, big = _universe(tree, t)
            S = planner.slice_finder(tree, t)
            assert tree.satisfies(S, t)
            assert len(set(S)) == len(S)
            # smallest valid set by exhaustive search
            best = None
            for k in range(0, len(S) + 1):
                if any(True for _ in _valid_sets(tree, t, k, closed, big)):
                    best = k
                    break
            assert best is not None and best <= len(S)


def test_refiner_keeps_constraint_and_never_worsens():
    for tree in _small_trees():
        W = max(tree.size_log(v) for v in range(tree.n_tensors))
        t = max(W - 3, 4)
        S1 = planner.slice_finder(tree, t)
        trace = []
        S2 = planner.slice_refiner(tree, t, S1, seed=11, trace=trace)
        for S in trace:
            assert tree.satisfies(S, t)
        assert tree.satisfies(S2, t)
        assert tree.eq3(S2) <= tree.eq3(S1)
        assert len(S2) <= len(S1)
        # no valid set of the same size beats the exhaustive optimum
        closed, big = _universe(tree, t)
        assert set(S2) <= set(closed)
        opt = min(tree.eq3(S) for S in _valid_sets(tree, t, len(S2), closed, big))
        assert opt <= tree.eq3(S2)


def test_theorem1_brute_force():
    """Theorem 1 (Sec. 3.2): if a valid (n-1)-set meets a valid n-set, some
    valid (n-1)-set costs no more than the n-set (equality only when the
    extra index spans every node)."""
    checked = 0
    for tree in list(_small_trees()):
        W = max(tree.size_log(v) for v in range(tree.n_tensors))
        t = max(W - 3, 4)
        closed, big = _universe(tree, t)
        n = len(planner.slice_finder(tree, t)) + 1
        small = list(_valid_sets(tree, t, n - 1, closed, big))
        if not small:
            continue
        best_small = min(tree.eq3(S) for S in small)
        for S1 in _valid_sets(tree, t, n, closed, big):
            if any(set(S1) & set(S2) for S2 in small):
                assert best_small <= tree.eq3(S1)
                checked += 1
    assert checked > 0


def test_eq2_overhead_matches_definition():
    tree = _c1_tree()
    S = planner.find_slices(tree, 8, seed=2)
    per_slice = sum(tree.node_cost(i, frozenset(S)) for i in range(len(tree.children)))
    assert tree.overhead(S) == per_slice * 2 ** len(S) / tree.eq1()
    assert tree.overhead([]) == 1.0


def test_greedy_hand_example():
    # leaves: L0=(a,b,c) L1=(c,d,e) L2=(e,f) L3=(b,f,g,h); open a,d,g,h.
    # phase 1: L2 (rank 2) joins its largest-rank neighbour L3 -> T4=(e,b,g,h)
    # phase 2 costs size(out)-size(a)-size(b): (0,1) -> 16-8-8=0,
    #   (0,4) -> 32-8-16=8, (1,4) -> 8; take (0,1) -> T5=(a,b,d,e);
    #   then (4,5) share b,e -> 16-16-16=-16.
    a, b, c, d, e, f, g, h = range(8)
    leaves = [(a, b, c), (c, d, e), (e, f), (b, f, g, h)]
    path = planner.greedy_path(leaves, np.full(8, 2))
    assert path == [(2, 3), (0, 1), (4, 5)]
    tree = planner.Tree(leaves, np.full(8, 2), [a, d, g, h], path)
    assert set(tree.idx[tree.root]) == {a, d, g, h}


def test_greedy_path_is_valid_tree():
    for tree in _small_trees():
        assert len(tree.children) == tree.n_leaves - 1


def test_splitmix64_published_value():
    # first output of splitmix64 seeded with 0 (Vigna's reference implementation)
    assert planner.SplitMix64(0).next() == 0xE220A8397B1DCDAF


def test_infeasible_target():
    tree = _c1_tree()
    with pytest.raises(planner.Infeasible):
        planner.slice_finder(tree, -1)
