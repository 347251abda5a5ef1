"""Fused stem groups (secondary slicing, Sec. 5.2) as planned on the host, no
GPU: the paper's Fig. 9 example and the groups on a stem path."""

import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "secondary_slicing_fig9.json")


def fig9_network():
    """A sub-path like Fig. 9's: T_0 = P (x) Q has 8 modes; three narrow steps
    absorb B1, B2, B3; five edges a1..a5 live through all of them; R closes
    the network. Index ids: a1..a5 = 0..4, c1..c3 = 5..7, d1..d3 = 8..10."""
    from tnc_inputs.network import TensorNetwork
    rng = np.random.default_rng(9)
    idx = [(0, 1, 2, 5), (3, 4, 6, 7), (5, 8), (6, 7, 9), (8, 9, 10), (0, 1, 2, 3, 4, 10)]
    ts = [((rng.standard_normal((2,) * len(i)) + 1j * rng.standard_normal((2,) * len(i))) / 2).astype(np.complex64)
          for i in idx]
    path = [(0, 1), (6, 2), (7, 3), (8, 4), (9, 5)]
    return TensorNetwork(ts, idx, np.full(11, 2, dtype=np.int64), (), [-1] * 6), path


def test_fig9_secondary_slicing_group(libtnc):
    """With the on-chip capacity set to 2^3 elements, the three steps form one
    group whose outer modes are the five crossing edges (2^5 subtasks) and
    whose largest inner sub-tensor has 2^3 elements, down from 2^8."""
    from paper_2205_00393_gb300 import Network
    gold = json.load(open(GOLDEN))
    tn_, path = fig9_network()
    net = Network.from_tn(tn_)
    net.set_path(path)
    net.set_option("stem_cap_log2", gold["max_log2_after"])
    net.set_option("stem_min_outer_log2", gold["subtasks_log2"])
    net.set_option("stem_coalesce_bits", 0)  # the paper's example picks modes by lifetime alone
    st = net.stats()
    assert st["max_log2_size"] == gold["max_log2_before"]
    assert st["stem_groups"] == [[1, 3, gold["crossing_edges"], gold["max_log2_after"], 0, 8, 6]]
    # with a smaller capacity the three steps no longer fit one group (each
    # runs in a shorter group or alone); fusion off leaves no group at all
    net.set_option("stem_cap_log2", 2)
    assert all(g[1] < 3 for g in net.stats()["stem_groups"])
    net.set_option("stem_cap_log2", 0)
    assert net.stats()["stem_groups"] == []


def test_groups_on_a_stem_path(libtnc):
    """On the time-ordered stem path of a 20-qubit circuit every contraction
    is a narrow stem step; groups cover consecutive steps, each with at least
    2^7 outer assignments and inner sub-tensors within the default cap
    (2^13 elements), most of them several steps long."""
    from paper_2205_00393_gb300 import Network
    from tnc_inputs import circuit_to_network, grid_rqc, stem_path
    c = grid_rqc(4, 5, 10, 11, n_open=4)
    tn_ = circuit_to_network(c).as_complex64()
    net = Network.from_tn(tn_)
    net.set_path(stem_path(tn_, c))
    st = net.stats()
    groups = st["stem_groups"]
    assert groups, "expected fused groups on a stem path"
    firsts = [g[0] for g in groups]
    assert len(set(firsts)) == len(firsts)
    assert st["stem_cap_log2"] == 13
    for first, n, nu, inner, per_slice, _, _ in groups:
        assert n >= 1 and nu >= 7 and inner <= 13 and per_slice == 0
    assert sum(1 for g in groups if g[1] >= 4) >= len(groups) // 2
    assert sum(g[1] for g in groups) >= len(st["nodes"]) // 2
