"""Leaf variants (batches of correlated amplitudes, Sec. 1 and 6.2), host
side: the bitstring helpers reproduce the projection vectors of
circuit_to_network(circuit, bitstring), the library classifies a node as
per-slice exactly when its subtree holds a sliced index or a variant leaf
(everything else is shared by all variants), and bad arguments are rejected
before any device work."""

import numpy as np
import pytest

from tnc_inputs import (bitstring_variants, circuit_to_network, grid_rqc, projection_leaves,
                        random_bitstrings)


def test_bitstring_helpers_reproduce_the_networks():
    c = grid_rqc(3, 4, 8, 1, n_open=2)
    bits = random_bitstrings(c, 8, 3)
    assert bits.shape == (8, 12) and set(np.unique(bits)) <= {0, 1}
    assert not bits[:, list(c.open_qubits)].any()
    leaves, data = bitstring_variants(c, bits)
    ids, closed = projection_leaves(c)
    assert leaves == ids and len(closed) == 10 and not set(closed) & set(c.open_qubits)
    base = circuit_to_network(c, bitstring=bits[0])
    for v, b in enumerate(bits):
        net = circuit_to_network(c, bitstring=b)
        for i, leaf in enumerate(leaves):
            assert np.array_equal(net.tensors[leaf], data[i][v])
            assert net.indices[leaf] == base.indices[leaf]
        # every other leaf is the same for all bitstrings
        others = [t for t in range(net.n_tensors) if t not in set(leaves)]
        assert all(np.array_equal(net.tensors[t], base.tensors[t]) for t in others)


def _per_slice(ref, path, S, variant_leaves):
    per = [bool(set(idx) & set(S)) or (i in variant_leaves) for i, idx in enumerate(ref.indices)]
    for (a, b) in path:
        per.append(per[a] or per[b])
    return per[ref.n_tensors:]


def test_variant_leaves_make_their_ancestors_per_slice(libtnc):
    from paper_2205_00393_gb300 import Network
    c = grid_rqc(3, 4, 8, 1, n_open=0)
    ref = circuit_to_network(c).as_complex64()
    net = Network.from_tn(ref)
    path = net.greedy_path()
    net.set_path(path)
    S = net.find_slices(8, 7)
    net.set_slices(S)
    before = [n[3] for n in net.stats()["nodes"]]
    leaves, data = bitstring_variants(c, random_bitstrings(c, 5, 1))
    net.set_leaf_variants(leaves, data)
    after = [n[3] for n in net.stats()["nodes"]]
    want = _per_slice(ref, [tuple(p) for p in path], S, set(leaves))
    want[-1] = True  # the final contraction runs per slice
    assert after == [int(w) for w in want]
    assert sum(after) > sum(before)            # the projections' ancestors now vary per variant
    assert sum(1 for x in after if not x) > 0  # and a shared part remains
    net.set_leaf_variants([], [])
    assert [n[3] for n in net.stats()["nodes"]] == before


def test_variant_arguments_are_checked(libtnc):
    from paper_2205_00393_gb300 import Network, TNCError
    c = grid_rqc(3, 4, 8, 1, n_open=0)
    net = Network.from_tn(circuit_to_network(c).as_complex64())
    net.set_path(net.greedy_path())
    leaves, data = bitstring_variants(c, random_bitstrings(c, 3, 1))
    torch = pytest.importorskip("torch")
    host = torch.empty(8, dtype=torch.complex128)  # never written: every call below fails its checks first
    with pytest.raises(TNCError):
        net.contract_variants(0, 1, out=host, stream=0)           # no variants yet
    with pytest.raises(TNCError):
        net.set_leaf_variants([leaves[0], leaves[0]], [data[0], data[0]])  # repeated leaf
    with pytest.raises(TNCError):
        net.set_leaf_variants([net.n_tensors], [data[0]])  # no such leaf
    net.set_leaf_variants(leaves, data)
    with pytest.raises(TNCError):
        net.contract_variants(0, 4, out=host, stream=0)           # 3 variants
    with pytest.raises(TNCError):
        net.contract_variants(1, 0, out=host, stream=0)
    with pytest.raises(TNCError):
        net.contract(0, 5, out=host, stream=0)                    # slice ids [0, 4): 1 slice x 4 variant copies
