"""Contraction paths given as input, besides the greedy one the library plans.

``stem_path`` builds the path of a stem in the sense of the paper's stem
(Sec. 4.2 after Huang et al.): one big tensor that absorbs small ones one after
another. It follows the circuit's time order, so the stem holds the qubits
that a gate has touched so far, like a state vector, and every absorption is
a narrow contraction (a gate: 2 or 4 contracted elements, 2 or 4 new ones).
This is the regime the paper's secondary slicing (Sec. 5.2) targets. No
arithmetic of the method lives here: the path is a list of SSA pairs, leaves
0..n-1 and step i creating tensor n + i.
"""


def stem_path(network, circuit):
    """SSA path for ``network = circuit_to_network(circuit)``.

    Per qubit a branch starts from its |0> vector and absorbs the qubit's
    single-qubit gates until the qubit meets its first two-qubit gate; that
    gate absorbs the branches of its fresh qubits and then joins the stem (on
    two fresh qubits it starts the stem, or joins it as an outer product).
    After that every gate on a qubit of the stem is absorbed by the stem.
    Finally the stem absorbs the branches of qubits that never met a
    two-qubit gate and the projection vectors of the closed qubits."""
    nq = circuit.n_qubits
    n_gates = len(circuit.gates)
    n_leaves = network.n_tensors
    path = []
    nxt = [n_leaves]

    def join(a, b):
        path.append((int(a), int(b)))
        nxt[0] += 1
        return nxt[0] - 1

    pending = list(range(nq))  # branch tensor per qubit until it joins the stem
    in_stem = [False] * nq
    stem = None
    for gi, g in enumerate(circuit.gates):
        leaf = nq + gi
        qs = list(g.qubits)
        if len(qs) == 1 and not in_stem[qs[0]]:
            pending[qs[0]] = join(pending[qs[0]], leaf)
            continue
        t = leaf
        for q in qs:
            if not in_stem[q]:
                t = join(t, pending[q])
                in_stem[q] = True
                pending[q] = None
        stem = t if stem is None else join(stem, t)
    for q in range(nq):
        if pending[q] is not None:
            stem = pending[q] if stem is None else join(stem, pending[q])
    for leaf in range(nq + n_gates, n_leaves):  # projection vectors of closed qubits
        stem = join(stem, leaf)
    return path

