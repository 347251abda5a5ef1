"""Contraction-tree planning twin (oracle; test infrastructure only).

An independent Python statement of the host-side planning steps, used to check
the C++ planner bit for bit (same paths, same slicing sets in the same order).

Paper passages followed:

* Contraction tree, node index sets s_V, Eq. 1 (time complexity), Eq. 2
  (slicing overhead): Sec. 2.1.1.
* Lifetime of an index (Definition 1): the set of tree tensors containing it.
  Correlated contractions: the tree nodes whose index set contains it
  (Supplementary, Sec. S1).
* Eq. 3 cost C(B, S) and the memory constraint |S cap s_e| >= |s_e| - t for
  every tree tensor e: Sec. 4.1.
* Stem, slice finder (Algorithm 1): Sec. 4.2.
* Slice refiner by simulated annealing (Algorithm 2) with
  find_critical_tensors (Algorithm 3) and find_candidate_indices
  (Algorithm 4): Sec. 4.3 and Supplementary S3.
* Greedy path with the rank-1/rank-2 absorption pre-process (Sec. 2.1.2).

Readings where the paper is silent (shared with the C++ planner):

* T.dim = sum of log2 w(e) over the indices of T that are not sliced.
* Stem: from the root, descend into the child whose subtree Eq. 1 cost is
  larger (tie: larger output size; tie: smaller SSA id) down to a leaf; M is
  the list of stem tensors from that leaf (M[0]) to the root output (M[N-1]).
* Algorithm 1 takes its selection line literally (the end with the smaller
  dim, M[N-1] on a tie); candidates are the unsliced closed indices of
  dimension 2 of sT, ordered by lifetime length within the current M
  (descending), then by index id; every tensor of M with dim <= t is pruned.
  A global fix-up then slices, for any tree tensor still above t (tensors in
  SSA order), its candidate with the longest lifetime over the whole tree.
* Algorithm 2: splitmix64 PRNG; the index is S_sorted[(r*|S|) >> 64];
  u = (r >> 11) * 2^-53 drawn only when C_new >= C_ori; candidates are the
  Algorithm 4 intersection minus S, closed, dimension 2, ascending; each
  candidate replaces the current occupant of the chosen slot; an index
  whose lifetime holds no critical tensor is removed from S; the temperature
  starts at T0 and is multiplied by alpha after each outer iteration until it
  drops below Tf; the best S seen (first on ties) is returned.
* Eq. 3 sums over the contraction nodes of the full tree.
"""

import heapq
import math

MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 (Steele, Lea, Flood 2014; Vigna's reference constants)."""

    def __init__(self, seed):
        self.state = int(seed) & MASK64

    def next(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)


def _log2_int(x):
    x = int(x)
    if x <= 0 or x & (x - 1):
        raise ValueError("dimension is not a power of two")
    return x.bit_length() - 1


# --------------------------------------------------------------------------
# greedy path
# --------------------------------------------------------------------------

def greedy_path(indices, dims):
    """SSA contraction path: rank<=2 absorption, then pairwise greedy, then
    outer products of disconnected remainders. Pairs are (smaller, larger)."""
    logd = {}
    live = {}
    for i, idx in enumerate(indices):
        live[i] = tuple(int(e) for e in idx)
    owners = {}
    for i, idx in live.items():
        for e in idx:
            owners.setdefault(e, set()).add(i)
            logd[e] = _log2_int(dims[e])
    nxt = len(indices)
    path = []

    def neighbours(i):
        out = set()
        for e in live[i]:
            out |= owners[e]
        out.discard(i)
        return out

    def do_contract(a, b):
        nonlocal nxt
        ia, ib = live.pop(a), live.pop(b)
        sb = set(ib)
        sa = set(ia)
        new = tuple([e for e in ia if e not in sb] + [e for e in ib if e not in sa])
        for e in ia:
            owners[e].discard(a)
        for e in ib:
            owners[e].discard(b)
        for e in new:
            owners[e].add(nxt)
        live[nxt] = new
        path.append((min(a, b), max(a, b)))
        nxt += 1
        return nxt - 1

    # phase 1: absorb rank-1 and rank-2 tensors into their largest-rank neighbour
    while True:
        cands = [i for i in live if len(live[i]) <= 2 and neighbours(i)]
        if not cands:
            break
        t = min(cands)
        nb = sorted(neighbours(t), key=lambda j: (-len(live[j]), j))
        do_contract(t, nb[0])

    # phase 2: greedy pairwise, cost = size(out) - size(a) - size(b)
    def size_log(idx):
        return sum(logd[e] for e in idx)

    def pair_key(a, b):
        ia, ib = live[a], live[b]
        sa, sb = set(ia), set(ib)
        out = [e for e in ia if e not in sb] + [e for e in ib if e not in sa]
        cost = (1 << size_log(out)) - (1 << size_log(ia)) - (1 << size_log(ib))
        return (cost, min(a, b), max(a, b))

    heap = []
    for a in sorted(live):
        for b in sorted(neighbours(a)):
            if a < b:
                heap.append(pair_key(a, b))
    heapq.heapify(heap)
    while heap:
        cost, a, b = heapq.heappop(heap)
        if a not in live or b not in live:
            continue
        c = do_contract(a, b)
        for j in sorted(neighbours(c)):
            heapq.heappush(heap, pair_key(c, j))

    # phase 3: disconnected remainders, ascending SSA order
    while len(live) > 1:
        ids = sorted(live)
        do_contract(ids[0], ids[1])
    return path


# --------------------------------------------------------------------------
# contraction tree bookkeeping
# --------------------------------------------------------------------------

class Tree:
    """Contraction tree B of a network: tensors 0..n-1 are leaves, tensor n+i is
    created by path step i. ``idx[v]`` is the index tuple of tree tensor v and
    ``node[i]`` the index set s_V of contraction i (union of its inputs)."""

    def __init__(self, indices, dims, open_ids, path):
        self.n_leaves = len(indices)
        self.dims = {int(e): int(dims[e]) for idx in indices for e in idx}
        self.logd = {e: _log2_int(w) for e, w in self.dims.items()}
        self.open = frozenset(int(e) for e in open_ids)
        self.idx = [tuple(int(e) for e in t) for t in indices]
        self.children = []
        self.node = []
        self.parent = [-1] * (self.n_leaves + len(path))
        used = set()
        if len(path) != self.n_leaves - 1:
            raise ValueError("path must have n-1 steps")
        for i, (a, b) in enumerate(path):
            a, b = int(a), int(b)
            v = self.n_leaves + i
            if a == b or a in used or b in used or a >= v or b >= v or a < 0 or b < 0:
                raise ValueError("invalid SSA path")
            used.add(a)
            used.add(b)
            ia, ib = self.idx[a], self.idx[b]
            sa, sb = set(ia), set(ib)
            self.idx.append(tuple([e for e in ia if e not in sb] + [e for e in ib if e not in sa]))
            self.children.append((a, b))
            self.node.append(frozenset(ia) | frozenset(ib))
            self.parent[a] = v
            self.parent[b] = v
        self.root = self.n_leaves + len(path) - 1
        if set(self.idx[self.root]) != set(self.open):
            raise ValueError("result indices differ from the open indices")

    @property
    def n_tensors(self):
        return len(self.idx)

    def all_indices(self):
        return sorted(self.dims)

    # Eq. 1 term of a node and subtree costs
    def node_cost(self, i, sliced=frozenset()):
        return 1 << sum(self.logd[e] for e in self.node[i] if e not in sliced)

    def eq1(self):
        """Eq. 1: sum over contraction nodes of prod_{e in s_V} w(e)."""
        return sum(self.node_cost(i) for i in range(len(self.node)))

    def eq3(self, sliced):
        """Eq. 3: sum_V 2^{|s_V| + |S| - |S cap s_V|} (w-weighted)."""
        sl = frozenset(sliced)
        mult = 1 << sum(self.logd[e] for e in sl)
        return mult * sum(self.node_cost(i, sl) for i in range(len(self.node)))

    def overhead(self, sliced):
        """Eq. 2: C_slice * 2^|S| / C_original."""
        return self.eq3(sliced) / self.eq1()

    def dim(self, v, sliced):
        return sum(self.logd[e] for e in self.idx[v] if e not in sliced)

    def size_log(self, v):
        return sum(self.logd[e] for e in self.idx[v])

    def satisfies(self, sliced, t):
        sl = frozenset(sliced)
        return all(self.dim(v, sl) <= t for v in range(self.n_tensors))

    def lifetime(self, e):
        """Definition 1: the tree tensors whose index set contains e (ascending)."""
        return [v for v in range(self.n_tensors) if e in self.idx[v]]

    def correlated_contractions(self, e):
        """Supplementary Def.: the contraction nodes whose index set contains e."""
        return [self.n_leaves + i for i in range(len(self.node)) if e in self.node[i]]

    def subtree_cost(self):
        cost = [0] * self.n_tensors
        for i, (a, b) in enumerate(self.children):
            cost[self.n_leaves + i] = cost[a] + cost[b] + self.node_cost(i)
        return cost

    def stem(self):
        """Stem tensors from the bottom leaf (M[0]) to the root output (M[-1])."""
        cost = self.subtree_cost()
        v = self.root
        out = [v]
        while v >= self.n_leaves:
            a, b = self.children[v - self.n_leaves]
            ka = (cost[a], self.size_log(a), -a)
            kb = (cost[b], self.size_log(b), -b)
            v = a if ka > kb else b
            out.append(v)
        out.reverse()
        return out


# --------------------------------------------------------------------------
# Algorithm 1: slice finder
# --------------------------------------------------------------------------

class Infeasible(ValueError):
    pass


def _sliceable(tree, e, sliced):
    return e not in sliced and e not in tree.open and tree.dims[e] == 2


def slice_finder(tree, t):
    """Algorithm 1 on the stem, then the global fix-up. Returns S in insertion order."""
    S = []
    Sset = set()
    M = list(tree.stem())
    while M:
        d0, d1 = tree.dim(M[0], Sset), tree.dim(M[-1], Sset)
        sT = M[0] if d0 < d1 else M[-1]
        if tree.dim(sT, Sset) > t:
            life = {}
            for v in M:
                for e in tree.idx[v]:
                    life[e] = life.get(e, 0) + 1
            cands = [e for e in tree.idx[sT] if _sliceable(tree, e, Sset)]
            cands.sort(key=lambda e: (-life[e], e))
            for e in cands:
                if tree.dim(sT, Sset) <= t:
                    break
                S.append(e)
                Sset.add(e)
            if tree.dim(sT, Sset) > t:
                raise Infeasible("target dim infeasible on the stem")
        M = [v for v in M if tree.dim(v, Sset) > t]
    glife = {}
    for v in range(tree.n_tensors):
        for e in tree.idx[v]:
            glife[e] = glife.get(e, 0) + 1
    for v in range(tree.n_tensors):
        while tree.dim(v, Sset) > t:
            cands = [e for e in tree.idx[v] if _sliceable(tree, e, Sset)]
            if not cands:
                raise Infeasible("target dim infeasible")
            cands.sort(key=lambda e: (-glife[e], e))
            S.append(cands[0])
            Sset.add(cands[0])
    return S


# --------------------------------------------------------------------------
# Algorithms 2-4: simulated-annealing refiner
# --------------------------------------------------------------------------

def find_critical_tensors(tree, lf, t, sliced):
    """Algorithm 3: the tensors of a lifetime whose dim equals t."""
    return [v for v in lf if tree.dim(v, sliced) == t]


def find_candidate_indices(tree, c_tensors):
    """Algorithm 4: intersection of the index sets of the critical tensors."""
    cand = set(tree.idx[c_tensors[0]])
    for v in c_tensors:
        cand &= set(tree.idx[v])
    return cand


def slice_refiner(tree, t, S0, seed, T0=1.0, Tf=1e-4, alpha=0.9, trace=None):
    """Algorithm 2. Returns the best slicing set seen (insertion order kept).

    ``trace`` (a list), if given, receives every slicing set that becomes
    current, so tests can check the constraint after every move."""
    rng = SplitMix64(seed)
    S = list(S0)
    C = tree.eq3(S)
    best, bestC = list(S), C
    lf = {e: tree.lifetime(e) for e in tree.all_indices()}
    T = float(T0)
    while True:
        if not S:
            break
        ss = sorted(S)
        r = rng.next()
        index = ss[(r * len(ss)) >> 64]
        Sset = set(S)
        c_tensors = find_critical_tensors(tree, lf[index], t, Sset)
        if not c_tensors:
            S.remove(index)
            C = tree.eq3(S)
            if trace is not None:
                trace.append(list(S))
            if C < bestC:
                best, bestC = list(S), C
        else:
            cand = find_candidate_indices(tree, c_tensors)
            cand = sorted(e for e in cand if _sliceable(tree, e, Sset))
            cur = index
            for can in cand:
                pos = S.index(cur)
                S_new = list(S)
                S_new[pos] = can
                Cn = tree.eq3(S_new)
                if Cn < C:
                    accept = True
                else:
                    u = (rng.next() >> 11) * (2.0 ** -53)
                    p = math.exp((float(C) - float(Cn)) / float(C) / T)
                    accept = u < p
                if accept:
                    S, C, cur = S_new, Cn, can
                    if trace is not None:
                        trace.append(list(S))
                    if C < bestC:
                        best, bestC = list(S), C
        T = T * alpha
        if T < Tf:
            break
    return best


def find_slices(tree, t, seed, T0=1.0, Tf=1e-4, alpha=0.9):
    """Algorithm 1 followed by Algorithm 2."""
    S1 = slice_finder(tree, t)
    return slice_refiner(tree, t, S1, seed, T0, Tf, alpha)
