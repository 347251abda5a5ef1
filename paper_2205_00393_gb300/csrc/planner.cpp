// Host-side planner of libtnc (see planner.hpp for the paper passages).
//
// Readings where the paper is silent (all deterministic, so that two
// independent implementations agree bit for bit):
//  * T.dim = sum of log2 w(e) over the unsliced indices of T.
//  * Stem (Sec. 4.2, "most computationally intensive path"): from the root,
//    descend into the child with the larger subtree Eq. 1 cost (ties: larger
//    output size, then smaller SSA id) down to a leaf. M[0] is that leaf,
//    M[N-1] the root output.
//  * Algorithm 1: the selection line is taken literally (the end with the
//    smaller dim; M[N-1] on a tie). Candidates are the unsliced closed
//    dimension-2 indices of sT ordered by lifetime length within the current
//    M (longest first), then by id; every tensor of M with dim <= t is pruned.
//    A global fix-up then slices, for each tree tensor still above t (in SSA
//    order), its candidate with the longest lifetime over the whole tree.
//  * Algorithm 2: splitmix64; index = S_sorted[(r*|S|) >> 64]; the uniform
//    draw u = (r >> 11) * 2^-53 is taken only when C_new >= C_ori; candidates
//    (Algorithm 4 result minus S, closed, dimension 2) ascending; each
//    candidate replaces the current occupant of the slot; an index whose
//    lifetime holds no critical tensor is dropped; T *= alpha after each outer
//    iteration until T < Tf; the best set seen (first on ties) is returned.
//  * Eq. 3 sums over all contraction nodes of the tree.
#include "planner.hpp"

#include <algorithm>
#include <cmath>
#include <map>
#include <queue>
#include <set>
#include <tuple>

namespace tnc {

// ---------------------------------------------------------------- Wide ----

void Wide::add_pow2(int e) {
    if (e < 0 || e >= 64 * W - 16) throw PlanError("cost exponent out of range");
    int i = e / 64;
    uint64_t v = 1ull << (e % 64);
    while (i < W) {
        uint64_t before = w[i];
        w[i] += v;
        if (w[i] >= before) return;
        v = 1;
        ++i;
    }
    throw PlanError("cost overflow");
}

void Wide::add(const Wide& o) {
    unsigned __int128 carry = 0;
    for (int i = 0; i < W; ++i) {
        unsigned __int128 s = (unsigned __int128)w[i] + o.w[i] + carry;
        w[i] = (uint64_t)s;
        carry = s >> 64;
    }
    if (carry) throw PlanError("cost overflow");
}

Wide Wide::shl(int s) const {
    Wide r;
    if (s < 0) throw PlanError("negative shift");
    int q = s / 64, b = s % 64;
    for (int i = W - 1; i >= 0; --i) {
        int src = i - q;
        if (src < 0) continue;
        uint64_t v = w[src] << b;
        if (b && src - 1 >= 0) v |= w[src - 1] >> (64 - b);
        r.w[i] = v;
    }
    // overflow check: bits shifted out
    if (bit_length() + s > 64 * W) throw PlanError("cost overflow");
    return r;
}

bool Wide::operator<(const Wide& o) const {
    for (int i = W - 1; i >= 0; --i)
        if (w[i] != o.w[i]) return w[i] < o.w[i];
    return false;
}

bool Wide::operator==(const Wide& o) const {
    for (int i = 0; i < W; ++i)
        if (w[i] != o.w[i]) return false;
    return true;
}

int Wide::bit_length() const {
    for (int i = W - 1; i >= 0; --i)
        if (w[i]) return 64 * i + 64 - __builtin_clzll(w[i]);
    return 0;
}

static int wide_bit(const Wide& x, int b) { return (int)((x.w[b / 64] >> (b % 64)) & 1); }

double Wide::to_double() const {
    int n = bit_length();
    if (n == 0) return 0.0;
    if (n <= 53) {
        uint64_t v = w[0];
        return (double)v;  // exact
    }
    // top 53 bits
    uint64_t mant = 0;
    for (int b = n - 1; b >= n - 53; --b) mant = (mant << 1) | (uint64_t)wide_bit(*this, b);
    int round = wide_bit(*this, n - 54);
    bool sticky = false;
    for (int b = n - 55; b >= 0 && !sticky; --b) sticky = wide_bit(*this, b);
    int exp = n - 53;
    if (round && (sticky || (mant & 1))) {
        ++mant;
        if (mant == (1ull << 53)) {
            mant >>= 1;
            ++exp;
        }
    }
    return std::ldexp((double)mant, exp);
}

std::string Wide::to_string() const {
    Wide x = *this;
    std::string out;
    auto is_zero = [](const Wide& v) {
        for (int i = 0; i < W; ++i)
            if (v.w[i]) return false;
        return true;
    };
    if (is_zero(x)) return "0";
    const uint64_t base = 1000000000000000000ull;  // 1e18
    std::vector<uint64_t> chunks;
    while (!is_zero(x)) {
        unsigned __int128 rem = 0;
        for (int i = W - 1; i >= 0; --i) {
            unsigned __int128 cur = (rem << 64) | x.w[i];
            x.w[i] = (uint64_t)(cur / base);
            rem = cur % base;
        }
        chunks.push_back((uint64_t)rem);
    }
    out = std::to_string(chunks.back());
    for (int i = (int)chunks.size() - 2; i >= 0; --i) {
        std::string s = std::to_string(chunks[i]);
        out += std::string(18 - s.size(), '0') + s;
    }
    return out;
}

// ------------------------------------------------------- greedy path -----

std::vector<Pair> greedy_path(const std::vector<std::vector<int64_t>>& leaves,
                              const std::vector<int>& logd) {
    const int n = (int)leaves.size();
    std::map<int, std::vector<int64_t>> live;
    std::vector<std::vector<int>> owners(logd.size());
    for (int i = 0; i < n; ++i) {
        live[i] = leaves[i];
        for (int64_t e : leaves[i]) owners[e].push_back(i);
    }
    int nxt = n;
    std::vector<Pair> path;

    auto neighbours = [&](int i) {
        std::set<int> out;
        for (int64_t e : live.at(i))
            for (int o : owners[e])
                if (o != i) out.insert(o);
        return out;
    };
    auto remove_owner = [&](int64_t e, int who) {
        auto& v = owners[e];
        v.erase(std::remove(v.begin(), v.end(), who), v.end());
    };
    auto do_contract = [&](int a, int b) {
        std::vector<int64_t> ia = live.at(a), ib = live.at(b);
        live.erase(a);
        live.erase(b);
        std::set<int64_t> sa(ia.begin(), ia.end()), sb(ib.begin(), ib.end());
        std::vector<int64_t> nw;
        for (int64_t e : ia)
            if (!sb.count(e)) nw.push_back(e);
        for (int64_t e : ib)
            if (!sa.count(e)) nw.push_back(e);
        for (int64_t e : ia) remove_owner(e, a);
        for (int64_t e : ib) remove_owner(e, b);
        for (int64_t e : nw) owners[e].push_back(nxt);
        live[nxt] = nw;
        path.emplace_back(std::min(a, b), std::max(a, b));
        return nxt++;
    };

    // phase 1: rank-1 / rank-2 absorption
    for (;;) {
        int t = -1;
        for (auto& kv : live) {
            if (kv.second.size() <= 2 && !neighbours(kv.first).empty()) {
                t = kv.first;
                break;
            }
        }
        if (t < 0) break;
        auto nb = neighbours(t);
        int best = -1;
        size_t best_rank = 0;
        for (int j : nb) {  // ascending ids: first max rank wins ties
            size_t r = live.at(j).size();
            if (best < 0 || r > best_rank) {
                best = j;
                best_rank = r;
            }
        }
        do_contract(t, best);
    }

    // phase 2: greedy on size(out) - size(a) - size(b)
    auto size_log = [&](const std::vector<int64_t>& idx) {
        int s = 0;
        for (int64_t e : idx) s += logd[e];
        return s;
    };
    using Key = std::tuple<__int128, int, int>;
    auto pair_key = [&](int a, int b) {
        const auto& ia = live.at(a);
        const auto& ib = live.at(b);
        std::set<int64_t> sa(ia.begin(), ia.end()), sb(ib.begin(), ib.end());
        int so = 0;
        for (int64_t e : ia)
            if (!sb.count(e)) so += logd[e];
        for (int64_t e : ib)
            if (!sa.count(e)) so += logd[e];
        int s1 = size_log(ia), s2 = size_log(ib);
        if (so > 125 || s1 > 125 || s2 > 125) throw PlanError("tensor too large for the greedy planner");
        __int128 cost = ((__int128)1 << so) - ((__int128)1 << s1) - ((__int128)1 << s2);
        return Key(cost, std::min(a, b), std::max(a, b));
    };
    std::priority_queue<Key, std::vector<Key>, std::greater<Key>> heap;
    for (auto& kv : live)
        for (int b : neighbours(kv.first))
            if (kv.first < b) heap.push(pair_key(kv.first, b));
    while (!heap.empty()) {
        Key k = heap.top();
        heap.pop();
        int a = std::get<1>(k), b = std::get<2>(k);
        if (!live.count(a) || !live.count(b)) continue;
        int c = do_contract(a, b);
        for (int j : neighbours(c)) heap.push(pair_key(c, j));
    }

    // phase 3: disconnected remainders in ascending id order
    while (live.size() > 1) {
        auto it = live.begin();
        int a = it->first;
        ++it;
        int b = it->first;
        do_contract(a, b);
    }
    return path;
}

// -------------------------------------------------------------- Tree -----

Tree::Tree(const std::vector<std::vector<int64_t>>& leaves, const std::vector<int>& logd_,
           const std::vector<int64_t>& open_ids, const std::vector<Pair>& path)
    : logd(logd_) {
    n_leaves = (int)leaves.size();
    is_open.assign(logd.size(), 0);
    in_net.assign(logd.size(), 0);
    for (int64_t e : open_ids) is_open[e] = 1;
    idx = leaves;
    for (auto& l : leaves)
        for (int64_t e : l) in_net[e] = 1;
    if ((int)path.size() != n_leaves - 1) throw PlanError("path must have n_tensors - 1 steps");
    parent.assign(n_leaves + path.size(), -1);
    std::vector<char> used(n_leaves + path.size(), 0);
    for (size_t i = 0; i < path.size(); ++i) {
        int a = path[i].first, b = path[i].second;
        int v = n_leaves + (int)i;
        if (a == b || a < 0 || b < 0 || a >= v || b >= v || used[a] || used[b])
            throw PlanError("invalid SSA path at step " + std::to_string(i));
        used[a] = used[b] = 1;
        const auto ia = idx[a];
        const auto ib = idx[b];
        std::set<int64_t> sa(ia.begin(), ia.end()), sb(ib.begin(), ib.end());
        std::vector<int64_t> out;
        for (int64_t e : ia)
            if (!sb.count(e)) out.push_back(e);
        for (int64_t e : ib)
            if (!sa.count(e)) out.push_back(e);
        idx.push_back(out);
        std::set<int64_t> un(sa);
        un.insert(sb.begin(), sb.end());
        node.emplace_back(un.begin(), un.end());
        children.emplace_back(a, b);
        parent[a] = parent[b] = v;
    }
    root = n_leaves + (int)path.size() - 1;
    std::set<int64_t> ro(idx[root].begin(), idx[root].end());
    std::set<int64_t> op(open_ids.begin(), open_ids.end());
    if (ro != op) throw PlanError("result indices differ from the open indices");
}

int Tree::size_log(int v) const {
    int s = 0;
    for (int64_t e : idx[v]) s += logd[e];
    return s;
}

int Tree::dim(int v, const std::vector<char>& sliced) const {
    int s = 0;
    for (int64_t e : idx[v])
        if (!sliced[e]) s += logd[e];
    return s;
}

Wide Tree::node_cost(int i, const std::vector<char>& sliced) const {
    int s = 0;
    for (int64_t e : node[i])
        if (!sliced[e]) s += logd[e];
    Wide r;
    r.add_pow2(s);
    return r;
}

Wide Tree::eq1() const {
    std::vector<char> none(logd.size(), 0);
    Wide r;
    for (size_t i = 0; i < node.size(); ++i) r.add(node_cost((int)i, none));
    return r;
}

Wide Tree::eq3(const std::vector<int64_t>& S) const {
    std::vector<char> sl(logd.size(), 0);
    int m = 0;
    for (int64_t e : S) {
        sl[e] = 1;
        m += logd[e];
    }
    Wide r;
    for (size_t i = 0; i < node.size(); ++i) r.add(node_cost((int)i, sl));
    return r.shl(m);
}

std::vector<Wide> Tree::subtree_cost() const {
    std::vector<char> none(logd.size(), 0);
    std::vector<Wide> c(idx.size());
    for (size_t i = 0; i < children.size(); ++i) {
        Wide w = c[children[i].first];
        w.add(c[children[i].second]);
        w.add(node_cost((int)i, none));
        c[n_leaves + i] = w;
    }
    return c;
}

std::vector<int> Tree::stem() const {
    auto cost = subtree_cost();
    int v = root;
    std::vector<int> out{v};
    while (v >= n_leaves) {
        int a = children[v - n_leaves].first, b = children[v - n_leaves].second;
        // compare (cost, size_log, -id)
        bool a_gt;
        if (!(cost[a] == cost[b])) a_gt = cost[b] < cost[a];
        else if (size_log(a) != size_log(b)) a_gt = size_log(a) > size_log(b);
        else a_gt = a < b;
        v = a_gt ? a : b;
        out.push_back(v);
    }
    std::reverse(out.begin(), out.end());
    return out;
}

std::vector<int> Tree::lifetime(int64_t e) const {
    std::vector<int> out;
    for (int v = 0; v < n_tensors(); ++v)
        for (int64_t x : idx[v])
            if (x == e) {
                out.push_back(v);
                break;
            }
    return out;
}

bool Tree::satisfies(const std::vector<int64_t>& S, int t) const {
    std::vector<char> sl(logd.size(), 0);
    for (int64_t e : S) sl[e] = 1;
    for (int v = 0; v < n_tensors(); ++v)
        if (dim(v, sl) > t) return false;
    return true;
}

bool Tree::sliceable(int64_t e, const std::vector<char>& sliced) const {
    return !sliced[e] && !is_open[e] && logd[e] == 1;
}

// -------------------------------------------------------- Algorithm 1 ----

std::vector<int64_t> slice_finder(const Tree& tree, int t) {
    std::vector<int64_t> S;
    std::vector<char> sl(tree.logd.size(), 0);
    std::vector<int> M = tree.stem();
    while (!M.empty()) {
        int d0 = tree.dim(M.front(), sl), d1 = tree.dim(M.back(), sl);
        int sT = d0 < d1 ? M.front() : M.back();
        if (tree.dim(sT, sl) > t) {
            std::map<int64_t, int> life;
            for (int v : M)
                for (int64_t e : tree.idx[v]) life[e] += 1;
            std::vector<int64_t> cands;
            for (int64_t e : tree.idx[sT])
                if (tree.sliceable(e, sl)) cands.push_back(e);
            std::sort(cands.begin(), cands.end(), [&](int64_t x, int64_t y) {
                if (life[x] != life[y]) return life[x] > life[y];
                return x < y;
            });
            for (int64_t e : cands) {
                if (tree.dim(sT, sl) <= t) break;
                S.push_back(e);
                sl[e] = 1;
            }
            if (tree.dim(sT, sl) > t) throw PlanError("target dim infeasible on the stem");
        }
        std::vector<int> keep;
        for (int v : M)
            if (tree.dim(v, sl) > t) keep.push_back(v);
        M.swap(keep);
    }
    std::vector<int> glife(tree.logd.size(), 0);
    for (int v = 0; v < tree.n_tensors(); ++v)
        for (int64_t e : tree.idx[v]) glife[e] += 1;
    for (int v = 0; v < tree.n_tensors(); ++v) {
        while (tree.dim(v, sl) > t) {
            int64_t best = -1;
            for (int64_t e : tree.idx[v]) {
                if (!tree.sliceable(e, sl)) continue;
                if (best < 0 || glife[e] > glife[best] || (glife[e] == glife[best] && e < best))
                    best = e;
            }
            if (best < 0) throw PlanError("target dim infeasible");
            S.push_back(best);
            sl[best] = 1;
        }
    }
    return S;
}

// ------------------------------------------------ Algorithms 2, 3, 4 -----

std::vector<int64_t> slice_refiner(const Tree& tree, int t, const std::vector<int64_t>& S0,
                                   uint64_t seed, double T0, double Tf, double alpha) {
    SplitMix64 rng(seed);
    std::vector<int64_t> S = S0;
    Wide C = tree.eq3(S);
    std::vector<int64_t> best = S;
    Wide bestC = C;
    std::map<int64_t, std::vector<int>> lf;
    double T = T0;
    for (;;) {
        if (S.empty()) break;
        std::vector<int64_t> ss = S;
        std::sort(ss.begin(), ss.end());
        uint64_t r = rng.next();
        int64_t index = ss[(size_t)(((unsigned __int128)r * ss.size()) >> 64)];
        std::vector<char> sl(tree.logd.size(), 0);
        for (int64_t e : S) sl[e] = 1;
        auto it = lf.find(index);
        if (it == lf.end()) it = lf.emplace(index, tree.lifetime(index)).first;
        // Algorithm 3: critical tensors of the lifetime
        std::vector<int> crit;
        for (int v : it->second)
            if (tree.dim(v, sl) == t) crit.push_back(v);
        if (crit.empty()) {
            S.erase(std::find(S.begin(), S.end(), index));
            C = tree.eq3(S);
            if (C < bestC) {
                best = S;
                bestC = C;
            }
        } else {
            // Algorithm 4: intersection of the critical tensors' index sets
            std::set<int64_t> cand(tree.idx[crit[0]].begin(), tree.idx[crit[0]].end());
            for (int v : crit) {
                std::set<int64_t> sv(tree.idx[v].begin(), tree.idx[v].end()), nx;
                for (int64_t e : cand)
                    if (sv.count(e)) nx.insert(e);
                cand.swap(nx);
            }
            std::vector<int64_t> cl;
            for (int64_t e : cand)
                if (tree.sliceable(e, sl)) cl.push_back(e);  // std::set iterates ascending
            int64_t cur = index;
            for (int64_t can : cl) {
                size_t pos = std::find(S.begin(), S.end(), cur) - S.begin();
                std::vector<int64_t> Sn = S;
                Sn[pos] = can;
                Wide Cn = tree.eq3(Sn);
                bool accept;
                if (Cn < C) {
                    accept = true;
                } else {
                    double u = (double)(rng.next() >> 11) * 0x1.0p-53;
                    double fc = C.to_double(), fn = Cn.to_double();
                    double p = std::exp((fc - fn) / fc / T);
                    accept = u < p;
                }
                if (accept) {
                    S = Sn;
                    C = Cn;
                    cur = can;
                    if (C < bestC) {
                        best = S;
                        bestC = C;
                    }
                }
            }
        }
        T = T * alpha;
        if (T < Tf) break;
    }
    return best;
}

}  // namespace tnc
