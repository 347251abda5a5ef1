// Host-side planner of libtnc: greedy contraction path, contraction-tree
// bookkeeping, Eq. 1/2/3 costs, lifetimes (Definition 1), the stem, the slice
// finder (Algorithm 1) and the simulated-annealing refiner (Algorithm 2 with
// Algorithms 3 and 4) of Liu et al., Sec. 2.1.1, 3.1, 4.1-4.3, Suppl. S3.
#pragma once

#include <cstdint>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

namespace tnc {

// Unsigned integer of 320 bits: Eq. 3 costs are sums of powers of two whose
// exponents exceed 128 on large trees, and they are compared exactly.
struct Wide {
    static constexpr int W = 5;
    uint64_t w[W] = {0, 0, 0, 0, 0};
    void add_pow2(int e);                 // += 2^e
    void add(const Wide& o);
    Wide shl(int s) const;                // * 2^s
    bool operator<(const Wide& o) const;
    bool operator==(const Wide& o) const;
    int bit_length() const;
    double to_double() const;             // correctly rounded, ties to even
    std::string to_string() const;        // decimal
};

struct PlanError : std::runtime_error {
    explicit PlanError(const std::string& m) : std::runtime_error(m) {}
};

using Pair = std::pair<int, int>;

// Greedy SSA path over leaves given as index-id lists; logd[e] = log2 w(e).
std::vector<Pair> greedy_path(const std::vector<std::vector<int64_t>>& leaves,
                              const std::vector<int>& logd);

class Tree {
public:
    Tree(const std::vector<std::vector<int64_t>>& leaves, const std::vector<int>& logd,
         const std::vector<int64_t>& open_ids, const std::vector<Pair>& path);

    int n_leaves = 0;
    int root = 0;
    std::vector<std::vector<int64_t>> idx;   // index ids of every tree tensor
    std::vector<Pair> children;              // per contraction node
    std::vector<std::vector<int64_t>> node;  // s_V per contraction node (sorted)
    std::vector<int> parent;                 // per tree tensor, -1 at the root
    std::vector<int> logd;                   // by index id
    std::vector<char> is_open;               // by index id
    std::vector<char> in_net;                // index id appears in the network

    int n_tensors() const { return (int)idx.size(); }
    int size_log(int v) const;
    int dim(int v, const std::vector<char>& sliced) const;
    Wide node_cost(int i, const std::vector<char>& sliced) const;
    Wide eq1() const;
    Wide eq3(const std::vector<int64_t>& S) const;
    std::vector<Wide> subtree_cost() const;
    std::vector<int> stem() const;
    std::vector<int> lifetime(int64_t e) const;
    bool satisfies(const std::vector<int64_t>& S, int t) const;
    bool sliceable(int64_t e, const std::vector<char>& sliced) const;
};

std::vector<int64_t> slice_finder(const Tree& tree, int t);
std::vector<int64_t> slice_refiner(const Tree& tree, int t, const std::vector<int64_t>& S0,
                                   uint64_t seed, double T0, double Tf, double alpha);

struct SplitMix64 {
    uint64_t state;
    explicit SplitMix64(uint64_t s) : state(s) {}
    uint64_t next() {
        state += 0x9E3779B97F4A7C15ull;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
};

}  // namespace tnc
