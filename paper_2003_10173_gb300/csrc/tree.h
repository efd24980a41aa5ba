// Cluster tree and block partition (host data).
#pragma once

#include <stdint.h>

#include <utility>
#include <vector>

struct h2_tree_s {
    int64_t N = 0;
    int dim = 0;
    int leaf = 0;
    int L = 0;                                       // leaves at level L
    int adm = 0;
    double eta = 0.0;
    std::vector<int64_t> perm;                       // tree position -> original index
    std::vector<std::vector<int64_t>> start, size;   // [level][box]
    std::vector<std::vector<double>> lo, hi;         // [level][box*dim + d]
    std::vector<std::vector<std::pair<int, int>>> far;  // [level] (t, s), both triangles, sorted
    std::vector<std::pair<int, int>> near;           // leaf level, both triangles, sorted
    int leaf_max = 0;
    bool admissible(int level, int t, int s) const;
};

namespace h2 {
// Level of the sibling pair that contains block (t, s) of `level`: one below
// the lowest common ancestor of t and s.
inline int pair_level(int level, int t, int s) {
    while (t != s) {
        t >>= 1;
        s >>= 1;
        --level;
    }
    return level + 1;
}
}  // namespace h2
