// KD cluster tree and block partition on the host (Section 3.1, Table 1;
// KD-tree ordering of Section 4.2 and Section 4.4).
//
// Rules: every box of a level is split while the largest box of that level
// exceeds the leaf size, so that all leaves share one depth; the split
// coordinate is the longer side of the box's bounding box (ties to the first
// coordinate); points are ordered by (coordinate, original index) and the
// first floor(|t|/2) form child 0.  Admissibility: WEAK admits every t != s;
// STRONG(eta) admits t != s with max(diam t, diam s) <= eta * dist(t, s) on
// axis-aligned bounding boxes.  The block tree recurses from (root, root);
// admissible pairs are far blocks, inadmissible leaf pairs near blocks.
#include "tree.h"

#include <algorithm>
#include <cmath>
#include <string>
#include <tuple>

#include "common.h"

namespace {

double norm_of(const double* v, int dim) {
    double s = 0.0;
    for (int d = 0; d < dim; ++d) {
        const double x = v[d] * v[d];
        s = s + x;
    }
    return std::sqrt(s);
}

}  // namespace

bool h2_tree_s::admissible(int level, int t, int s) const {
    if (t == s) return false;
    if (adm == H2_ADM_WEAK) return true;
    const double* lt = &lo[level][(size_t)t * dim];
    const double* ht = &hi[level][(size_t)t * dim];
    const double* ls = &lo[level][(size_t)s * dim];
    const double* hs = &hi[level][(size_t)s * dim];
    double et[3], es[3], gap[3];
    for (int d = 0; d < dim; ++d) {
        et[d] = ht[d] - lt[d];
        es[d] = hs[d] - ls[d];
        const double g1 = ls[d] - ht[d], g2 = lt[d] - hs[d];
        gap[d] = std::max(0.0, std::max(g1, g2));
    }
    const double dist = norm_of(gap, dim);
    const double diam = std::max(norm_of(et, dim), norm_of(es, dim));
    return diam <= eta * dist;
}

namespace h2 {

h2_tree_s* make_tree(const double* coords, int64_t N, int dim, int leaf, int adm, double eta) {
    if (!coords || N < 1 || dim < 1 || dim > 3 || leaf < 2)
        fail(H2_ERR_INVALID_ARG, "h2_tree_create: need coords, n >= 1, 1 <= dim <= 3, leaf >= 2");
    if (N > (int64_t)1 << 30) fail(H2_ERR_INVALID_ARG, "h2_tree_create: n too large");
    if (adm != H2_ADM_WEAK && adm != H2_ADM_STRONG) fail(H2_ERR_INVALID_ARG, "h2_tree_create: bad adm");
    if (adm == H2_ADM_STRONG && !(eta > 0.0 && std::isfinite(eta)))
        fail(H2_ERR_INVALID_ARG, "h2_tree_create: eta must be positive");
    for (int64_t i = 0; i < N * dim; ++i)
        if (!std::isfinite(coords[i])) fail(H2_ERR_INVALID_ARG, "h2_tree_create: non-finite coordinate");
    auto* t = new h2_tree_s();
    try {
        t->N = N;
        t->dim = dim;
        t->leaf = leaf;
        t->adm = adm;
        t->eta = eta;
        int L = 0;
        while ((N + ((int64_t)1 << L) - 1) >> L > leaf) ++L;
        if (L > H2_MAX_LEVELS - 1) fail(H2_ERR_INVALID_ARG, "h2_tree_create: tree too deep");
        t->L = L;
        t->perm.resize(N);
        for (int64_t i = 0; i < N; ++i) t->perm[i] = i;
        t->start.assign(L + 1, {});
        t->size.assign(L + 1, {});
        t->start[0] = {0};
        t->size[0] = {N};
        std::vector<double> key;
        for (int l = 0; l < L; ++l) {
            const size_t nb = t->start[l].size();
            t->start[l + 1].resize(2 * nb);
            t->size[l + 1].resize(2 * nb);
            for (size_t b = 0; b < nb; ++b) {
                const int64_t a = t->start[l][b], m = t->size[l][b];
                int64_t* idx = t->perm.data() + a;
                double lo3[3], hi3[3];
                for (int d = 0; d < dim; ++d) {
                    lo3[d] = INFINITY;
                    hi3[d] = -INFINITY;
                }
                for (int64_t i = 0; i < m; ++i)
                    for (int d = 0; d < dim; ++d) {
                        const double x = coords[idx[i] * dim + d];
                        lo3[d] = std::min(lo3[d], x);
                        hi3[d] = std::max(hi3[d], x);
                    }
                int sd = 0;
                double best = hi3[0] - lo3[0];
                for (int d = 1; d < dim; ++d) {
                    const double e = hi3[d] - lo3[d];
                    if (e > best) {
                        best = e;
                        sd = d;
                    }
                }
                std::sort(idx, idx + m, [&](int64_t p, int64_t q) {
                    const double xp = coords[p * dim + sd], xq = coords[q * dim + sd];
                    if (xp != xq) return xp < xq;
                    return p < q;
                });
                const int64_t h = m / 2;
                t->start[l + 1][2 * b] = a;
                t->size[l + 1][2 * b] = h;
                t->start[l + 1][2 * b + 1] = a + h;
                t->size[l + 1][2 * b + 1] = m - h;
            }
        }
        t->lo.assign(L + 1, {});
        t->hi.assign(L + 1, {});
        for (int l = 0; l <= L; ++l) {
            const size_t nb = t->start[l].size();
            t->lo[l].resize(nb * dim);
            t->hi[l].resize(nb * dim);
            for (size_t b = 0; b < nb; ++b) {
                for (int d = 0; d < dim; ++d) {
                    double mn = INFINITY, mx = -INFINITY;
                    for (int64_t i = 0; i < t->size[l][b]; ++i) {
                        const double x = coords[t->perm[t->start[l][b] + i] * dim + d];
                        mn = std::min(mn, x);
                        mx = std::max(mx, x);
                    }
                    t->lo[l][b * dim + d] = mn;
                    t->hi[l][b * dim + d] = mx;
                }
            }
        }
        int lm = 0;
        for (int64_t s : t->size[L]) lm = std::max<int>(lm, (int)s);
        t->leaf_max = lm;
        // block tree
        t->far.assign(L + 1, {});
        std::vector<std::tuple<int, int, int>> stack{{0, 0, 0}};
        while (!stack.empty()) {
            auto [l, a, b] = stack.back();
            stack.pop_back();
            if (t->admissible(l, a, b)) {
                t->far[l].push_back({a, b});
            } else if (l == L) {
                t->near.push_back({a, b});
            } else {
                for (int ca = 2 * a; ca <= 2 * a + 1; ++ca)
                    for (int cb = 2 * b; cb <= 2 * b + 1; ++cb) stack.push_back({l + 1, ca, cb});
            }
        }
        for (auto& f : t->far) std::sort(f.begin(), f.end());
        std::sort(t->near.begin(), t->near.end());
    } catch (...) {
        delete t;
        throw;
    }
    return t;
}

}  // namespace h2
