// Host planner of the cluster method (Section 6 of arXiv:1708.03912, after Sauter and
// Schwab, Ch. 7): the hierarchical cluster tree over the degrees of freedom and the
// partition of the DOF pairs into admissible cluster pairs (far field, approximated by
// Chebyshev interpolation of the kernel) and inadmissible leaf pairs (near field, exact
// entries).  Pure host code, deterministic.
//
// Construction (the paper leaves these choices open):
//   * a cluster with more than `leaf` DOFs is split in two by the coordinate of its DOF
//     vertices along the longest side of their bounding box (ties: the lowest axis), at the
//     middle of that side: DOFs strictly below go to the first son, in their current order;
//     should a son be empty, the DOFs sorted by (coordinate, index) are split at the median;
//   * the cluster box is the smallest hyper-cube containing the supports of the cluster's
//     basis functions (the cells around their vertices), centred on their bounding box;
//     diameter = side sqrt(d), distance = the distance of the two cubes;
//   * (sigma, tau) is admissible when eta dist(sigma, tau) >= max(diam sigma, diam tau); the
//     partition is the recursion over pairs from (root, root) that keeps admissible pairs,
//     keeps pairs of leaves as near field, and otherwise replaces the non-leaf members of the
//     pair by their sons (both when neither is a leaf).
// Nodes are numbered in creation order (depth first, first son first); a node's DOFs are a
// contiguous range of the tree-order permutation.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "cluster.h"

namespace fl {

int build_cluster_plan(const Plan& P, double eta, int leaf, ClusterPlan& C) {
    if (leaf < 1 || !(eta >= 0.0)) return FL_EINVAL;
    const int d = P.dim, nvpc = P.nvpc;
    const int64_t n = P.n;
    C = ClusterPlan();
    C.dim = d;
    C.eta = eta;
    C.leaf = leaf;
    C.n = n;
    // support box of every DOF
    std::vector<double> lo(n * d), hi(n * d), X(n * d);
    for (int64_t i = 0; i < n; ++i) {
        const int v = P.vod[i];
        for (int k = 0; k < d; ++k) {
            X[i * d + k] = P.V[(int64_t)v * d + k];
            lo[i * d + k] = INFINITY;
            hi[i * d + k] = -INFINITY;
        }
        for (int q = P.v2c_ptr[v]; q < P.v2c_ptr[v + 1]; ++q) {
            const int K = P.v2c[q];
            for (int a = 0; a < nvpc; ++a) {
                const int w = P.C[(int64_t)K * nvpc + a];
                for (int k = 0; k < d; ++k) {
                    const double x = P.V[(int64_t)w * d + k];
                    lo[i * d + k] = std::min(lo[i * d + k], x);
                    hi[i * d + k] = std::max(hi[i * d + k], x);
                }
            }
        }
    }
    C.perm.resize(n);
    std::iota(C.perm.begin(), C.perm.end(), 0);
    // explicit stack: (range, level, parent slot to fill), children created first son first
    struct Item {
        int64_t lo, hi;
        int level, parent, which;
    };
    std::vector<Item> stack;
    stack.push_back({0, n, 0, -1, 0});
    std::vector<int> tmp;
    while (!stack.empty()) {
        const Item it = stack.back();
        stack.pop_back();
        const int c = (int)C.lo.size();
        if (it.parent >= 0) C.son[2 * it.parent + it.which] = c;
        C.lo.push_back((int)it.lo);
        C.hi.push_back((int)it.hi);
        C.son.push_back(-1);
        C.son.push_back(-1);
        C.level.push_back(it.level);
        double blo[2] = {INFINITY, INFINITY}, bhi[2] = {-INFINITY, -INFINITY};
        for (int64_t p = it.lo; p < it.hi; ++p) {
            const int i = C.perm[p];
            for (int k = 0; k < d; ++k) {
                blo[k] = std::min(blo[k], lo[(int64_t)i * d + k]);
                bhi[k] = std::max(bhi[k], hi[(int64_t)i * d + k]);
            }
        }
        double side = 0.0;
        for (int k = 0; k < d; ++k) {
            C.center.push_back((blo[k] + bhi[k]) / 2.0);
            side = std::max(side, bhi[k] - blo[k]);
        }
        C.side.push_back(side);
        C.depth = std::max(C.depth, it.level);
        if (it.hi - it.lo <= leaf) continue;
        // split axis and middle of the DOF vertices' bounding box
        double vlo[2] = {INFINITY, INFINITY}, vhi[2] = {-INFINITY, -INFINITY};
        for (int64_t p = it.lo; p < it.hi; ++p)
            for (int k = 0; k < d; ++k) {
                vlo[k] = std::min(vlo[k], X[(int64_t)C.perm[p] * d + k]);
                vhi[k] = std::max(vhi[k], X[(int64_t)C.perm[p] * d + k]);
            }
        int ax = 0;
        for (int k = 1; k < d; ++k)
            if (vhi[k] - vlo[k] > vhi[ax] - vlo[ax]) ax = k;
        const double mid = (vlo[ax] + vhi[ax]) / 2.0;
        tmp.clear();
        int64_t nfirst = 0;
        for (int64_t p = it.lo; p < it.hi; ++p)
            if (X[(int64_t)C.perm[p] * d + ax] < mid) tmp.push_back(C.perm[p]), ++nfirst;
        for (int64_t p = it.lo; p < it.hi; ++p)
            if (!(X[(int64_t)C.perm[p] * d + ax] < mid)) tmp.push_back(C.perm[p]);
        if (nfirst == 0 || nfirst == it.hi - it.lo) {
            std::sort(tmp.begin(), tmp.end(), [&](int a, int b) {
                const double xa = X[(int64_t)a * d + ax], xb = X[(int64_t)b * d + ax];
                return xa < xb || (xa == xb && a < b);
            });
            nfirst = (it.hi - it.lo) / 2;
        }
        std::copy(tmp.begin(), tmp.end(), C.perm.begin() + it.lo);
        // the second son is pushed first so that the first son is created (numbered) first
        stack.push_back({it.lo + nfirst, it.hi, it.level + 1, c, 1});
        stack.push_back({it.lo, it.lo + nfirst, it.level + 1, c, 0});
    }
    const int nn = (int)C.lo.size();
    C.nodes = nn;
    // block partition by the recursion over pairs, in the recursion's order
    const double sqd = std::sqrt((double)d);
    auto diam = [&](int a) { return C.side[a] * sqd; };
    auto dist = [&](int a, int b) {
        double acc = 0.0;
        for (int k = 0; k < d; ++k) {
            const double g = std::max(0.0, std::fabs(C.center[(int64_t)a * d + k] - C.center[(int64_t)b * d + k]) -
                                               (C.side[a] + C.side[b]) / 2.0);
            acc += g * g;
        }
        return std::sqrt(acc);
    };
    auto is_leaf = [&](int a) { return C.son[2 * a] < 0; };
    std::vector<std::pair<int, int>> st;
    st.push_back({0, 0});
    while (!st.empty()) {
        const auto pr = st.back();
        st.pop_back();
        const int a = pr.first, b = pr.second;
        if (eta * dist(a, b) >= std::max(diam(a), diam(b))) {
            C.far.push_back(a);
            C.far.push_back(b);
        } else if (is_leaf(a) && is_leaf(b)) {
            C.near.push_back(a);
            C.near.push_back(b);
        } else {
            // children in reverse so that the stack visits them in the recursion's order
            std::vector<std::pair<int, int>> kids;
            if (is_leaf(a)) {
                for (int q = 0; q < 2; ++q) kids.push_back({a, C.son[2 * b + q]});
            } else if (is_leaf(b)) {
                for (int q = 0; q < 2; ++q) kids.push_back({C.son[2 * a + q], b});
            } else {
                for (int q = 0; q < 2; ++q)
                    for (int r = 0; r < 2; ++r) kids.push_back({C.son[2 * a + q], C.son[2 * b + r]});
            }
            for (auto k = kids.rbegin(); k != kids.rend(); ++k) st.push_back(*k);
        }
    }
    return FL_OK;
}

}  // namespace fl
