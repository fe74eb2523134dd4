// Conforming refinement of marked cells for the adaptive loop (Section 7 of arXiv:1708.03912:
// meshes refined without hanging nodes).  Host code.
//
// 1D: a marked interval (a, b) becomes (a, m), (m, b), m its midpoint.
// 2D: newest-vertex bisection.  A triangle (v0, v1, v2) has newest vertex v0 and refinement
// edge {v1, v2}; bisection at the midpoint m of that edge gives (m, v0, v1) and (m, v2, v0)
// (the orientation is kept).  The set of edges to halve is closed before any cell is split:
// it starts with the refinement edges of the marked cells, and whenever an edge enters it the
// refinement edges of the (at most two) cells on that edge enter too (a worklist over an
// edge -> cells table), so no edge is halved on one side only.  Then every cell whose
// refinement edge is halved is bisected, and each child once more if its own refinement edge
// (an edge of the parent) is halved; a cell ends as 1, 2, 3 or 4 cells.  The closure is the
// smallest one that contains the marked cells' edges, so the mesh does not depend on the order
// in which the cells are listed.
// Output numbering: the old vertices keep their ids, the midpoints follow in the order in
// which the cells are split (cells in input order; in a cell the refinement edge's midpoint
// first, then those of its first and second child); every cell is replaced in place by its
// children, first child's subtree first.
#include <algorithm>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "context.h"

namespace fl {

int refine_mesh(int dim, int64_t nv, const double* V, int64_t nc, const int32_t* C, const uint8_t* marks,
                int64_t cap_v, int64_t cap_c, double* V_out, int32_t* C_out, int64_t* nv_out, int64_t* nc_out,
                std::string& err) {
    if (dim != 1 && dim != 2) { err = "dim must be 1 or 2"; return FL_EINVAL; }
    if (nv < 1 || nc < 1 || !V || !C || !marks || !nv_out || !nc_out) {
        err = "empty mesh or NULL pointer";
        return FL_EINVAL;
    }
    const int nvpc = dim + 1;
    for (int64_t i = 0; i < nc * nvpc; ++i)
        if (C[i] < 0 || C[i] >= nv) { err = "cell vertex index out of range"; return FL_EINVAL; }
    if (dim == 1) {
        int64_t nm = 0;
        for (int64_t K = 0; K < nc; ++K) nm += marks[K] != 0;
        *nv_out = nv + nm;
        *nc_out = nc + nm;
        if (cap_v < nv + nm || cap_c < nc + nm || !V_out || !C_out) {
            err = "output capacity too small (sizes needed are in *n_vertices_out, *n_cells_out)";
            return FL_EINVAL;
        }
        std::memcpy(V_out, V, sizeof(double) * nv);
        int64_t v = nv, c = 0;
        for (int64_t K = 0; K < nc; ++K) {
            const int32_t a = C[2 * K], b = C[2 * K + 1];
            if (marks[K]) {
                V_out[v] = (V[a] + V[b]) / 2.0;
                C_out[2 * c] = a;
                C_out[2 * c + 1] = (int32_t)v;
                C_out[2 * c + 2] = (int32_t)v;
                C_out[2 * c + 3] = b;
                ++v;
                c += 2;
            } else {
                C_out[2 * c] = a;
                C_out[2 * c + 1] = b;
                ++c;
            }
        }
        return FL_OK;
    }
    // edges of the mesh: id per sorted vertex pair; per cell its three edges (v1v2 first)
    std::unordered_map<int64_t, int32_t> eid;
    eid.reserve((size_t)(3 * nc));
    std::vector<int32_t> cedge(3 * nc);
    std::vector<int32_t> e_a, e_b;
    auto key = [&](int32_t a, int32_t b) { return (int64_t)std::min(a, b) * nv + std::max(a, b); };
    for (int64_t K = 0; K < nc; ++K) {
        const int32_t* t = C + 3 * K;
        const int32_t pairs[3][2] = {{t[1], t[2]}, {t[0], t[1]}, {t[2], t[0]}};
        for (int j = 0; j < 3; ++j) {
            const int64_t k = key(pairs[j][0], pairs[j][1]);
            auto it = eid.find(k);
            if (it == eid.end()) {
                it = eid.emplace(k, (int32_t)e_a.size()).first;
                e_a.push_back(std::min(pairs[j][0], pairs[j][1]));
                e_b.push_back(std::max(pairs[j][0], pairs[j][1]));
            }
            cedge[3 * K + j] = it->second;
        }
    }
    const int64_t ne = (int64_t)e_a.size();
    // edge -> cells
    std::vector<int32_t> ptr(ne + 1, 0), adj(3 * nc);
    for (int64_t i = 0; i < 3 * nc; ++i) ++ptr[cedge[i] + 1];
    for (int64_t e = 0; e < ne; ++e) ptr[e + 1] += ptr[e];
    {
        std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t i = 0; i < 3 * nc; ++i) adj[fill[cedge[i]]++] = (int32_t)(i / 3);
    }
    for (int64_t e = 0; e < ne; ++e)
        if (ptr[e + 1] - ptr[e] > 2) { err = "non-conforming mesh: an edge in more than two cells"; return FL_EINVAL; }
    // closure of the set of halved edges
    std::vector<uint8_t> half(ne, 0);
    std::vector<int32_t> work;
    for (int64_t K = 0; K < nc; ++K)
        if (marks[K] && !half[cedge[3 * K]]) {
            half[cedge[3 * K]] = 1;
            work.push_back(cedge[3 * K]);
        }
    while (!work.empty()) {
        const int32_t e = work.back();
        work.pop_back();
        for (int32_t q = ptr[e]; q < ptr[e + 1]; ++q) {
            const int32_t r = cedge[3 * adj[q]];
            if (!half[r]) {
                half[r] = 1;
                work.push_back(r);
            }
        }
    }
    // sizes: one midpoint per halved edge; a cell with j halved edges becomes j + 1 cells
    int64_t nh = 0, ncells = 0;
    for (int64_t e = 0; e < ne; ++e) nh += half[e];
    for (int64_t K = 0; K < nc; ++K) ncells += 1 + half[cedge[3 * K]] + half[cedge[3 * K + 1]] + half[cedge[3 * K + 2]];
    *nv_out = nv + nh;
    *nc_out = ncells;
    if (cap_v < nv + nh || cap_c < ncells || !V_out || !C_out) {
        err = "output capacity too small (sizes needed are in *n_vertices_out, *n_cells_out)";
        return FL_EINVAL;
    }
    std::memcpy(V_out, V, sizeof(double) * 2 * nv);
    std::vector<int32_t> mid(ne, -1);
    int64_t v = nv, c = 0;
    auto midpoint = [&](int32_t e) {
        if (mid[e] < 0) {
            const int32_t a = e_a[e], b = e_b[e];
            V_out[2 * v] = (V[2 * a] + V[2 * b]) / 2.0;
            V_out[2 * v + 1] = (V[2 * a + 1] + V[2 * b + 1]) / 2.0;
            mid[e] = (int32_t)v++;
        }
        return mid[e];
    };
    auto emit = [&](int32_t a, int32_t b, int32_t d) {
        C_out[3 * c] = a;
        C_out[3 * c + 1] = b;
        C_out[3 * c + 2] = d;
        ++c;
    };
    for (int64_t K = 0; K < nc; ++K) {
        const int32_t v0 = C[3 * K], v1 = C[3 * K + 1], v2 = C[3 * K + 2];
        if (!half[cedge[3 * K]]) {
            emit(v0, v1, v2);
            continue;
        }
        const int32_t m = midpoint(cedge[3 * K]);
        // first child (m, v0, v1): refinement edge v0v1
        const int32_t e01 = cedge[3 * K + 1], e20 = cedge[3 * K + 2];
        if (half[e01]) {
            const int32_t m1 = midpoint(e01);
            emit(m1, m, v0);
            emit(m1, v1, m);
        } else {
            emit(m, v0, v1);
        }
        // second child (m, v2, v0): refinement edge v2v0
        if (half[e20]) {
            const int32_t m2 = midpoint(e20);
            emit(m2, m, v2);
            emit(m2, v0, m);
        } else {
            emit(m, v2, v0);
        }
    }
    return FL_OK;
}

}  // namespace fl
