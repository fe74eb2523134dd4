// Symmetry reduction, host part (Section 7 of arXiv:1708.03912, "Exploiting Symmetry").
//
// Omega and the data are invariant under the rotation B by 2 pi / K.  The caller meshes the
// sector {0 <= phi <= 2 pi / K}; the whole mesh is its K rotated copies with the vertices on
// the cut rays (and the centre) merged.  The reduced problem is the Galerkin problem on the
// periodic subspace: one unknown per orbit {B^l v} of DOFs.  With exact integrals the whole
// matrix A is rotation invariant, so P^T A P / K (P the DOF-orbit incidence) has entries
// (|O_r| / K) sum_{j in O_c} A[rep_r, j]: only the rows of one representative per orbit are
// needed, i.e. the element pairs with a cell in a representative's support, about N^2 / K of
// the N^2 / 2 pairs of the whole mesh.  The tile list is cut down to the tiles that touch such
// a cell; compose writes the representatives' rows, and the fold takes the symmetric part of
// the row formula (the touching-pair quadrature is rotation invariant only to its own error).
//
// Numbering (shared with the planner's other parts): whole vertices in order of first
// appearance over (copy, sector vertex), cells copy by copy; an orbit is represented by the
// lowest sector vertex among its copy-0 vertices, orbits numbered by that vertex, ascending.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace fl {

void replicate_sector(int64_t nv, const double* V, int64_t nc, const int32_t* C, int K, std::vector<double>& W,
                      std::vector<int32_t>& CW, std::vector<int>& vmap) {
    const double tol = 1e-10, cell = 1e-9;
    W.clear();
    vmap.assign((size_t)K * nv, -1);
    // hash grid of cell size 1e-9 >= tol: a match lies in the 3 x 3 neighbourhood
    std::unordered_map<uint64_t, std::vector<int>> grid;
    auto key = [](int64_t a, int64_t b) { return (uint64_t)(a * 2654435761LL) ^ (uint64_t)(b * 40503LL + 0x9e3779b9LL); };
    for (int l = 0; l < K; ++l) {
        const double c = std::cos(2.0 * M_PI * l / K), s = std::sin(2.0 * M_PI * l / K);
        for (int64_t v = 0; v < nv; ++v) {
            const double x = c * V[2 * v] - s * V[2 * v + 1];
            const double y = s * V[2 * v] + c * V[2 * v + 1];
            const int64_t gx = (int64_t)std::floor(x / cell), gy = (int64_t)std::floor(y / cell);
            int hit = -1;
            for (int64_t a = gx - 1; a <= gx + 1; ++a)
                for (int64_t b = gy - 1; b <= gy + 1; ++b) {
                    auto it = grid.find(key(a, b));
                    if (it == grid.end()) continue;
                    for (int w : it->second)
                        if (std::fabs(W[2 * w] - x) <= tol && std::fabs(W[2 * w + 1] - y) <= tol &&
                            (hit < 0 || w < hit))
                            hit = w;
                }
            if (hit < 0) {
                hit = (int)(W.size() / 2);
                W.push_back(x);
                W.push_back(y);
                grid[key(gx, gy)].push_back(hit);
            }
            vmap[(size_t)l * nv + v] = hit;
        }
    }
    CW.resize((size_t)K * nc * 3);
    for (int l = 0; l < K; ++l)
        for (int64_t k = 0; k < nc * 3; ++k) CW[(size_t)l * nc * 3 + k] = vmap[(size_t)l * nv + C[k]];
}

int plan_symmetry(Plan& P, int K, int64_t nvs, const std::vector<int>& vmap, std::string& err) {
    if (P.dim != 2 || K < 2) {
        err = "symmetry reduction: 2D, K >= 2";
        return FL_EINVAL;
    }
    // sector vertex whose copy-0 image is a given whole vertex
    std::vector<int> inv0(P.nv, -1);
    for (int64_t v = 0; v < nvs; ++v) inv0[vmap[v]] = (int)v;
    // orbit key of every whole vertex
    std::vector<int> key_of(P.nv, -1);
    for (int64_t v = 0; v < nvs; ++v) {
        int key = INT32_MAX;
        for (int l = 0; l < K; ++l) {
            const int u = inv0[vmap[(size_t)l * nvs + v]];
            if (u >= 0) key = std::min(key, u);
        }
        for (int l = 0; l < K; ++l) key_of[vmap[(size_t)l * nvs + v]] = key;
    }
    for (int64_t w = 0; w < P.nv; ++w)
        if (key_of[w] < 0 || key_of[w] == INT32_MAX) {
            err = "symmetry reduction: a vertex outside every orbit (not a rotated sector mesh?)";
            return FL_EINVAL;
        }
    // orbits of DOFs, numbered by key
    std::vector<int> keys;
    for (int64_t i = 0; i < P.n; ++i) keys.push_back(key_of[P.vod[i]]);
    std::vector<int> sorted_keys(keys);
    std::sort(sorted_keys.begin(), sorted_keys.end());
    sorted_keys.erase(std::unique(sorted_keys.begin(), sorted_keys.end()), sorted_keys.end());
    P.sym_K = K;
    P.n_red = (int64_t)sorted_keys.size();
    P.red_vertex = sorted_keys;
    std::vector<int> rank(nvs, -1);
    for (size_t r = 0; r < sorted_keys.size(); ++r) rank[sorted_keys[r]] = (int)r;
    std::vector<std::vector<int>> mem(P.n_red);
    for (int64_t i = 0; i < P.n; ++i) mem[rank[keys[i]]].push_back((int)i);
    P.red_ptr.assign(P.n_red + 1, 0);
    P.red_mem.clear();
    for (int64_t r = 0; r < P.n_red; ++r) {
        P.red_mem.insert(P.red_mem.end(), mem[r].begin(), mem[r].end());
        P.red_ptr[r + 1] = (int)P.red_mem.size();
    }
    P.red_rep.assign(P.n_red, -1);
    P.red_row.assign(P.n, -1);
    for (int64_t r = 0; r < P.n_red; ++r) {
        const int i = P.dov[vmap[sorted_keys[r]]];  // copy 0 of the representing sector vertex
        if (i < 0) {
            err = "symmetry reduction: an orbit's representative is not a DOF";
            return FL_EINVAL;
        }
        P.red_rep[r] = i;
        P.red_row[i] = (int)r;
    }
    // cells in the supports of the representatives, and the blocks that hold one
    std::vector<char> rowblk(P.nblk, 0);
    for (int64_t r = 0; r < P.n_red; ++r) {
        const int v = P.vod[P.red_rep[r]];
        for (int q = P.v2c_ptr[v]; q < P.v2c_ptr[v + 1]; ++q) rowblk[P.iperm[P.v2c[q]] / TILE] = 1;
    }
    // tiles touching such a block; positions of the kept tiles by upper-triangle index
    std::vector<int> tiles;
    std::vector<int64_t> toff(1, 0);
    P.tri_list.assign(P.nblk * (P.nblk + 1) / 2, -1);
    int64_t t = 0;
    for (int64_t I = 0; I < P.nblk; ++I)
        for (int64_t J = I; J < P.nblk; ++J, ++t) {
            if (!rowblk[I] && !rowblk[J]) continue;
            P.tri_list[t] = (int64_t)(tiles.size() / 2);
            tiles.push_back((int)I);
            tiles.push_back((int)J);
            const int64_t nI = P.L_ptr[I + 1] - P.L_ptr[I], nJ = P.L_ptr[J + 1] - P.L_ptr[J];
            toff.push_back(toff.back() + nI * nJ);
        }
    P.tiles.swap(tiles);
    P.toff.swap(toff);
    return FL_OK;
}

}  // namespace fl
