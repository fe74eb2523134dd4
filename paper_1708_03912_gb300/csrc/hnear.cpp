// Host planner of the cluster method's near field assembled directly (Section 6 of
// arXiv:1708.03912: the inadmissible pairs are assembled into a sparse matrix by local
// computations).  Pure host code, deterministic.
//
// A near-field entry (i, j) is the stiffness-matrix entry a(phi_i, phi_j).  Its terms are
//   * the separated pairs at vertex-graph distance >= 2 of a cell of supp phi_i and one of
//     supp phi_j (off-diagonal blocks): they lie in the tiles (I, J) of the element blocks
//     holding the two DOFs, so only the tiles that some near-field entry touches are
//     computed: the product of the block sets of every inadmissible leaf pair;
//   * the touching, near and identical pairs and the diagonal blocks, which the dense
//     assembly's contribution slots already hold per entry, except that the part of a
//     diagonal block that sums over all far cells and the boundary term become, for x in K,
//     C/(2s) times the integral over the boundary of N(K) of n.(x - y) |x - y|^{-d-2s}, with
//     N(K) the union of K, its touching cells and the cells at vertex-graph distance 1 and n
//     pointing into N(K) (divergence theorem: that integral is 2s times the integral of the
//     kernel outside N(K), which is the far cells plus the complement of Omega).
// This file lists the tiles and, per cell, the facets of the boundary of N(K) with their
// classes; the device part is in assemble.cu (assemble_hnear).
#include <algorithm>
#include <cmath>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cluster.h"

namespace fl {
namespace {

int hw_threads() { return (int)std::max(1u, std::min(std::thread::hardware_concurrency(), 32u)); }

template <typename Fn>
void run_threads(int nthr, Fn fn) {
    std::vector<std::thread> th;
    for (int t = 1; t < nthr; ++t) th.emplace_back(fn, t);
    fn(0);
    for (auto& x : th) x.join();
}

// fn(lo, hi) over contiguous ranges of [0, n), one per thread
template <typename Fn>
void parallel_ranges(int64_t n, Fn fn) {
    const int nthr = hw_threads();
    const int64_t chunk = (n + nthr - 1) / nthr;
    run_threads(nthr, [&](int t) {
        const int64_t lo = (int64_t)t * chunk, hi = std::min(n, lo + chunk);
        if (lo < hi) fn(lo, hi);
    });
}

}  // namespace

int plan_hnear(const Plan& P, const ClusterPlan& C, HNearPlan& Q, std::string& err) {
    Q = HNearPlan();
    const int d = P.dim, m = P.nvpc;
    const int64_t nc = P.nc, nv = P.nv, nf = P.nf, nblk = P.nblk;
    if (C.n != P.n) {
        err = "cluster plan and mesh plan disagree";
        return FL_EINVAL;
    }
    // ---- tiles: the element blocks of every leaf's DOFs, crossed over the inadmissible pairs
    std::vector<std::vector<int>> leaf_blk(C.nodes);
    std::vector<char> need(C.nodes, 0);
    for (size_t b = 0; b < C.near.size(); ++b) need[C.near[b]] = 1;
    for (int a = 0; a < C.nodes; ++a) {
        if (!need[a]) continue;
        std::vector<int>& L = leaf_blk[a];
        for (int p = C.lo[a]; p < C.hi[a]; ++p) {
            const int i = C.perm[p];
            for (int q = P.occ_ptr[i]; q < P.occ_ptr[i + 1]; ++q) L.push_back(P.occ_blk[q]);
        }
        std::sort(L.begin(), L.end());
        L.erase(std::unique(L.begin(), L.end()), L.end());
    }
    std::vector<std::vector<int>> rows(nblk);
    for (size_t b = 0; b + 1 < C.near.size(); b += 2) {
        const std::vector<int>& A = leaf_blk[C.near[b]];
        const std::vector<int>& B = leaf_blk[C.near[b + 1]];
        for (int I : A)
            for (int J : B) rows[std::min(I, J)].push_back(std::max(I, J));
    }
    parallel_ranges(nblk, [&](int64_t lo, int64_t hi) {
        for (int64_t I = lo; I < hi; ++I) {
            std::vector<int>& r = rows[I];
            std::sort(r.begin(), r.end());
            r.erase(std::unique(r.begin(), r.end()), r.end());
        }
    });
    Q.trow_ptr.assign(nblk + 1, 0);
    Q.toff.assign(1, 0);
    for (int64_t I = 0; I < nblk; ++I) {
        std::vector<int>& r = rows[I];
        const int64_t nI = P.L_ptr[I + 1] - P.L_ptr[I];
        for (int J : r) {
            Q.tiles.push_back((int)I);
            Q.tiles.push_back(J);
            Q.toff.push_back(Q.toff.back() + nI * (P.L_ptr[J + 1] - P.L_ptr[J]));
        }
        Q.trow_ptr[I + 1] = (int)(Q.tiles.size() / 2);
        std::vector<int>().swap(r);
    }
    // ---- per tile, the row cells of block I that pair with some cell of block J in a near-field
    // entry (a DOF of one in a leaf, a DOF of the other in a leaf near-paired with it); the far
    // kernel skips the other rows, whose contributions no near-field entry reads
    {
        std::vector<int> lidx(C.nodes, -1);
        int nl = 0;
        for (int a = 0; a < C.nodes; ++a)
            if (C.son[2 * a] < 0) lidx[a] = nl++;
        const int64_t words = (nl + 63) / 64;
        std::vector<uint64_t> adj((size_t)nl * words, 0);
        for (size_t b = 0; b + 1 < C.near.size(); b += 2) {
            const int a = lidx[C.near[b]], c = lidx[C.near[b + 1]];
            adj[(size_t)a * words + c / 64] |= 1ull << (c % 64);
        }
        std::vector<int> dof_leaf(P.n, -1);
        for (int a = 0; a < C.nodes; ++a)
            if (lidx[a] >= 0)
                for (int p = C.lo[a]; p < C.hi[a]; ++p) dof_leaf[C.perm[p]] = lidx[a];
        // leaves of each internal cell's DOFs (up to nvpc, -1 padded)
        std::vector<int> cl((size_t)nc * m, -1);
        for (int64_t k = 0; k < nc; ++k)
            for (int a = 0; a < m; ++a) {
                const int i = P.cdof[k * m + a];
                cl[k * m + a] = i >= 0 ? dof_leaf[i] : -1;
            }
        const int64_t nt = (int64_t)Q.tiles.size() / 2;
        Q.rowmask.assign(nt, 0u);
        // leaves of every block's cells
        std::vector<int> bl_ptr(nblk + 1, 0), bl;
        {
            std::vector<int> U;
            for (int64_t J = 0; J < nblk; ++J) {
                U.clear();
                for (int64_t k = J * TILE; k < std::min(nc, (J + 1) * TILE); ++k)
                    for (int a = 0; a < m; ++a)
                        if (cl[k * m + a] >= 0) U.push_back(cl[k * m + a]);
                std::sort(U.begin(), U.end());
                U.erase(std::unique(U.begin(), U.end()), U.end());
                bl.insert(bl.end(), U.begin(), U.end());
                bl_ptr[J + 1] = (int)bl.size();
            }
        }
        parallel_ranges(nt, [&](int64_t t0, int64_t t1) {
            for (int64_t t = t0; t < t1; ++t) {
                const int I = Q.tiles[2 * t], J = Q.tiles[2 * t + 1];
                uint32_t mask = 0;
                for (int kk = 0; kk < TILE; ++kk) {
                    const int64_t k = (int64_t)I * TILE + kk;
                    if (k >= nc) break;
                    bool need = false;
                    for (int a = 0; a < m && !need; ++a) {
                        const int la = cl[k * m + a];
                        if (la < 0) continue;
                        const uint64_t* row = &adj[(size_t)la * words];
                        for (int q = bl_ptr[J]; q < bl_ptr[J + 1]; ++q) {
                            const int lb = bl[q];
                            if ((row[lb / 64] >> (lb % 64)) & 1ull) {
                                need = true;
                                break;
                            }
                        }
                    }
                    if (need) mask |= 1u << kk;
                }
                Q.rowmask[t] = mask;
            }
        });
    }
    // ---- facet table: the boundary facets of Omega (ids 0 .. nf-1, as in the mesh plan), then
    // one oriented copy per (internal cell M, facet e of M) with the normal pointing into M
    const int64_t ntab = nf + (int64_t)m * nc;
    Q.F.assign(ntab * d, -1);
    Q.FN.assign(ntab * d, 0.0);
    Q.FLEN.assign(ntab, 0.0);
    std::copy(P.F.begin(), P.F.end(), Q.F.begin());
    std::copy(P.FN.begin(), P.FN.end(), Q.FN.begin());
    std::copy(P.FLEN.begin(), P.FLEN.end(), Q.FLEN.begin());
    std::unordered_map<uint64_t, int> bfac;  // boundary facet by its (sorted) vertices
    for (int64_t f = 0; f < nf; ++f) {
        const uint64_t key = d == 1 ? (uint64_t)P.F[f]
                                    : ((uint64_t)P.F[2 * f] << 32) | (uint32_t)P.F[2 * f + 1];
        bfac.emplace(key, (int)f);
    }
    // per (internal cell, facet): the neighbouring internal cell across it (-1: none), and the
    // facet id to use when it bounds N(K)
    std::vector<int> nbc(m * nc, -1), fid(m * nc, -1);
    for (int64_t M = 0; M < nc; ++M) {
        const int Ko = P.perm[M];
        const int* c = &P.C[(int64_t)Ko * m];
        for (int e = 0; e < m; ++e) {
            int va, vb, vr;  // facet vertices (1D: va = vb) and the cell's other vertex
            if (d == 1) {
                va = vb = c[e];
                vr = c[1 - e];
            } else {
                va = std::min(c[e], c[(e + 1) % 3]);
                vb = std::max(c[e], c[(e + 1) % 3]);
                vr = c[(e + 2) % 3];
            }
            int other = -1;
            for (int q = P.v2c_ptr[va]; q < P.v2c_ptr[va + 1] && other < 0; ++q) {
                const int K2 = P.v2c[q];
                if (K2 == Ko) continue;
                const int* c2 = &P.C[(int64_t)K2 * m];
                bool hasb = false;
                for (int x = 0; x < m; ++x) hasb = hasb || c2[x] == vb;
                if (hasb) other = K2;
            }
            const int64_t slot = (int64_t)m * M + e;
            if (other >= 0) {
                nbc[slot] = P.iperm[other];
                const int64_t f = nf + slot;
                fid[slot] = (int)f;
                if (d == 1) {
                    Q.F[f] = va;
                    Q.FN[f] = P.V[vr] > P.V[va] ? 1.0 : -1.0;
                    Q.FLEN[f] = 1.0;
                } else {
                    const double tx = P.V[2 * vb] - P.V[2 * va], ty = P.V[2 * vb + 1] - P.V[2 * va + 1];
                    const double L = std::hypot(tx, ty);
                    double nx = -ty / L, ny = tx / L;
                    if (nx * (P.V[2 * vr] - P.V[2 * va]) + ny * (P.V[2 * vr + 1] - P.V[2 * va + 1]) < 0) {
                        nx = -nx;
                        ny = -ny;
                    }
                    Q.F[2 * f] = va;
                    Q.F[2 * f + 1] = vb;
                    Q.FN[2 * f] = nx;
                    Q.FN[2 * f + 1] = ny;
                    Q.FLEN[f] = L;
                }
            } else {
                const uint64_t key = d == 1 ? (uint64_t)va : ((uint64_t)va << 32) | (uint32_t)vb;
                auto it = bfac.find(key);
                if (it == bfac.end()) {
                    err = "a facet with one cell is not a boundary facet";
                    return FL_EINVAL;
                }
                fid[slot] = it->second;
            }
        }
    }
    // ---- per cell with DOFs: the facets of the boundary of N(K) and their classes
    // (2 / 3: shares two / one vertex with K, only boundary facets of Omega can; 1: a vertex
    // is a mesh neighbour of a vertex of K; 0: the rest)
    // in parallel over ranges of cells; the ranges' lists are concatenated in cell order
    const int nthr = hw_threads();
    const int64_t chunk = (nc + nthr - 1) / nthr;
    struct Part {
        std::vector<int> cnt, fac, cls;
        std::string err;
    };
    std::vector<Part> parts(nthr);
    auto work = [&](int th) {
        Part& o = parts[th];
        const int64_t k0 = (int64_t)th * chunk, k1 = std::min(nc, k0 + chunk);
        if (k0 >= k1) return;
        std::vector<int64_t> mark0(nv, -1), mark1(nv, -1);
        std::vector<std::pair<int, int>> lst;
        for (int64_t k = k0; k < k1; ++k) {
            int c0 = 0;
            if (P.hasdof[k]) {
                const int Ko = P.perm[k];
                const int* c = &P.C[(int64_t)Ko * m];
                for (int a = 0; a < m; ++a) {
                    mark0[c[a]] = k;
                    mark1[c[a]] = k;
                    for (int q = P.nbr_ptr[c[a]]; q < P.nbr_ptr[c[a] + 1]; ++q) mark1[P.nbr[q]] = k;
                }
                const int* N0 = &P.ex_idx[P.ex_ptr[k]];
                const int* N1 = &P.ex_idx[P.ex_ptr[k + 1]];
                lst.clear();
                for (const int* it = N0; it != N1; ++it) {
                    const int M = *it;
                    for (int e = 0; e < m; ++e) {
                        const int64_t slot = (int64_t)m * M + e;
                        const int ob = nbc[slot];
                        if (ob >= 0 && std::binary_search(N0, N1, ob)) continue;  // inside N(K)
                        const int f = fid[slot];
                        int sh = 0, n1 = 0;
                        for (int x = 0; x < d; ++x) {
                            const int v = Q.F[(int64_t)f * d + x];
                            sh += mark0[v] == k;
                            n1 += mark1[v] == k;
                        }
                        int cls;
                        if (sh > 0) {
                            if (ob >= 0) {
                                o.err = "internal: a facet inside Omega touches K on the boundary of N(K)";
                                return;
                            }
                            cls = (d == 1 || sh == 2) ? 2 : 3;
                        } else {
                            cls = n1 > 0 ? 1 : 0;
                        }
                        lst.push_back({f, cls});
                    }
                }
                std::sort(lst.begin(), lst.end());
                for (const auto& pr : lst) {
                    o.fac.push_back(pr.first);
                    o.cls.push_back(pr.second);
                }
                c0 = (int)lst.size();
            }
            o.cnt.push_back(c0);
        }
    };
    run_threads(nthr, work);
    for (const Part& o : parts)
        if (!o.err.empty()) {
            err = o.err;
            return FL_EINVAL;
        }
    Q.ef_ptr.assign(nc + 1, 0);
    {
        int64_t k = 0;
        for (const Part& o : parts)
            for (int c : o.cnt) {
                Q.ef_ptr[k + 1] = Q.ef_ptr[k] + c;
                ++k;
            }
    }
    Q.ef_fac.reserve(Q.ef_ptr[nc]);
    Q.ef_cls.reserve(Q.ef_ptr[nc]);
    for (const Part& o : parts) {
        Q.ef_fac.insert(Q.ef_fac.end(), o.fac.begin(), o.fac.end());
        Q.ef_cls.insert(Q.ef_cls.end(), o.cls.begin(), o.cls.end());
    }
    return FL_OK;
}

}  // namespace fl
