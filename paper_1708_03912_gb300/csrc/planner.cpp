// Host planner: mesh ingest, boundary facets, degrees of freedom, combinatorial
// classes of element pairs, quadrature tables and the maps that let every device
// reduction run in a fixed order.
//
// Paper references (arXiv:1708.03912): mesh, facets dP_h and DOF set I_h -- Section 3;
// element-pair decomposition a^{KxK'} + a^{Kxe} -- Section 5; Gauss-type rules of
// class-dependent order -- Appendix B (orders fixed per class here).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>
#include <unordered_map>

#include "internal.h"

namespace fl {

// Gauss-Legendre nodes/weights on [0,1] (ascending nodes): Newton iteration on the
// three-term recurrence of the Legendre polynomials, in long double.
void gauss01(int k, std::vector<double>& x, std::vector<double>& w) {
    x.assign(k, 0.0);
    w.assign(k, 0.0);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < k; ++i) {
        long double z = std::cos(pi * (i + 0.75L) / (k + 0.5L));
        long double p0 = 1, p1 = z, dp = 1;
        for (int it = 0; it < 200; ++it) {
            p0 = 1;
            p1 = z;
            for (int j = 2; j <= k; ++j) {
                long double p2 = ((2 * j - 1) * z * p1 - (j - 1) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = k * (z * p1 - p0) / (z * z - 1);
            long double dz = p1 / dp;
            z -= dz;
            if (std::fabs((double)dz) < 1e-19) break;
        }
        p0 = 1;
        p1 = z;
        for (int j = 2; j <= k; ++j) {
            long double p2 = ((2 * j - 1) * z * p1 - (j - 1) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        dp = k * (z * p1 - p0) / (z * z - 1);
        // z_i decreases with i; store ascending on [0,1]
        x[k - 1 - i] = (double)((1 + z) / 2);
        w[k - 1 - i] = (double)(1 / ((1 - z * z) * dp * dp));
    }
}

// 1D: Gauss on [0,1].  2D: collapsed (Duffy) product rule on the reference triangle
// {l1, l2 >= 0, l1 + l2 <= 1}: l1 = t_a, l2 = t_b (1 - t_a), weight w_a w_b (1 - t_a),
// points a-major.
Rule make_rule(int dim, int k) {
    Rule r;
    r.k = k;
    std::vector<double> t, w;
    gauss01(k, t, w);
    if (dim == 1) {
        r.q = k;
        for (int a = 0; a < k; ++a) {
            r.lam.push_back(t[a]);
            r.w.push_back(w[a]);
            r.phi.push_back(1 - t[a]);
            r.phi.push_back(t[a]);
        }
    } else {
        r.q = k * k;
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b) {
                double l1 = t[a], l2 = t[b] * (1 - t[a]);
                r.lam.push_back(l1);
                r.lam.push_back(l2);
                r.w.push_back(w[a] * w[b] * (1 - t[a]));
                r.phi.push_back(1 - l1 - l2);
                r.phi.push_back(l1);
                r.phi.push_back(l2);
            }
    }
    return r;
}

static void csr_from_lists(const std::vector<std::vector<int>>& L, std::vector<int>& ptr, std::vector<int>& ent) {
    ptr.assign(L.size() + 1, 0);
    for (size_t i = 0; i < L.size(); ++i) ptr[i + 1] = ptr[i] + (int)L[i].size();
    ent.resize(ptr.back());
    for (size_t i = 0; i < L.size(); ++i) std::copy(L[i].begin(), L[i].end(), ent.begin() + ptr[i]);
}

static uint32_t spread16(uint32_t x) {
    x &= 0xffff;
    x = (x | (x << 8)) & 0x00ff00ff;
    x = (x | (x << 4)) & 0x0f0f0f0f;
    x = (x | (x << 2)) & 0x33333333;
    x = (x | (x << 1)) & 0x55555555;
    return x;
}

int plan_mesh(Plan& P, int dim, int64_t nv, const double* V, int64_t nc, const int32_t* C, std::string& err,
              const std::vector<char>* first) {
    if (dim != 1 && dim != 2) { err = "dim must be 1 or 2"; return FL_EINVAL; }
    if (nv < dim + 1 || nc < 1 || !V || !C) { err = "empty mesh or NULL arrays"; return FL_EINVAL; }
    if (nv > (1LL << 30) || nc > (1LL << 29)) { err = "mesh too large"; return FL_EINVAL; }
    P.dim = dim;
    P.nvpc = dim + 1;
    P.nv = nv;
    P.nc = nc;
    const int m = P.nvpc;
    P.V.assign(V, V + nv * dim);
    P.C.assign(C, C + nc * m);
    for (int64_t i = 0; i < nc * m; ++i)
        if (P.C[i] < 0 || P.C[i] >= nv) { err = "cell vertex index out of range"; return FL_EINVAL; }
    for (int64_t i = 0; i < nv * dim; ++i)
        if (!std::isfinite(P.V[i])) { err = "non-finite vertex coordinate"; return FL_EINVAL; }
    double scale = 0;
    for (double x : P.V) scale = std::max(scale, std::fabs(x));
    if (scale == 0) scale = 1;
    P.jac.assign(nc, 0.0);
    for (int64_t k = 0; k < nc; ++k) {
        int* c = &P.C[k * m];
        if (dim == 1) {
            if (P.V[c[0]] > P.V[c[1]]) std::swap(c[0], c[1]);
            double h = P.V[c[1]] - P.V[c[0]];
            if (!(h > 0)) { err = "degenerate interval"; return FL_EINVAL; }
            P.jac[k] = h;
        } else {
            const double *a = &P.V[2 * c[0]], *b = &P.V[2 * c[1]], *d = &P.V[2 * c[2]];
            double det = (b[0] - a[0]) * (d[1] - a[1]) - (b[1] - a[1]) * (d[0] - a[0]);
            if (det < 0) { std::swap(c[1], c[2]); det = -det; }
            if (!(det > 2e-14 * scale * scale)) { err = "degenerate triangle"; return FL_EINVAL; }
            if (c[0] == c[1] || c[1] == c[2] || c[0] == c[2]) { err = "repeated vertex in a cell"; return FL_EINVAL; }
            P.jac[k] = det;
        }
    }
    // boundary facets with inward normals
    P.F.clear();
    P.FN.clear();
    P.FLEN.clear();
    if (dim == 1) {
        std::vector<int> cnt(nv, 0), owner(nv, -1);
        for (int64_t k = 0; k < nc; ++k)
            for (int a = 0; a < 2; ++a) { cnt[P.C[2 * k + a]]++; owner[P.C[2 * k + a]] = (int)k; }
        for (int64_t v = 0; v < nv; ++v) {
            if (cnt[v] > 2) { err = "vertex shared by more than two intervals"; return FL_EINVAL; }
            if (cnt[v] == 1) {
                P.F.push_back((int)v);
                P.FN.push_back(P.C[2 * owner[v]] == v ? 1.0 : -1.0);
                P.FLEN.push_back(1.0);
            }
        }
    } else {
        std::unordered_map<uint64_t, int> idx;
        std::vector<int> ek, eo, ecount;
        std::vector<uint64_t> keys;
        for (int64_t k = 0; k < nc; ++k) {
            const int* c = &P.C[3 * k];
            for (int e = 0; e < 3; ++e) {
                int p = c[e], q = c[(e + 1) % 3], r = c[(e + 2) % 3];
                uint64_t key = ((uint64_t)std::min(p, q) << 32) | (uint32_t)std::max(p, q);
                auto it = idx.find(key);
                if (it == idx.end()) {
                    idx.emplace(key, (int)keys.size());
                    keys.push_back(key);
                    ek.push_back((int)k);
                    eo.push_back(r);
                    ecount.push_back(1);
                } else {
                    ecount[it->second]++;
                }
            }
        }
        std::vector<int> order(keys.size());
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(), [&](int a, int b) { return keys[a] < keys[b]; });
        for (int e : order) {
            if (ecount[e] > 2) { err = "edge shared by more than two triangles"; return FL_EINVAL; }
            if (ecount[e] != 1) continue;
            int p = (int)(keys[e] >> 32), q = (int)(keys[e] & 0xffffffffu), r = eo[e];
            double tx = P.V[2 * q] - P.V[2 * p], ty = P.V[2 * q + 1] - P.V[2 * p + 1];
            double L = std::hypot(tx, ty);
            double nx = -ty / L, ny = tx / L;
            if (nx * (P.V[2 * r] - P.V[2 * p]) + ny * (P.V[2 * r + 1] - P.V[2 * p + 1]) < 0) { nx = -nx; ny = -ny; }
            P.F.push_back(p);
            P.F.push_back(q);
            P.FN.push_back(nx);
            P.FN.push_back(ny);
            P.FLEN.push_back(L);
        }
    }
    P.nf = (int64_t)P.FLEN.size();
    P.onb.assign(nv, 0);
    for (int v : P.F) P.onb[v] = 1;
    // adjacency
    std::vector<std::vector<int>> v2c(nv), nb(nv), v2f(nv);
    for (int64_t k = 0; k < nc; ++k)
        for (int a = 0; a < m; ++a) {
            int v = P.C[k * m + a];
            v2c[v].push_back((int)k);
            for (int b = 0; b < m; ++b)
                if (b != a) nb[v].push_back(P.C[k * m + b]);
        }
    for (auto& l : nb) {
        std::sort(l.begin(), l.end());
        l.erase(std::unique(l.begin(), l.end()), l.end());
    }
    for (int64_t f = 0; f < P.nf; ++f)
        for (int a = 0; a < dim; ++a) v2f[P.F[f * dim + a]].push_back((int)f);
    csr_from_lists(v2c, P.v2c_ptr, P.v2c);
    csr_from_lists(nb, P.nbr_ptr, P.nbr);
    csr_from_lists(v2f, P.v2f_ptr, P.v2f);
    // spatial (Morton) order of cells
    std::vector<double> cx(nc), cy(nc, 0.0);
    double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300};
    for (int64_t k = 0; k < nc; ++k) {
        double sx = 0, sy = 0;
        for (int a = 0; a < m; ++a) {
            sx += P.V[dim * P.C[k * m + a]];
            if (dim == 2) sy += P.V[2 * P.C[k * m + a] + 1];
        }
        cx[k] = sx / m;
        cy[k] = sy / m;
        lo[0] = std::min(lo[0], cx[k]);
        hi[0] = std::max(hi[0], cx[k]);
        lo[1] = std::min(lo[1], cy[k]);
        hi[1] = std::max(hi[1], cy[k]);
    }
    std::vector<uint64_t> key(nc);
    for (int64_t k = 0; k < nc; ++k) {
        double fx = (hi[0] > lo[0]) ? (cx[k] - lo[0]) / (hi[0] - lo[0]) : 0.0;
        double fy = (hi[1] > lo[1]) ? (cy[k] - lo[1]) / (hi[1] - lo[1]) : 0.0;
        uint32_t ix = (uint32_t)std::min(65535.0, fx * 65535.0), iy = (uint32_t)std::min(65535.0, fy * 65535.0);
        uint32_t z = (dim == 1) ? (uint32_t)std::min(4294967295.0, fx * 4294967295.0) : (spread16(ix) | (spread16(iy) << 1));
        key[k] = ((uint64_t)z << 32) | (uint64_t)k;
    }
    std::sort(key.begin(), key.end());
    // cells flagged `first` ahead of the others, each part in Morton order
    if (first) std::stable_partition(key.begin(), key.end(), [&](uint64_t x) { return (*first)[x & 0xffffffffu] != 0; });
    P.perm.resize(nc);
    P.iperm.resize(nc);
    for (int64_t i = 0; i < nc; ++i) {
        P.perm[i] = (int)(key[i] & 0xffffffffu);
        P.iperm[P.perm[i]] = (int)i;
    }
    return FL_OK;
}

int plan_dofs(Plan& P, int paper_all, std::string& err) {
    const int m = P.nvpc, dim = P.dim;
    const int64_t nc = P.nc, nv = P.nv;
    P.paper_all = paper_all;
    P.vod.clear();
    P.dov.assign(nv, -1);
    for (int64_t v = 0; v < nv; ++v)
        if (paper_all || !P.onb[v]) {
            P.dov[v] = (int)P.vod.size();
            P.vod.push_back((int)v);
        }
    P.n = (int64_t)P.vod.size();
    if (P.n == 0) { err = "mesh has no degrees of freedom"; return FL_EINVAL; }
    // internal arrays
    P.cdof.assign(nc * m, -1);
    P.hasdof.assign(nc, 0);
    for (int64_t k = 0; k < nc; ++k) {
        int K = P.perm[k];
        for (int a = 0; a < m; ++a) {
            int d = P.dov[P.C[(int64_t)K * m + a]];
            P.cdof[k * m + a] = d;
            if (d >= 0) P.hasdof[k] = 1;
        }
    }
    // blocks and local DOF lists
    P.nblk = (nc + TILE - 1) / TILE;
    P.L_ptr.assign(P.nblk + 1, 0);
    P.L_dof.clear();
    P.loc.assign(nc * m, -1);
    P.maxL = 0;
    for (int64_t B = 0; B < P.nblk; ++B) {
        std::vector<int> L;
        for (int64_t k = B * TILE; k < std::min(nc, (B + 1) * TILE); ++k)
            for (int a = 0; a < m; ++a)
                if (P.cdof[k * m + a] >= 0) L.push_back(P.cdof[k * m + a]);
        std::sort(L.begin(), L.end());
        L.erase(std::unique(L.begin(), L.end()), L.end());
        for (int64_t k = B * TILE; k < std::min(nc, (B + 1) * TILE); ++k)
            for (int a = 0; a < m; ++a) {
                int d = P.cdof[k * m + a];
                if (d >= 0) P.loc[k * m + a] = (int)(std::lower_bound(L.begin(), L.end(), d) - L.begin());
            }
        P.maxL = std::max(P.maxL, (int)L.size());
        P.L_dof.insert(P.L_dof.end(), L.begin(), L.end());
        P.L_ptr[B + 1] = (int)P.L_dof.size();
    }
    // incidence: for each block position, (lane*m + slot) entries in lane order
    {
        std::vector<std::vector<int>> inc(P.L_dof.size());
        for (int64_t k = 0; k < nc; ++k) {
            int64_t B = k / TILE;
            int lane = (int)(k % TILE);
            for (int a = 0; a < m; ++a)
                if (P.loc[k * m + a] >= 0) inc[P.L_ptr[B] + P.loc[k * m + a]].push_back(lane * m + a);
        }
        csr_from_lists(inc, P.inc_ptr, P.inc_ent);
    }
    // the tile list is built on first use (ensure_plan_tiles)
    P.tiles.clear();
    P.toff.clear();
    // occurrences of each DOF in block lists
    {
        std::vector<std::vector<int>> ob(P.n), ol(P.n);
        for (int64_t B = 0; B < P.nblk; ++B)
            for (int p = P.L_ptr[B]; p < P.L_ptr[B + 1]; ++p) {
                ob[P.L_dof[p]].push_back((int)B);
                ol[P.L_dof[p]].push_back(p - P.L_ptr[B]);
            }
        csr_from_lists(ob, P.occ_ptr, P.occ_blk);
        std::vector<int> tmp;
        csr_from_lists(ol, tmp, P.occ_loc);
    }
    // pair classes, in parallel over ranges of original cells.  Per-range outputs are
    // concatenated in cell order, so nothing depends on the number of threads.
    const int nthr = (int)std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
    const int64_t chunk = (nc + nthr - 1) / nthr;
    struct Part {
        std::vector<int> ex, ef_f, ef_c, tp_type, tp_vert, tp_cell, np_a, np_b;
    };
    std::vector<Part> parts(nthr);
    std::vector<int64_t> ex_off(nc), ef_off(nc);
    std::vector<int> ex_len(nc), ef_len(nc, 0);
    auto classify = [&](int t) {
        Part& o = parts[t];
        const int64_t K0 = (int64_t)t * chunk, K1 = std::min(nc, K0 + chunk);
        if (K0 >= K1) return;
        std::vector<int64_t> vs0(nv, -1), vs1(nv, -1), cs(nc, -1), fs(std::max<int64_t>(P.nf, 1), -1);
        std::vector<int> n1, touch, nearc;
        std::vector<std::pair<int, int>> efl;
        for (int64_t K = K0; K < K1; ++K) {
            const int* c = &P.C[K * m];
            const int k = P.iperm[K];
            n1.clear();
            for (int a = 0; a < m; ++a) {
                vs0[c[a]] = K;
                vs1[c[a]] = K;
                n1.push_back(c[a]);
            }
            for (int a = 0; a < m; ++a)
                for (int q = P.nbr_ptr[c[a]]; q < P.nbr_ptr[c[a] + 1]; ++q) {
                    const int u = P.nbr[q];
                    if (vs1[u] != K) {
                        vs1[u] = K;
                        n1.push_back(u);
                    }
                }
            touch.clear();
            nearc.clear();
            cs[K] = K;
            for (int a = 0; a < m; ++a)
                for (int q = P.v2c_ptr[c[a]]; q < P.v2c_ptr[c[a] + 1]; ++q) {
                    const int M = P.v2c[q];
                    if (cs[M] != K) {
                        cs[M] = K;
                        touch.push_back(M);
                    }
                }
            for (int u : n1) {
                if (vs0[u] == K) continue;
                for (int q = P.v2c_ptr[u]; q < P.v2c_ptr[u + 1]; ++q) {
                    const int M = P.v2c[q];
                    if (cs[M] != K) {
                        cs[M] = K;
                        nearc.push_back(M);
                    }
                }
            }
            std::sort(touch.begin(), touch.end());
            std::sort(nearc.begin(), nearc.end());
            // exclusion list of the far-field kernel (internal indices)
            const size_t e0 = o.ex.size();
            ex_off[K] = (int64_t)e0;
            o.ex.push_back(k);
            for (int M : touch) o.ex.push_back(P.iperm[M]);
            for (int M : nearc) o.ex.push_back(P.iperm[M]);
            std::sort(o.ex.begin() + e0, o.ex.end());
            ex_len[K] = (int)(o.ex.size() - e0);
            // touching pairs, canonical: lower original index plays K
            for (int M : touch) {
                if (M < K) continue;
                const int km = P.iperm[M];
                if (!P.hasdof[k] && !P.hasdof[km]) continue;
                const int* d = &P.C[(int64_t)M * m];
                int sv[3], ns = 0;
                for (int a = 0; a < m; ++a)
                    for (int b = 0; b < m; ++b)
                        if (c[a] == d[b]) sv[ns++] = c[a];
                int tv[5] = {-1, -1, -1, -1, -1};
                int type;
                if (dim == 1) {
                    // left interval has the shared vertex as its right end
                    const int left = (c[1] == sv[0]) ? (int)K : M, right = (left == K) ? M : (int)K;
                    tv[0] = P.C[(int64_t)left * 2];
                    tv[1] = sv[0];
                    tv[2] = P.C[(int64_t)right * 2 + 1];
                    type = 2;
                    o.tp_cell.push_back(left);
                    o.tp_cell.push_back(right);
                } else if (ns == 2) {
                    type = 0;
                    tv[0] = sv[0];
                    tv[1] = sv[1];
                    for (int a = 0; a < 3; ++a)
                        if (c[a] != sv[0] && c[a] != sv[1]) tv[2] = c[a];
                    for (int a = 0; a < 3; ++a)
                        if (d[a] != sv[0] && d[a] != sv[1]) tv[3] = d[a];
                    o.tp_cell.push_back((int)K);
                    o.tp_cell.push_back(M);
                } else {
                    type = 1;
                    int ia = 0, ib = 0;
                    for (int a = 0; a < 3; ++a) {
                        if (c[a] == sv[0]) ia = a;
                        if (d[a] == sv[0]) ib = a;
                    }
                    tv[0] = sv[0];
                    tv[1] = c[(ia + 1) % 3];
                    tv[2] = c[(ia + 2) % 3];
                    tv[3] = d[(ib + 1) % 3];
                    tv[4] = d[(ib + 2) % 3];
                    o.tp_cell.push_back((int)K);
                    o.tp_cell.push_back(M);
                }
                o.tp_type.push_back(type);
                for (int a = 0; a < 5; ++a) o.tp_vert.push_back(tv[a]);
            }
            // near separated pairs, unordered by internal index
            for (int M : nearc) {
                const int km = P.iperm[M];
                if (km < k) continue;
                if (!P.hasdof[k] && !P.hasdof[km]) continue;
                o.np_a.push_back(k);
                o.np_b.push_back(km);
            }
            // boundary facets handled individually (touching or at distance 1)
            if (P.hasdof[k]) {
                efl.clear();
                for (int v : n1)
                    for (int q = P.v2f_ptr[v]; q < P.v2f_ptr[v + 1]; ++q) {
                        const int f = P.v2f[q];
                        if (fs[f] == K) continue;
                        fs[f] = K;
                        int sh = 0;
                        for (int a = 0; a < dim; ++a) sh += (vs0[P.F[(int64_t)f * dim + a]] == K) ? 1 : 0;
                        const int cls = (sh == 0) ? 1 : (dim == 1 ? 2 : (sh == 2 ? 2 : 3));
                        efl.push_back({f, cls});
                    }
                std::sort(efl.begin(), efl.end());
                ef_off[K] = (int64_t)o.ef_f.size();
                ef_len[K] = (int)efl.size();
                for (auto& pr : efl) {
                    o.ef_f.push_back(pr.first);
                    o.ef_c.push_back(pr.second);
                }
            }
        }
    };
    {
        std::vector<std::thread> th;
        for (int t = 1; t < nthr; ++t) th.emplace_back(classify, t);
        classify(0);
        for (auto& x : th) x.join();
    }
    P.np_a.clear();
    P.np_b.clear();
    P.tp_type.clear();
    P.tp_vert.clear();
    P.tp_cell.clear();
    for (auto& o : parts) {
        P.np_a.insert(P.np_a.end(), o.np_a.begin(), o.np_a.end());
        P.np_b.insert(P.np_b.end(), o.np_b.begin(), o.np_b.end());
        P.tp_type.insert(P.tp_type.end(), o.tp_type.begin(), o.tp_type.end());
        P.tp_vert.insert(P.tp_vert.end(), o.tp_vert.begin(), o.tp_vert.end());
        P.tp_cell.insert(P.tp_cell.end(), o.tp_cell.begin(), o.tp_cell.end());
    }
    // exclusion and facet lists in internal order
    P.ex_ptr.assign(nc + 1, 0);
    P.ef_ptr.assign(nc + 1, 0);
    for (int64_t k = 0; k < nc; ++k) {
        const int K = P.perm[k];
        P.ex_ptr[k + 1] = P.ex_ptr[k] + ex_len[K];
        P.ef_ptr[k + 1] = P.ef_ptr[k] + ef_len[K];
    }
    P.ex_idx.resize(P.ex_ptr[nc]);
    P.ef_fac.resize(P.ef_ptr[nc]);
    P.ef_cls.resize(P.ef_ptr[nc]);
    for (int64_t k = 0; k < nc; ++k) {
        const int K = P.perm[k];
        const Part& o = parts[K / chunk];
        std::copy(o.ex.begin() + ex_off[K], o.ex.begin() + ex_off[K] + ex_len[K], P.ex_idx.begin() + P.ex_ptr[k]);
        if (ef_len[K]) {
            std::copy(o.ef_f.begin() + ef_off[K], o.ef_f.begin() + ef_off[K] + ef_len[K], P.ef_fac.begin() + P.ef_ptr[k]);
            std::copy(o.ef_c.begin() + ef_off[K], o.ef_c.begin() + ef_off[K] + ef_len[K], P.ef_cls.begin() + P.ef_ptr[k]);
        }
    }
    std::vector<Part>().swap(parts);
    // element -> (near pair, role), pairs in increasing order
    {
        std::vector<int> cnt(nc + 1, 0);
        for (size_t p = 0; p < P.np_a.size(); ++p) {
            cnt[P.np_a[p] + 1]++;
            cnt[P.np_b[p] + 1]++;
        }
        for (int64_t k = 0; k < nc; ++k) cnt[k + 1] += cnt[k];
        P.enp_ptr = cnt;
        P.enp_ent.assign(cnt[nc], 0);
        std::vector<int> cur(cnt.begin(), cnt.end() - 1);
        for (size_t p = 0; p < P.np_a.size(); ++p) {
            P.enp_ent[cur[P.np_a[p]]++] = (int)(2 * p);
            P.enp_ent[cur[P.np_b[p]]++] = (int)(2 * p + 1);
        }
    }
    // contribution slots and the sparse near-field pattern with its gather lists
    const int64_t ntp = (int64_t)P.tp_type.size(), nnp = (int64_t)P.np_a.size();
    P.tp_slot.resize(ntp);
    int64_t cur = 0;
    for (int64_t p = 0; p < ntp; ++p) {
        const int nl = (P.tp_type[p] == 0) ? 4 : (P.tp_type[p] == 1 ? 5 : 3);
        P.tp_slot[p] = cur;
        cur += nl * nl;
    }
    P.np_slot0 = cur;
    cur += nnp * m * m;
    P.el_slot0 = cur;
    cur += nc * m * m;
    P.nslots = cur;
    // Rows of the sparse near-field part are generated row by row from inverse incidence
    // maps (dof -> cells -> element block / touching pairs / near pairs), sorted on
    // (column, slot) and turned into CSR pieces; threads own contiguous row ranges and
    // their pieces are concatenated in row order.
    std::vector<int> c2t_ptr(nc + 1, 0), c2t;  // original cell -> touching pairs
    for (int64_t p = 0; p < ntp; ++p) {
        c2t_ptr[P.tp_cell[2 * p] + 1]++;
        c2t_ptr[P.tp_cell[2 * p + 1] + 1]++;
    }
    for (int64_t K = 0; K < nc; ++K) c2t_ptr[K + 1] += c2t_ptr[K];
    c2t.resize(c2t_ptr[nc]);
    {
        std::vector<int> cur(c2t_ptr.begin(), c2t_ptr.end() - 1);
        for (int64_t p = 0; p < ntp; ++p) {
            c2t[cur[P.tp_cell[2 * p]]++] = (int)p;
            c2t[cur[P.tp_cell[2 * p + 1]]++] = (int)p;
        }
    }
    struct RowPart {
        std::vector<int> cnt, col;           // per row: number of distinct columns; columns
        std::vector<int64_t> gcnt, slot;     // per distinct column: number of slots; slots
    };
    std::vector<RowPart> rparts(nthr);
    const int64_t rchunk = (P.n + nthr - 1) / nthr;
    auto build_rows = [&](int t) {
        RowPart& o = rparts[t];
        const int64_t i0 = (int64_t)t * rchunk, i1 = std::min(P.n, i0 + rchunk);
        std::vector<std::pair<int, int64_t>> e;
        std::vector<int> tps, cols;
        std::vector<int64_t> placed;
        // per column: the row that last used it, its slot count and its write position
        std::vector<int64_t> mark(P.n, -1);
        std::vector<int> ccount(P.n, 0);
        std::vector<int64_t> cpos(P.n, 0);
        e.reserve(4096);
        const int64_t rows_here = std::max<int64_t>(0, i1 - i0);
        o.cnt.reserve(rows_here);
        o.col.reserve(rows_here * 48);
        o.gcnt.reserve(rows_here * 48);
        o.slot.reserve(rows_here * 160);
        for (int64_t i = i0; i < i1; ++i) {
            const int v = P.vod[i];
            e.clear();
            tps.clear();
            for (int q = P.v2c_ptr[v]; q < P.v2c_ptr[v + 1]; ++q) {
                const int K = P.v2c[q];
                const int k = P.iperm[K];
                int a = 0;
                for (int x = 0; x < m; ++x)
                    if (P.C[(int64_t)K * m + x] == v) a = x;
                // element block, row a (internal slots follow the oriented cell order)
                for (int b = 0; b < m; ++b) {
                    const int j = P.cdof[(int64_t)k * m + b];
                    if (j >= 0) e.push_back({j, P.el_slot0 + (int64_t)k * m * m + a * m + b});
                }
                for (int q2 = c2t_ptr[K]; q2 < c2t_ptr[K + 1]; ++q2) tps.push_back(c2t[q2]);
                // near pairs of cell k in either role
                for (int q2 = P.enp_ptr[k]; q2 < P.enp_ptr[k + 1]; ++q2) {
                    const int ent = P.enp_ent[q2];
                    const int64_t pp = ent >> 1;
                    const int role = ent & 1;
                    const int other = role ? P.np_a[pp] : P.np_b[pp];
                    for (int b = 0; b < m; ++b) {
                        const int j = P.cdof[(int64_t)other * m + b];
                        if (j < 0) continue;
                        const int64_t sl = role ? P.np_slot0 + pp * m * m + b * m + a : P.np_slot0 + pp * m * m + a * m + b;
                        e.push_back({j, sl});
                    }
                }
            }
            std::sort(tps.begin(), tps.end());
            tps.erase(std::unique(tps.begin(), tps.end()), tps.end());
            for (int p2 : tps) {
                const int nl = (P.tp_type[p2] == 0) ? 4 : (P.tp_type[p2] == 1 ? 5 : 3);
                const int* tv = &P.tp_vert[5 * (int64_t)p2];
                int a = -1;
                for (int x = 0; x < nl; ++x)
                    if (tv[x] == v) a = x;
                if (a < 0) continue;
                for (int b = 0; b < nl; ++b) {
                    const int j = P.dov[tv[b]];
                    if (j >= 0) e.push_back({j, P.tp_slot[p2] + a * nl + b});
                }
            }
            // bucket the entries by column (columns ascending, slots ascending within one)
            cols.clear();
            for (const auto& pr : e) {
                if (mark[pr.first] != i) {
                    mark[pr.first] = i;
                    ccount[pr.first] = 0;
                    cols.push_back(pr.first);
                }
                ccount[pr.first]++;
            }
            std::sort(cols.begin(), cols.end());
            int64_t pos = 0;
            for (int c : cols) {
                cpos[c] = pos;
                pos += ccount[c];
            }
            placed.resize(pos);
            for (const auto& pr : e) placed[cpos[pr.first]++] = pr.second;
            int64_t start = 0;
            for (int c : cols) {
                const int64_t end = start + ccount[c];
                for (int64_t q = start + 1; q < end; ++q) {  // insertion sort of the column's slots
                    const int64_t x = placed[q];
                    int64_t r = q - 1;
                    while (r >= start && placed[r] > x) {
                        placed[r + 1] = placed[r];
                        --r;
                    }
                    placed[r + 1] = x;
                }
                o.col.push_back(c);
                o.gcnt.push_back(ccount[c]);
                start = end;
            }
            o.slot.insert(o.slot.end(), placed.begin(), placed.end());
            o.cnt.push_back((int)cols.size());
        }
    };
    {
        std::vector<std::thread> th;
        for (int t = 1; t < nthr; ++t) th.emplace_back(build_rows, t);
        build_rows(0);
        for (auto& x : th) x.join();
    }
    // concatenate: offsets per part first, then the copies in parallel
    std::vector<int64_t> coff(nthr + 1, 0), soff(nthr + 1, 0);
    for (int t = 0; t < nthr; ++t) {
        coff[t + 1] = coff[t] + (int64_t)rparts[t].col.size();
        soff[t + 1] = soff[t] + (int64_t)rparts[t].slot.size();
    }
    P.csr_ptr.assign(P.n + 1, 0);
    {
        int64_t row = 0;
        for (auto& o : rparts)
            for (int c : o.cnt) {
                P.csr_ptr[row + 1] = P.csr_ptr[row] + c;
                ++row;
            }
    }
    P.csr_col.resize(coff[nthr]);
    P.g_ptr.resize(coff[nthr] + 1);
    P.g_slot.resize(soff[nthr]);
    P.g_ptr[coff[nthr]] = soff[nthr];
    {
        auto copy_part = [&](int t) {
            const RowPart& o = rparts[t];
            std::copy(o.col.begin(), o.col.end(), P.csr_col.begin() + coff[t]);
            std::copy(o.slot.begin(), o.slot.end(), P.g_slot.begin() + soff[t]);
            int64_t acc = soff[t];
            for (size_t z = 0; z < o.gcnt.size(); ++z) {
                P.g_ptr[coff[t] + z] = acc;
                acc += o.gcnt[z];
            }
        };
        std::vector<std::thread> th;
        for (int t = 1; t < nthr; ++t) th.emplace_back(copy_part, t);
        copy_part(0);
        for (auto& x : th) x.join();
    }
    return FL_OK;
}

void ensure_plan_tiles(Plan& P) {
    if (!P.tiles.empty() || P.sym_K) return;
    const int64_t nb = P.nblk, nt = nb * (nb + 1) / 2;
    // row I holds tiles (I, I) .. (I, nb - 1), whose partial blocks take n_I sum_{J >= I} n_J entries
    std::vector<int64_t> suf(nb + 1, 0), row_t(nb + 1, 0), row_o(nb + 1, 0);
    for (int64_t J = nb - 1; J >= 0; --J) suf[J] = suf[J + 1] + (P.L_ptr[J + 1] - P.L_ptr[J]);
    for (int64_t I = 0; I < nb; ++I) {
        row_t[I + 1] = row_t[I] + (nb - I);
        row_o[I + 1] = row_o[I] + (int64_t)(P.L_ptr[I + 1] - P.L_ptr[I]) * suf[I];
    }
    P.tiles.resize(2 * nt);
    P.toff.resize(nt + 1);
    P.toff[nt] = row_o[nb];
    // threads take row ranges of about equal tile counts
    const int nthr = (int)std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
    auto rows = [&](int t) {
        const int64_t a = (int64_t)(std::lower_bound(row_t.begin(), row_t.end(), nt * t / nthr) - row_t.begin());
        const int64_t b = (int64_t)(std::lower_bound(row_t.begin(), row_t.end(), nt * (t + 1) / nthr) - row_t.begin());
        for (int64_t I = a; I < std::min(b, nb); ++I) {
            const int64_t nI = P.L_ptr[I + 1] - P.L_ptr[I];
            int64_t k = row_t[I], off = row_o[I];
            for (int64_t J = I; J < nb; ++J, ++k) {
                P.tiles[2 * k] = (int)I;
                P.tiles[2 * k + 1] = (int)J;
                P.toff[k] = off;
                off += nI * (P.L_ptr[J + 1] - P.L_ptr[J]);
            }
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nthr; ++t) th.emplace_back(rows, t);
    rows(0);
    for (auto& x : th) x.join();
}

int64_t plan_tile_count(const Plan& P) {
    return (P.tiles.empty() && !P.sym_K) ? P.nblk * (P.nblk + 1) / 2 : (int64_t)P.tiles.size() / 2;
}

}  // namespace fl
