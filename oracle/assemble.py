"""Element-pair assembly of the dense stiffness matrix (oracle; test infrastructure only).

The matrix is A^s_ij = a(phi_i, phi_j) with the bilinear form of Section 2,

  a(u,v) = C(d,s)/2 ∫_Ω∫_Ω (u(x)-u(y))(v(x)-v(y)) / |x-y|^{d+2s}
         + C(d,s)/(2s) ∫_Ω u v(x) ∫_∂Ω n_y·(x-y) / |x-y|^{d+2s},

split as in Section 5 into a sum over ordered element pairs a^{K×K'} (eq.
elementPair) plus a sum over element/boundary-facet pairs a^{K×e} (eq.
elementPairBoundary); the sum printed there with a(phi_i, phi_i) on the left is
read as a(phi_i, phi_j).

Quadrature reading (the paper defers the rules to Sauter-Schwab and its
Appendix B; all orders are options, see QuadOrders):

* separated pairs (no common vertex): collapsed Gauss rule of order k_near
  (vertex-graph distance 1) or k_far (distance >= 2) on both elements.  The
  unordered pair {K,K'} contributes -C Σ w_a w_b phi_i(x_a) phi_j(y_b) k_ab to
  the off-diagonal block and C Σ_a w_a phi_i phi_j(x_a) Σ_b w_b k_ab to the
  block of K (and symmetrically to K'), k = |x-y|^{-d-2s}; the sign agrees with
  Section 6, where disjoint supports give -C ∬ k phi psi.
* touching pairs {K,K'} (K the lower cell index; shared vertices P, Q taken in
  the order they appear in K's counter-clockwise vertex list, cells rotated to
  start at a shared vertex): relative coordinates in which the whole integrand is
  homogeneous of degree -2s, so the radial integral is done in closed form and
  only smooth angular variables are left to Gauss-Legendre:
    identical (2D)   : 1D integral over the direction, three pieces of [0, pi),
                       2 k_touch points per piece (the direction integrand sharpens
                       on anisotropic cells; this rule costs 6 k_touch evaluations);
    common edge (2D) : 2D integral over the l1-unit directions of
                       (x1-y1, x2, y2), four pieces;
    common vertex(2D): Duffy map of K×K' into [0,1]^4, two regions, 3D Gauss of
                       order k_vertex;
    1D               : identical in closed form, common vertex by a Duffy map.
* boundary term: 1D facets are points, so the inner integral is a point value;
  in 2D the inner edge integral uses Gauss order k_near/k_far for
  non-touching pairs; touching pairs (e an edge of K, or e and K sharing one
  vertex) use the same homogeneity trick with order k_bnd.

Everything is float64 and deliberately plain: loops over elements, numpy over
the partner elements of one element at a time.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import gamma

from . import rules
from .mesh import OracleMesh


def frac_constant(d: int, s: float) -> float:
    """C(d,s) = 2^{2s} s Γ(s + d/2) / (π^{d/2} Γ(1 - s))  (Section 2)."""
    return 2.0 ** (2 * s) * s * gamma(s + d / 2.0) / (math.pi ** (d / 2.0) * gamma(1.0 - s))


@dataclass(frozen=True)
class QuadOrders:
    k_far: int = 4
    k_near: int = 6
    k_touch: int = 8     # common-edge pairs; identical pairs use 2 * k_touch angular points per piece
    k_bnd: int = 8
    k_vertex: int = 6    # common-vertex pairs


# ---------------------------------------------------------------- points ----
def cell_points(mesh: OracleMesh, ks, order: int):
    """Quadrature on cells ks: points [M,q,d], weights [M,q], reference shapes [q,d+1]."""
    ks = np.atleast_1d(ks)
    if mesh.dim == 1:
        t, w = rules.gauss01(order)
        a = mesh.V[mesh.C[ks, 0], 0]
        b = mesh.V[mesh.C[ks, 1], 0]
        x = (a[:, None] + (b - a)[:, None] * t[None, :])[..., None]
        return x, w[None, :] * (b - a)[:, None], np.stack([1.0 - t, t], axis=1)
    lam, w = rules.triangle(order)
    P = mesh.V[mesh.C[ks]]  # M,3,2
    x = (P[:, None, 0, :] + lam[None, :, 0:1] * (P[:, None, 1, :] - P[:, None, 0, :])
         + lam[None, :, 1:2] * (P[:, None, 2, :] - P[:, None, 0, :]))
    return x, w[None, :] * (2.0 * mesh.vol[ks])[:, None], rules.p1_shape(lam)


# ------------------------------------------------------------ separated ----
def separated_blocks(mesh, s, C, k, others, order):
    """Unordered separated pairs {K_k, K_m}, m in others, with the order-`order` rule.

    Returns off [M,d+1,d+1] (rows: vertices of K_k, cols: vertices of K_m),
    the summed block of K_k, and the blocks of each K_m.
    """
    d = mesh.dim
    xa, wa, pha = cell_points(mesh, k, order)
    xa, wa = xa[0], wa[0]
    yb, wb, phb = cell_points(mesh, others, order)
    diff = xa[None, :, None, :] - yb[:, None, :, :]
    r2 = np.sum(diff * diff, axis=-1)
    ker = r2 ** (-(d + 2.0 * s) / 2.0)
    Kw = ker * wa[None, :, None] * wb[:, None, :]
    off = -C * np.einsum("ai,mab,bj->mij", pha, Kw, phb)
    blk_k = C * np.einsum("ai,aj,a->ij", pha, pha, Kw.sum(axis=(0, 2)))
    blk_m = C * np.einsum("bi,bj,mb->mij", phb, phb, Kw.sum(axis=1))
    return off, blk_k, blk_m


# ------------------------------------------------------------- touching ----
def identical_1d(mesh, s, C, k):
    """a^{K×K} in 1D: (g_i g_j) ∬ |x-y|^{1-2s} in closed form."""
    h = mesh.vol[k]
    v = C * h ** (1.0 - 2.0 * s) / ((2.0 - 2.0 * s) * (3.0 - 2.0 * s))
    return list(mesh.C[k]), v * np.array([[1.0, -1.0], [-1.0, 1.0]])


def common_vertex_1d(mesh, s, C, k, m, kt):
    """Both orders of a 1D pair sharing one vertex: Duffy map, radial part exact."""
    ck, cm = mesh.C[k], mesh.C[m]
    if ck[1] == cm[0]:
        left, right = k, m
    else:
        left, right = m, k
    a, v = mesh.C[left]
    b = mesh.C[right][1]
    h1, h2 = mesh.vol[left], mesh.vol[right]
    cK = np.array([1.0, -1.0, 0.0])
    cKt = np.array([0.0, -1.0, 1.0])
    t, w = rules.gauss01(kt)
    acc = np.zeros((3, 3))
    for eta, we in zip(t, w):
        d1 = cK - cKt * eta
        d2 = cK * eta - cKt
        acc += we * (np.outer(d1, d1) * (h1 + h2 * eta) ** (-1.0 - 2.0 * s)
                     + np.outer(d2, d2) * (h1 * eta + h2) ** (-1.0 - 2.0 * s))
    return [a, v, b], C * h1 * h2 / (3.0 - 2.0 * s) * acc


_GHAT = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])


def identical_2d(mesh, s, C, k, kt):
    """a^{K×K} in 2D: polar coordinates in z = x^ - y^ with the overlap |T∩(T+z)|."""
    P = mesh.V[mesh.C[k]]
    J = np.stack([P[1] - P[0], P[2] - P[0]], axis=1)
    detJ = 2.0 * mesh.vol[k]
    acc = np.zeros((3, 3))
    for lo, hi in ((0.0, math.pi / 2), (math.pi / 2, 3 * math.pi / 4), (3 * math.pi / 4, math.pi)):
        th, w = rules.gauss_on(lo, hi, kt)
        u = np.stack([np.cos(th), np.sin(th)], axis=1)
        rho = 2.0 / (np.abs(u[:, 0] + u[:, 1]) + np.abs(u[:, 0]) + np.abs(u[:, 1]))
        Ju = u @ J.T
        nrm2 = np.sum(Ju * Ju, axis=1)
        g = u @ _GHAT.T
        f = w * nrm2 ** (-(1.0 + s)) * rho ** (2.0 - 2.0 * s)
        acc += np.einsum("m,mi,mj->ij", f, g, g)
    beta = 2.0 / ((2.0 - 2.0 * s) * (3.0 - 2.0 * s) * (4.0 - 2.0 * s))
    return list(mesh.C[k]), 0.5 * C * detJ ** 2 * beta * acc


def _square_grid(kt):
    t, w = rules.gauss01(kt)
    U, Vv = np.meshgrid(t, t, indexing="ij")
    W = np.outer(w, w)
    return U.ravel(), Vv.ravel(), W.ravel()


def common_edge_2d(mesh, s, C, k, m, kt):
    """Both orders of a pair with a common edge [P,Q]: radial integral in
    (x1-y1, x2, y2) exact, four smooth pieces of the l1 directions by Gauss."""
    ck, cm = list(mesh.C[k]), list(mesh.C[m])
    P, Q = [v for v in ck if v in cm]
    R = [v for v in ck if v not in (P, Q)][0]
    Rt = [v for v in cm if v not in (P, Q)][0]
    VP, VQ, VR, VRt = mesh.V[[P, Q, R, Rt]]
    cz = np.array([-1.0, 1.0, 0.0, 0.0])
    cx = np.array([0.0, -1.0, 1.0, 0.0])
    cy = np.array([0.0, 1.0, 0.0, -1.0])
    a, b, c = VQ - VP, VR - VQ, -(VRt - VQ)
    u, v, W = _square_grid(kt)
    acc = np.zeros((4, 4))
    pieces = []
    # face z1 >= 0: lambda = max(w2, 1 - w2)
    w2 = u / 2; w3 = v * (1 - w2); pieces.append((1.0, w2, w3, W * 0.5 * (1 - u / 2), 1 - w2))
    w2 = (1 + u) / 2; w3 = v * (1 - w2); pieces.append((1.0, w2, w3, W * 0.25 * (1 - u), w2))
    # face z1 <= 0: lambda = max(1 - w3, w3)
    w3 = u / 2; w2 = v * (1 - w3); pieces.append((-1.0, w2, w3, W * 0.5 * (1 - u / 2), 1 - w3))
    w3 = (1 + u) / 2; w2 = v * (1 - w3); pieces.append((-1.0, w2, w3, W * 0.25 * (1 - u), w3))
    for sig, w2, w3, wt, lam in pieces:
        w1 = sig * (1.0 - w2 - w3)
        dphi = np.outer(w1, cz) + np.outer(w2, cx) + np.outer(w3, cy)
        xy = np.outer(w1, a) + np.outer(w2, b) + np.outer(w3, c)
        r2 = np.sum(xy * xy, axis=1)
        f = wt * lam ** (2.0 * s - 3.0) * r2 ** (-(1.0 + s))
        acc += np.einsum("m,mi,mj->ij", f, dphi, dphi)
    scale = C * (2 * mesh.vol[k]) * (2 * mesh.vol[m]) / ((3.0 - 2.0 * s) * (4.0 - 2.0 * s))
    return [P, Q, R, Rt], scale * acc


def _rotate_to(cell, P):
    cell = list(cell)
    i = cell.index(P)
    return cell[i:] + cell[:i]


def common_vertex_2d(mesh, s, C, k, m, kt):
    """Both orders of a pair with one common vertex P: Duffy map to [0,1]^4 in two
    regions, radial variable exact (its power is xi^{3-2s}), 3D Gauss on the rest."""
    ck, cm = list(mesh.C[k]), list(mesh.C[m])
    P = [v for v in ck if v in cm][0]
    _, Q, R = _rotate_to(ck, P)
    _, Qt, Rt = _rotate_to(cm, P)
    VP, VQ, VR, VQt, VRt = mesh.V[[P, Q, R, Qt, Rt]]
    e = np.eye(5)
    c1, c2, c3, c4 = e[1] - e[0], e[2] - e[1], -(e[3] - e[0]), -(e[4] - e[3])
    a1, a2, a3, a4 = VQ - VP, VR - VQ, -(VQt - VP), -(VRt - VQt)
    t, w = rules.gauss01(kt)
    E1, E2, E3 = np.meshgrid(t, t, t, indexing="ij")
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel()
    E1, E2, E3 = E1.ravel(), E2.ravel(), E3.ravel()
    acc = np.zeros((5, 5))
    one = np.ones_like(E1)
    for x1, x2, y1, y2 in ((one, E1, E2, E2 * E3), (E2, E2 * E3, one, E1)):
        dphi = np.outer(x1, c1) + np.outer(x2, c2) + np.outer(y1, c3) + np.outer(y2, c4)
        xy = np.outer(x1, a1) + np.outer(x2, a2) + np.outer(y1, a3) + np.outer(y2, a4)
        r2 = np.sum(xy * xy, axis=1)
        f = W * E2 * r2 ** (-(1.0 + s))
        acc += np.einsum("m,mi,mj->ij", f, dphi, dphi)
    scale = C * (2 * mesh.vol[k]) * (2 * mesh.vol[m]) / (4.0 - 2.0 * s)
    return [P, Q, R, Qt, Rt], scale * acc


# ------------------------------------------------------------- boundary ----
def boundary_touch_1d(mesh, s, C, k, f, e_is_dof):
    """a^{K×e}, e a vertex of K: ∫_K phi_i phi_j |x-e|^{-2s} in closed form."""
    e = mesh.facets[f, 0]
    other = [v for v in mesh.C[k] if v != e][0]
    h = mesh.vol[k]
    a = np.array([1.0, 0.0])
    b = np.array([-1.0, 1.0])
    M = (np.outer(a, b) + np.outer(b, a)) / (2.0 - 2.0 * s) + np.outer(b, b) / (3.0 - 2.0 * s)
    if e_is_dof:
        M = M + np.outer(a, a) / (1.0 - 2.0 * s)
    return [e, other], C / (2.0 * s) * h ** (1.0 - 2.0 * s) * M


def boundary_own_edge_2d(mesh, s, C, k, f, kb):
    """a^{K×e} with e an edge of K (interior DOFs: only phi_R, R opposite e, is
    nonzero on K and phi_R = x2 vanishes on e).  Polar coordinates in
    (x1 - t, x2); the radial integral is exact, three angular pieces by Gauss."""
    E0, E1 = mesh.facets[f]
    R = [v for v in mesh.C[k] if v not in (E0, E1)][0]
    n = mesh.normals[f]
    VE0, VE1, VR = mesh.V[[E0, E1, R]]
    H = float(np.dot(n, VR - VE1))
    a, b = VE1 - VE0, VR - VE1
    acc = 0.0
    for sig, lo, hi, lamf in ((1.0, 0.0, 0.5, lambda w: 1 - w), (1.0, 0.5, 1.0, lambda w: w),
                              (-1.0, 0.0, 1.0, lambda w: np.ones_like(w))):
        om, wt = rules.gauss_on(lo, hi, kb)
        o1, o2 = sig * (1 - om), om
        xy = np.outer(o1, a) + np.outer(o2, b)
        r2 = np.sum(xy * xy, axis=1)
        kern = H * o2 * r2 ** (-(1.0 + s))
        acc += np.sum(wt * kern * o2 ** 2 * lamf(om) ** (2.0 * s - 3.0))
    val = C / (2.0 * s) * 2 * mesh.vol[k] * mesh.facet_len[f] * acc / ((3.0 - 2.0 * s) * (4.0 - 2.0 * s))
    return [R], np.array([[val]])


def boundary_vertex_2d(mesh, s, C, k, f, kb):
    """a^{K×e} with e and K sharing one vertex P: Duffy map of K×e to [0,1]^3 in
    two regions; xi-powers 1-2s+m (m = 0,1,2 from phi_i phi_j) integrated exactly."""
    fa, fb = mesh.facets[f]
    ck = list(mesh.C[k])
    P = fa if fa in ck else fb
    E1 = fb if P == fa else fa
    _, Q, R = _rotate_to(ck, P)
    n = mesh.normals[f]
    VP, VQ, VR, VE1 = mesh.V[[P, Q, R, E1]]
    e = np.eye(3)
    av = e[0]
    bx, by = e[1] - e[0], e[2] - e[1]
    gq, gr, ge = VQ - VP, VR - VQ, VE1 - VP
    u, v, W = _square_grid(kb)
    acc = np.zeros((3, 3))
    one = np.ones_like(u)
    for x1, x2, t, jac in ((one, u, v, one), (u, u * v, one, u)):
        xp = np.outer(x1, gq) + np.outer(x2, gr)
        N = xp @ n
        xy = xp - np.outer(t, ge)
        r2 = np.sum(xy * xy, axis=1)
        D = r2 ** (-(1.0 + s))
        bh = np.outer(x1, bx) + np.outer(x2, by)
        wgt = W * jac * N * D
        Mx = (np.outer(av, av) * wgt.sum() / (2.0 - 2.0 * s)
              + (np.einsum("m,i,mj->ij", wgt, av, bh) + np.einsum("m,mi,j->ij", wgt, bh, av)) / (3.0 - 2.0 * s)
              + np.einsum("m,mi,mj->ij", wgt, bh, bh) / (4.0 - 2.0 * s))
        acc += Mx
    val = C / (2.0 * s) * 2 * mesh.vol[k] * mesh.facet_len[f] * acc
    return [P, Q, R], val


def facet_sum(mesh, s, C, k, Y0, Y1, n, flen, order):
    """C/(2s) ∫_K phi_i phi_j(x) Σ_e ∫_e n_e·(x-y) |x-y|^{-d-2s} dy dx over the facets e from Y0
    to Y1 (1D: the points Y0, flen unused) with unit normals n and lengths flen, by the
    order-`order` rules on K and on every e.  With the inward normals of the boundary facets of
    Omega this is the boundary term; by the divergence theorem, with the normals pointing into a
    region N, the inner integral is (2s) ∫_{R^d minus N} |x-y|^{-d-2s} dy for x in N."""
    d = mesh.dim
    xa, wa, pha = cell_points(mesh, k, order)
    xa, wa = xa[0], wa[0]
    if d == 1:
        diff = xa[None, :, :] - Y0[:, None, :]
        nd = np.sum(n[:, None, :] * diff, axis=-1)
        r2 = np.sum(diff * diff, axis=-1)
        B = np.sum(nd * r2 ** (-(1.0 + 2.0 * s) / 2.0), axis=0)
    else:
        t, wt = rules.gauss01(order)
        y = Y0[:, None, :] + t[None, :, None] * (Y1 - Y0)[:, None, :]
        wy = wt[None, :] * flen[:, None]
        diff = xa[None, :, None, :] - y[:, None, :, :]
        nd = np.einsum("fd,fqbd->fqb", n, diff)
        r2 = np.sum(diff * diff, axis=-1)
        B = np.sum(nd * r2 ** (-(2.0 + 2.0 * s) / 2.0) * wy[:, None, :], axis=(0, 2))
    return C / (2.0 * s) * np.einsum("ai,aj,a->ij", pha, pha, wa * B)


def boundary_separated(mesh, s, C, k, fs, order):
    """Σ over non-touching facets fs of a^{K×e} with the order-`order` Gauss rule."""
    Y0 = mesh.V[mesh.facets[fs, 0]]
    Y1 = mesh.V[mesh.facets[fs, -1]]
    return facet_sum(mesh, s, C, k, Y0, Y1, mesh.normals[fs], mesh.facet_len[fs], order)


def near_region_facets(mesh, k):
    """The boundary of N(K), the union of cell k and the cells touching it or at vertex-graph
    distance 1 from it (the cells whose pairs with k are integrated locally).  Returns
    (Y0, Y1, n, flen, verts, bidx): per facet its end points (1D: Y1 = Y0), the unit normal
    pointing into N(K), its length (1 in 1D), its vertex ids and the index of the boundary facet
    of Omega it is, or -1 for a facet between a cell of N(K) and one outside it."""
    shared, near = mesh.classify_cells(k)
    inN = (shared > 0) | near
    Y0, Y1, nrm, flen, verts, bidx = [], [], [], [], [], []
    if mesh.dim == 1:
        for m in np.nonzero(inN)[0]:
            for side, v in enumerate(mesh.C[m]):
                others = [c for c in mesh.cells_of_vertex[v] if c != m]
                if others and inN[others[0]]:
                    continue
                f = -1
                if not others:
                    f = int(np.nonzero(mesh.facets[:, 0] == v)[0][0])
                Y0.append(mesh.V[v])
                Y1.append(mesh.V[v])
                nrm.append([1.0 if side == 0 else -1.0])  # into the interval m
                flen.append(1.0)
                verts.append([v])
                bidx.append(f)
    else:
        for m in np.nonzero(inN)[0]:
            a, b, c = mesh.C[m]
            for p, q, r in ((a, b, c), (b, c, a), (c, a, b)):
                key = (min(p, q), max(p, q))
                other = [o for o, _ in mesh.edge_owners[key] if o != m]
                if other and inN[other[0]]:
                    continue
                P0, P1 = mesh.V[key[0]], mesh.V[key[1]]
                if other:
                    f = -1
                    t = P1 - P0
                    n = np.array([-t[1], t[0]]) / np.hypot(t[0], t[1])
                    if np.dot(n, mesh.V[r] - P0) < 0:
                        n = -n
                    ln = float(np.hypot(t[0], t[1]))
                else:
                    f = mesh.facet_of_edge[(int(key[0]), int(key[1]))]
                    n = mesh.normals[f]
                    ln = mesh.facet_len[f]
                Y0.append(P0)
                Y1.append(P1)
                nrm.append(n)
                flen.append(ln)
                verts.append([key[0], key[1]])
                bidx.append(f)
    return (np.array(Y0).reshape(-1, mesh.dim), np.array(Y1).reshape(-1, mesh.dim),
            np.array(nrm).reshape(-1, mesh.dim), np.array(flen), np.array(verts, dtype=np.int64).reshape(-1, mesh.dim),
            np.array(bidx, dtype=np.int64))


# ------------------------------------------------------------- assembly ----
class _Sink:
    """Accumulates local blocks into the requested rows of the dense matrix."""

    def __init__(self, n, rows, dov):
        self.dov = dov
        self.rowpos = -np.ones(n, dtype=np.int64)
        self.rowpos[rows] = np.arange(len(rows))
        self.A = np.zeros((len(rows), n))

    def add(self, rverts, cverts, blk):
        ri = self.dov[np.asarray(rverts)]
        ci = self.dov[np.asarray(cverts)]
        for a, i in enumerate(ri):
            if i < 0 or self.rowpos[i] < 0:
                continue
            for b, j in enumerate(ci):
                if j >= 0:
                    self.A[self.rowpos[i], j] += blk[a, b]

    def add_off(self, kverts, mverts, off):
        """off[m] rows kverts, cols mverts[m]; plus the transposed blocks."""
        n = self.A.shape[1]
        ri = self.dov[kverts]
        ci = self.dov[mverts]  # M, d+1
        for a, i in enumerate(ri):
            if i < 0 or self.rowpos[i] < 0:
                continue
            msk = ci >= 0
            self.A[self.rowpos[i]] += np.bincount(ci[msk], weights=off[:, a, :][msk], minlength=n)
        rp = np.where(ci >= 0, self.rowpos[np.maximum(ci, 0)], -1)
        for b, j in enumerate(ri):
            if j < 0:
                continue
            msk = rp >= 0
            if msk.any():
                self.A[:, j] += np.bincount(rp[msk], weights=off[:, b, :][msk], minlength=self.A.shape[0])


def assemble_matrix(mesh: OracleMesh, s: float, orders: QuadOrders = QuadOrders(),
                    dof_mode: str = "interior", rows=None, chunk: int = 4096, regional: bool = False,
                    far_offdiag: bool = True, self_term: str = "pairs"):
    """Dense A^s (or the rows `rows` of it) in the DOF numbering of mesh.dofs().

    Returns (A, vertex_of_dof).  Loops over elements K in index order and, for
    each, over partner elements K' and boundary facets e (Section 5).
    regional=True drops the boundary term, which gives the regional fractional
    Laplacian of Section 2.  far_offdiag=False leaves out the off-diagonal blocks
    -C ∬ phi_i(x) phi_j(y) k of the separated pairs at vertex-graph distance >= 2
    (the far field of Section 6) and keeps everything else, their diagonal-block
    terms included: the sparse near-field part N of A = N + F.

    self_term="near_region" computes the diagonal blocks from local data only, as the
    near-field assembly of the cluster method needs (Section 6: the near field is assembled
    by local computations).  For x in K, the far pairs' diagonal-block terms and the
    boundary term add up to C ∫_{R^d minus N(K)} |x-y|^{-d-2s} dy, N(K) the union of K and
    the cells touching it or at vertex-graph distance 1 (these pairs stay as they are); by
    the divergence theorem that is C/(2s) times the integral over the boundary of N(K) of
    n·(x-y)|x-y|^{-d-2s}, n pointing into N(K).  Its facets that share a vertex with K are
    boundary facets of Omega and keep the singular rules of the boundary term; the others
    take Gauss order k_near (vertex-graph distance 1 from K) or k_far.  Only the diagonal
    blocks change: the entries of two DOFs whose supports share no cell are those of
    "pairs"."""
    if not 0.0 < s < 1.0:
        raise ValueError("s must lie in (0, 1)")
    if self_term not in ("pairs", "near_region"):
        raise ValueError(self_term)
    near_region = self_term == "near_region"
    if near_region and regional:
        raise ValueError("the near-region form includes the boundary term; regional=True is not supported")
    d = mesh.dim
    if d == 2 and dof_mode == "paper" and s < 0.5 and not regional:
        raise NotImplementedError("2D boundary DOFs (paper mode, s < 1/2) are not supported")
    C = frac_constant(d, s)
    vod, dov = mesh.dofs(s, dof_mode)
    n = len(vod)
    rows = np.arange(n) if rows is None else np.asarray(rows, dtype=np.int64)
    sink = _Sink(n, rows, dov)
    nc = mesh.nc
    has_dof = (dov[mesh.C] >= 0).any(axis=1)
    active = np.zeros(nc, dtype=bool)
    for r in rows:
        active[mesh.cells_of_vertex[vod[r]]] = True
    blocks = np.zeros((nc, d + 1, d + 1))  # per-cell sums of the diagonal-block terms
    idx = np.arange(nc)
    for k in range(nc):
        if not active[k]:
            continue
        shared, near = mesh.classify_cells(k)
        partner = (idx != k) & ~(active & (idx < k)) & (has_dof | has_dof[k])
        # touching pairs
        # (the rules depend on vertex labels, so the lower cell index always plays K)
        for m in np.nonzero(partner & (shared > 0))[0]:
            lo, hi = min(k, m), max(k, m)
            if d == 1:
                loc, blk = common_vertex_1d(mesh, s, C, lo, hi, orders.k_touch)
            elif shared[m] == 2:
                loc, blk = common_edge_2d(mesh, s, C, lo, hi, orders.k_touch)
            else:
                loc, blk = common_vertex_2d(mesh, s, C, lo, hi, orders.k_vertex)
            sink.add(loc, loc, blk)
        # separated pairs (with near_region, the far pairs' diagonal-block terms are left to
        # the boundary of N(K) below)
        for sel, order, keep_off, keep_diag in (((shared == 0) & near, orders.k_near, True, True),
                                                ((shared == 0) & ~near, orders.k_far, far_offdiag, not near_region)):
            ms = np.nonzero(partner & sel)[0]
            for c0 in range(0, len(ms), chunk):
                mm = ms[c0:c0 + chunk]
                off, blk_k, blk_m = separated_blocks(mesh, s, C, k, mm, order)
                if keep_diag:
                    blocks[k] += blk_k
                    blocks[mm] += blk_m
                if keep_off:
                    sink.add_off(mesh.C[k], mesh.C[mm], off)
        # identical pair
        if has_dof[k]:
            loc, blk = identical_1d(mesh, s, C, k) if d == 1 else identical_2d(mesh, s, C, k, 2 * orders.k_touch)
            sink.add(loc, loc, blk)
        if has_dof[k] and near_region:
            Y0, Y1, nrm, flen, verts, bidx = near_region_facets(mesh, k)
            m0, m1 = mesh.rings(k)
            fsh = m0[verts].sum(axis=1)
            fnear = (fsh == 0) & m1[verts].any(axis=1)
            for q in np.nonzero(fsh > 0)[0]:
                f = int(bidx[q])
                if f < 0:
                    raise AssertionError("a facet between two cells of N(K) cannot touch K")
                if d == 1:
                    loc, blk = boundary_touch_1d(mesh, s, C, k, f, dov[mesh.facets[f, 0]] >= 0)
                elif fsh[q] == 2:
                    loc, blk = boundary_own_edge_2d(mesh, s, C, k, f, orders.k_bnd)
                else:
                    loc, blk = boundary_vertex_2d(mesh, s, C, k, f, orders.k_bnd)
                sink.add(loc, loc, blk)
            for sel, order in ((fnear, orders.k_near), (~fnear & (fsh == 0), orders.k_far)):
                if sel.any():
                    blocks[k] += facet_sum(mesh, s, C, k, Y0[sel], Y1[sel], nrm[sel], flen[sel], order)
        elif has_dof[k] and not regional:
            # boundary facets
            fsh, fnear = mesh.classify_facets(k)
            for f in np.nonzero(fsh > 0)[0]:
                if d == 1:
                    e = mesh.facets[f, 0]
                    loc, blk = boundary_touch_1d(mesh, s, C, k, f, dov[e] >= 0)
                elif fsh[f] == 2:
                    loc, blk = boundary_own_edge_2d(mesh, s, C, k, f, orders.k_bnd)
                else:
                    loc, blk = boundary_vertex_2d(mesh, s, C, k, f, orders.k_bnd)
                sink.add(loc, loc, blk)
            for sel, order in ((fnear & (fsh == 0), orders.k_near), (~fnear & (fsh == 0), orders.k_far)):
                fs = np.nonzero(sel)[0]
                if len(fs):
                    blocks[k] += boundary_separated(mesh, s, C, k, fs, order)
    for k in range(nc):
        if has_dof[k]:
            sink.add(mesh.C[k], mesh.C[k], blocks[k])
    return sink.A, vod


def nearfield_pattern(mesh: OracleMesh, s: float, dof_mode: str = "interior"):
    """Boolean n x n: (i, j) such that some cell of supp phi_i shares a vertex with, or
    lies at vertex-graph distance 1 from, some cell of supp phi_j (pure combinatorics)."""
    vod, dov = mesh.dofs(s, dof_mode)
    n = len(vod)
    close = np.zeros((mesh.nc, mesh.nc), dtype=bool)  # cell pairs touching or near
    for k in range(mesh.nc):
        shared, near = mesh.classify_cells(k)
        close[k] = (shared > 0) | near
    # cells of each DOF's support
    S = np.zeros((n, mesh.nc), dtype=bool)
    for i, v in enumerate(vod):
        S[i, mesh.cells_of_vertex[v]] = True
    Si = S.astype(np.int64)
    return (Si @ close.astype(np.int64) @ Si.T) > 0


def load_vector(mesh: OracleMesh, s: float, f_nodal=None, dof_mode: str = "interior"):
    """b_i = ∫ f phi_i.  f = 1 when f_nodal is None (b_i = Σ_{K∋i} |K|/(d+1));
    otherwise f is the P1 interpolant of the nodal values, b = M f (P1 mass matrix)."""
    vod, dov = mesh.dofs(s, dof_mode)
    n = len(vod)
    d = mesh.dim
    if f_nodal is None:
        b = np.zeros(n)
        for k in range(mesh.nc):
            for v in mesh.C[k]:
                if dov[v] >= 0:
                    b[dov[v]] += mesh.vol[k] / (d + 1)
        return b
    F = np.asarray(f_nodal, dtype=np.float64)
    one_col = F.ndim == 1
    F = F.reshape(mesh.nv, -1)
    b = np.zeros((n, F.shape[1]))
    Mloc = (np.ones((d + 1, d + 1)) + np.eye(d + 1)) / ((d + 1) * (d + 2))
    for k in range(mesh.nc):
        cell = mesh.C[k]
        contrib = mesh.vol[k] * Mloc @ F[cell]
        for a, v in enumerate(cell):
            if dov[v] >= 0:
                b[dov[v]] += contrib[a]
    return b[:, 0] if one_col else b
