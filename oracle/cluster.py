"""Cluster method (Section 6): hierarchical cluster tree, admissible cluster pairs and
the Chebyshev approximation of the far field (oracle; test infrastructure only).

Section 6 (following Sauter and Schwab, Ch. 7) approximates a(phi, psi) on an admissible
pair of clusters (sigma, tau), where the supports are disjoint and
a(phi, psi) = -C(d,s) int int k(x,y) phi(x) psi(y), by interpolating the kernel
k(x,y) = |x-y|^{-d-2s} with tensor Chebyshev polynomials of order m on the two cluster
boxes; the far-field coefficients int phi L_alpha are computed on the leaves by Gauss
quadrature of order m+1 and moved up the tree with the shift coefficients
L_alpha^sigma(xi_beta^tau).  Inadmissible pairs of leaves form the near field, kept as
exact matrix entries.  The matrix-vector product is near-field product + upward pass +
kernel couplings + downward pass.

Readings (the paper leaves these open):
* leaves hold at most `leaf` DOFs (leaf = 1 gives the single-index leaves of the paper's
  definition); a cluster with more is split in two by the coordinate of its DOF vertices
  along the longest side of their bounding box (ties: the lowest axis) at the middle of
  that side, DOFs strictly below the middle going to the first son; should one son be
  empty, the DOFs sorted by (coordinate, index) are split at the median instead;
* the cluster box is the smallest hyper-cube containing the supports of the cluster's
  basis functions, centred on their bounding box; its diameter is side * sqrt(d), the
  distance of two clusters that of their cubes;
* the admissible pairs come from the recursion over pairs started at (root, root): an
  admissible pair is kept, a pair of leaves is near field, otherwise the non-leaf
  clusters of the pair are replaced by their sons (both when both are not leaves);
* Chebyshev points of order m on [c - L/2, c + L/2]: c + (L/2) cos((2k - 1) pi / (2m)),
  k = 1..m; tensor index alpha = alpha_0 * m + alpha_1 in 2D.
Everything is float64 and deliberately plain (Python loops over clusters and blocks).
"""
from __future__ import annotations

import math

import numpy as np

from . import rules
from .assemble import frac_constant
from .mesh import OracleMesh


class ClusterTree:
    """Nodes in creation order (root first, depth-first, first son before second).

    dofs[c] (DOF indices, tree order), center[c], side[c], sons[c] (list), level[c]."""

    def __init__(self, mesh: OracleMesh, s: float, leaf: int = 32, dof_mode: str = "interior"):
        self.mesh = mesh
        self.d = mesh.dim
        vod, _ = mesh.dofs(s, dof_mode)
        self.vod = vod
        self.n = len(vod)
        X = mesh.V[vod]  # DOF vertex coordinates
        # bounding box of each DOF's support (the cells around its vertex)
        lo = np.empty((self.n, self.d))
        hi = np.empty((self.n, self.d))
        for i, v in enumerate(vod):
            P = mesh.V[mesh.C[mesh.cells_of_vertex[v]].ravel()]
            lo[i] = P.min(axis=0)
            hi[i] = P.max(axis=0)
        self.dofs, self.center, self.side, self.sons, self.level = [], [], [], [], []

        def make(idx, lev):
            c = len(self.dofs)
            blo = lo[idx].min(axis=0)
            bhi = hi[idx].max(axis=0)
            self.dofs.append(np.array(idx, dtype=np.int64))
            self.center.append((blo + bhi) / 2.0)
            self.side.append(float(np.max(bhi - blo)))
            self.sons.append([])
            self.level.append(lev)
            if len(idx) > leaf:
                P = X[idx]
                ext = P.max(axis=0) - P.min(axis=0)
                k = int(np.argmax(ext))  # first maximum: ties go to the lowest axis
                mid = (P[:, k].min() + P[:, k].max()) / 2.0
                first = [i for i in idx if X[i, k] < mid]
                second = [i for i in idx if not X[i, k] < mid]
                if not first or not second:
                    srt = sorted(idx, key=lambda i: (X[i, k], i))
                    h = len(srt) // 2
                    first, second = srt[:h], srt[h:]
                self.sons[c] = [make(first, lev + 1), make(second, lev + 1)]
            return c

        make(list(range(self.n)), 0)
        self.center = np.array(self.center)
        self.side = np.array(self.side)

    def diam(self, c):
        return self.side[c] * math.sqrt(self.d)

    def dist(self, a, b):
        g = np.maximum(0.0, np.abs(self.center[a] - self.center[b]) - (self.side[a] + self.side[b]) / 2.0)
        return float(np.sqrt(np.sum(g * g)))


def block_partition(tree: ClusterTree, eta: float = 1.0):
    """(far, near): lists of cluster pairs (sigma, tau), admissible and near-field leaf pairs,
    in the order of the recursion from (root, root)."""
    far, near = [], []

    def rec(a, b):
        if eta * tree.dist(a, b) >= max(tree.diam(a), tree.diam(b)):
            far.append((a, b))
        elif not tree.sons[a] and not tree.sons[b]:
            near.append((a, b))
        elif not tree.sons[a]:
            for bb in tree.sons[b]:
                rec(a, bb)
        elif not tree.sons[b]:
            for aa in tree.sons[a]:
                rec(aa, b)
        else:
            for aa in tree.sons[a]:
                for bb in tree.sons[b]:
                    rec(aa, bb)

    rec(0, 0)
    return far, near


def cheb_points_1d(c, L, m):
    k = np.arange(1, m + 1)
    return c + 0.5 * L * np.cos((2 * k - 1) * np.pi / (2 * m))


def lagrange_1d(nodes, t):
    """[len(t), m]: the Lagrange basis of `nodes` evaluated at t."""
    t = np.atleast_1d(t)
    m = len(nodes)
    out = np.ones((len(t), m))
    for k in range(m):
        for l in range(m):
            if l != k:
                out[:, k] *= (t - nodes[l]) / (nodes[k] - nodes[l])
    return out


def cheb_points(tree: ClusterTree, c, m):
    """[m^d, d] tensor Chebyshev points of cluster c (alpha = alpha_0 m + alpha_1)."""
    pts = [cheb_points_1d(tree.center[c][k], tree.side[c], m) for k in range(tree.d)]
    if tree.d == 1:
        return pts[0][:, None]
    g0, g1 = np.meshgrid(pts[0], pts[1], indexing="ij")
    return np.stack([g0.ravel(), g1.ravel()], axis=1)


def lagrange(tree: ClusterTree, c, m, x):
    """[len(x), m^d]: tensor Lagrange polynomials L_alpha^c at points x [., d]."""
    x = np.atleast_2d(x)
    Ls = [lagrange_1d(cheb_points_1d(tree.center[c][k], tree.side[c], m), x[:, k]) for k in range(tree.d)]
    if tree.d == 1:
        return Ls[0]
    return (Ls[0][:, :, None] * Ls[1][:, None, :]).reshape(len(x), m * m)


def leaf_coefficients(tree: ClusterTree, c, m):
    """[|c|, m^d]: int phi_i L_alpha^c for the DOFs i of leaf c, Gauss order m+1 per cell."""
    mesh = tree.mesh
    out = np.zeros((len(tree.dofs[c]), m ** tree.d))
    for r, i in enumerate(tree.dofs[c]):
        v = tree.vod[i]
        for K in mesh.cells_of_vertex[v]:
            cell = mesh.C[K]
            a = int(np.nonzero(cell == v)[0][0])
            if tree.d == 1:
                t, w = rules.gauss01(m + 1)
                x0, x1 = mesh.V[cell[0], 0], mesh.V[cell[1], 0]
                x = (x0 + (x1 - x0) * t)[:, None]
                phi = (1.0 - t) if a == 0 else t
                wt = w * (x1 - x0)
            else:
                lam, w = rules.triangle(m + 1)
                P = mesh.V[cell]
                x = P[0] + lam[:, 0:1] * (P[1] - P[0]) + lam[:, 1:2] * (P[2] - P[0])
                phi = rules.p1_shape(lam)[:, a]
                wt = w * 2.0 * mesh.vol[K]
            out[r] += (wt * phi) @ lagrange(tree, c, m, x)
    return out


def shift_matrix(tree: ClusterTree, parent, son, m):
    """[m^d (son), m^d (parent)]: L_alpha^parent(xi_beta^son)."""
    return lagrange(tree, parent, m, cheb_points(tree, son, m))


def kernel_matrix(tree: ClusterTree, a, b, m, s):
    """[m^d, m^d]: k(xi_alpha^a, xi_beta^b) = |xi - xi'|^{-d-2s}."""
    pa, pb = cheb_points(tree, a, m), cheb_points(tree, b, m)
    r2 = np.sum((pa[:, None, :] - pb[None, :, :]) ** 2, axis=-1)
    return r2 ** (-(tree.d + 2.0 * s) / 2.0)


def hmatvec(A, mesh: OracleMesh, s: float, x, m: int = 4, eta: float = 1.0, leaf: int = 32,
            dof_mode: str = "interior"):
    """y ~ A x: exact near-field entries of A on the inadmissible leaf pairs, Chebyshev far
    field of order m on the admissible pairs (upward pass, couplings, downward pass)."""
    tree = ClusterTree(mesh, s, leaf, dof_mode)
    far, near = block_partition(tree, eta)
    x = np.asarray(x, dtype=np.float64)
    y = np.zeros(tree.n)
    for a, b in near:
        ia, ib = tree.dofs[a], tree.dofs[b]
        y[ia] += A[np.ix_(ia, ib)] @ x[ib]
    nc = len(tree.dofs)
    md = m ** tree.d
    coef = {c: leaf_coefficients(tree, c, m) for c in range(nc) if not tree.sons[c]}
    xh = np.zeros((nc, md))
    for c in reversed(range(nc)):  # sons are created after their father
        if tree.sons[c]:
            for sn in tree.sons[c]:
                xh[c] += shift_matrix(tree, c, sn, m).T @ xh[sn]
        else:
            xh[c] = coef[c].T @ x[tree.dofs[c]]
    yh = np.zeros((nc, md))
    for a, b in far:
        yh[a] += kernel_matrix(tree, a, b, m, s) @ xh[b]
    for c in range(nc):  # fathers first
        for sn in tree.sons[c]:
            yh[sn] += shift_matrix(tree, c, sn, m) @ yh[c]
        if not tree.sons[c]:
            y[tree.dofs[c]] += -frac_constant(tree.d, s) * (coef[c] @ yh[c])
    return y


def _far_field_coefficients(tree: ClusterTree, far, s: float, x, m: int):
    """yh[c]: for every node c, sum over the admissible pairs (rho, tau) with rho c or an ancestor
    of c of the kernel couplings of tau's far-field coefficients of x, expanded in c's Chebyshev
    basis (upward pass, couplings, downward pass of the product)."""
    nc = len(tree.dofs)
    md = m ** tree.d
    coef = {c: leaf_coefficients(tree, c, m) for c in range(nc) if not tree.sons[c]}
    xh = np.zeros((nc, md))
    for c in reversed(range(nc)):
        if tree.sons[c]:
            for sn in tree.sons[c]:
                xh[c] += shift_matrix(tree, c, sn, m).T @ xh[sn]
        else:
            xh[c] = coef[c].T @ x[tree.dofs[c]]
    yh = np.zeros((nc, md))
    for a, b in far:
        yh[a] += kernel_matrix(tree, a, b, m, s) @ xh[b]
    for c in range(nc):
        for sn in tree.sons[c]:
            yh[sn] += shift_matrix(tree, c, sn, m) @ yh[c]
    return yh


def strong_form_cluster(mesh: OracleMesh, s: float, u_dof, m: int = 4, eta: float = 1.0, leaf: int = 32,
                        k_cell: int = 3, k_edge: int = 4, k_near: int = 16, dof_mode: str = "interior",
                        cells=None):
    """(-Delta)^s u_h at the cell-rule points of every cell [nc, q] by the cluster method
    (Section 6): for a point x0 of cell K0, i0 the DOF of K0 closest to x0 and sigma its leaf,
    u = u_N + u_F with u_N the part on the DOFs of sigma's inadmissible partners; the strong form
    of u_N is Lemma 4.1's (strong_form with u_N), and that of u_F, whose support lies in
    admissible partners' boxes away from x0, is -C int k(x0, y) u_F(y) dy, approximated by
    Chebyshev interpolation: -C sum_alpha L_alpha^sigma(x0) yh_sigma[alpha], yh from the
    product's upward pass, couplings and downward pass applied to u.

    Readings: ties in "closest" go to the lower DOF index; a cell without a DOF vertex (all its
    vertices on the boundary) belongs to no support, so its points take the strong form of u
    itself (no far part).  With `cells`, only the points of those cells: [len(cells), q]."""
    from .adaptive import cell_rule_points, strong_form

    tree = ClusterTree(mesh, s, leaf, dof_mode)
    far, near = block_partition(tree, eta)
    u_dof = np.asarray(u_dof, dtype=np.float64)
    yh = _far_field_coefficients(tree, far, s, u_dof, m)
    C = frac_constant(tree.d, s)
    leaf_of = np.empty(tree.n, dtype=np.int64)
    for c in range(len(tree.dofs)):
        if not tree.sons[c]:
            leaf_of[tree.dofs[c]] = c
    partners = {}
    for a, b in near:
        partners.setdefault(a, []).append(b)
    _, dov = mesh.dofs(s, dof_mode)
    X, _, _ = cell_rule_points(mesh, k_cell)
    q = X.shape[1]
    cells = np.arange(mesh.nc) if cells is None else np.asarray(cells)
    out = np.zeros((len(cells), q))
    opts = dict(k_cell=k_cell, k_edge=k_edge, k_near=k_near, dof_mode=dof_mode)
    for row, k0 in enumerate(cells):
        dofs = [int(dov[v]) for v in mesh.C[k0] if dov[v] >= 0]
        if not dofs:
            out[row] = strong_form(mesh, s, u_dof, cells=[k0], **opts)[0]
            continue
        cache = {}
        for a in range(q):
            x0 = X[k0, a]
            dist = [float(np.sum((mesh.V[tree.vod[i]] - x0) ** 2)) for i in dofs]
            i0 = min(zip(dist, dofs))[1]
            sigma = int(leaf_of[i0])
            if sigma not in cache:
                uN = np.zeros_like(u_dof)
                for tau in partners.get(sigma, []):
                    uN[tree.dofs[tau]] = u_dof[tree.dofs[tau]]
                cache[sigma] = strong_form(mesh, s, uN, cells=[k0], **opts)[0]
            out[row, a] = cache[sigma][a] - C * float(lagrange(tree, sigma, m, x0[None, :])[0] @ yh[sigma])
    return out
