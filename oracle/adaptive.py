"""Adaptive refinement (Section 4, Appendix A): the strong form of the fractional Laplacian
of a finite element function, the Babuska-Rheinboldt indicators and maximum marking
(oracle; test infrastructure only).

Lemma 4.1 (proved in Appendix A) turns (-Delta)^s u(x) for u in V_h and x inside an element
K0 into regular integrals over element boundaries: eq. (8) for s != 1 - d/2, eq. (9) (a
logarithmic kernel) for s = 1 - d/2, i.e. s = 1/2 in 1D.  n_y is the outward normal of the
element whose boundary is integrated.  Here the formula is evaluated literally: for every
point, the boundary of K0 and, for every other element K, its boundary, each edge by Gauss
quadrature (in 1D the boundaries are two points): of order k_near on the three edges of K0
(whichever element's boundary they are part of), where |x - y| gets small, and of order
k_edge on every other edge.  The points are those of the cell rule of order k_cell
(collapsed Gauss in 2D, Gauss in 1D).

The indicators (eq. BRindicators) are eta_i^2 = sum_{K in S_i} h_K^{2s} ||f - (-Delta)^s u||^2_{L2(K)}
over the patch S_i of the elements containing node i, the L2 norms by the same cell rule;
h_K is the diameter (longest edge) of K.  Maximum marking with threshold theta (Section 7:
0.8) marks the nodes with eta_i >= theta max_j eta_j; their patches are refined.
"""
from __future__ import annotations

import math

import numpy as np

from . import rules
from .assemble import frac_constant
from .mesh import OracleMesh


def _nodal(mesh: OracleMesh, s: float, u_dof, dof_mode="interior"):
    vod, _ = mesh.dofs(s, dof_mode)
    u = np.zeros(mesh.nv)
    u[vod] = u_dof
    return u


def cell_rule_points(mesh: OracleMesh, k_cell: int):
    """Points [nc, q, d] and weights [nc, q] of the cell rule of order k_cell on every cell,
    with the reference coordinates [q, d]."""
    if mesh.dim == 1:
        t, w = rules.gauss01(k_cell)
        a = mesh.V[mesh.C[:, 0], 0]
        b = mesh.V[mesh.C[:, 1], 0]
        x = a[:, None] + (b - a)[:, None] * t[None, :]
        return x[..., None], w[None, :] * (b - a)[:, None], t[:, None]
    lam, w = rules.triangle(k_cell)
    P = mesh.V[mesh.C]
    x = P[:, None, 0] + lam[None, :, 0:1] * (P[:, None, 1] - P[:, None, 0]) + \
        lam[None, :, 1:2] * (P[:, None, 2] - P[:, None, 0])
    return x, w[None, :] * 2.0 * mesh.vol[:, None], lam


def _gradient(mesh: OracleMesh, k, u):
    """Gradient of the linear function with nodal values u on cell k."""
    cell = mesh.C[k]
    if mesh.dim == 1:
        return np.array([(u[cell[1]] - u[cell[0]]) / (mesh.V[cell[1], 0] - mesh.V[cell[0], 0])])
    P = mesh.V[cell]
    J = np.array([P[1] - P[0], P[2] - P[0]])  # rows: edge vectors
    return np.linalg.solve(J, np.array([u[cell[1]] - u[cell[0]], u[cell[2]] - u[cell[0]]]))


def _boundary_arrays(mesh: OracleMesh, k_edge):
    """Quadrature on the boundaries of all cells, one row per (cell, facet): vertex keys
    [nc, F, 2] (sorted ids; 1D: the vertex twice), points [nc, F, g, d], weights [nc, F, g],
    outward normals [nc, F, d], nodal interpolation weights [nc, F, g, d+1]."""
    nc, d = mesh.nc, mesh.dim
    if d == 1:
        keys = np.stack([np.stack([mesh.C[:, 0], mesh.C[:, 0]], 1), np.stack([mesh.C[:, 1], mesh.C[:, 1]], 1)], 1)
        Y = mesh.V[mesh.C][:, :, None, :]                    # [nc, 2, 1, 1]
        W = np.ones((nc, 2, 1))
        N = np.tile(np.array([[-1.0], [1.0]]), (nc, 1, 1))
        B = np.zeros((nc, 2, 1, 2))
        B[:, 0, 0, 0] = 1.0
        B[:, 1, 0, 1] = 1.0
        return keys, Y, W, N, B
    t, w = rules.gauss01(k_edge)
    P = mesh.V[mesh.C]                                        # [nc, 3, 2]
    centroid = P.mean(axis=1)
    keys, Y, W, N, B = [], [], [], [], []
    for a, b in ((0, 1), (1, 2), (2, 0)):
        e = P[:, b] - P[:, a]
        L = np.hypot(e[:, 0], e[:, 1])
        n = np.stack([e[:, 1], -e[:, 0]], 1) / L[:, None]
        flip = np.sum(n * (P[:, a] - centroid), axis=1) < 0
        n[flip] = -n[flip]
        keys.append(np.sort(np.stack([mesh.C[:, a], mesh.C[:, b]], 1), axis=1))
        Y.append(P[:, a, None, :] + t[None, :, None] * e[:, None, :])
        W.append(w[None, :] * L[:, None])
        N.append(n)
        bary = np.zeros((nc, len(t), 3))
        bary[:, :, a] = 1.0 - t[None, :]
        bary[:, :, b] = t[None, :]
        B.append(bary)
    return np.stack(keys, 1), np.stack(Y, 1), np.stack(W, 1), np.stack(N, 1), np.stack(B, 1)


def strong_form(mesh: OracleMesh, s: float, u_dof, k_cell: int = 3, k_edge: int = 4, k_near: int = 16,
                dof_mode: str = "interior", cells=None, with_abs: bool = False):
    """(-Delta)^s u_h at the cell-rule points of every cell: [nc, q] (Lemma 4.1); with `cells`,
    only at the points of those cells: [len(cells), q].  with_abs: also C times the sum of the
    absolute values of all terms at each point (the size of what the sum cancels, which sets the
    rounding error of any evaluation of it, this one included)."""
    d = mesh.dim
    C = frac_constant(d, s)
    u = _nodal(mesh, s, u_dof, dof_mode)
    X, _, ref = cell_rule_points(mesh, k_cell)
    q = X.shape[1]
    log_case = abs(s - (1.0 - d / 2.0)) < 1e-14
    m = d + 2.0 * s - 2.0
    grads = np.array([_gradient(mesh, k, u) for k in range(mesh.nc)])      # [nc, d]
    far = _boundary_arrays(mesh, k_edge)
    near = _boundary_arrays(mesh, k_near)
    keys = far[0]
    all_cells = np.arange(mesh.nc)
    cells = all_cells if cells is None else np.asarray(cells)
    out = np.zeros((len(cells), q))
    out_abs = np.zeros((len(cells), q))

    def terms(x, ux, arrays, sel, k0, idx):
        """The integrals over the facets sel ([nc, F] mask) of the boundaries of the cells idx,
        with the weights of eq. (8)/(9): 1/m (log case: 1) and -u(x)/(2s) on K0's own boundary,
        1/(2s m) (log case: 1/(2s)) and -u(y)/(2s) on every other cell's boundary."""
        Y, W, N, B = (a[idx] for a in arrays[1:])
        sel = sel[idx]
        diff = x - Y                                          # [cells, F, g, d]
        r = np.sqrt(np.sum(diff * diff, axis=-1))
        gn = np.sum(N * grads[idx][:, None, :], axis=-1)      # [cells, F]
        nd = np.sum(N[:, :, None, :] * diff, axis=-1)         # [cells, F, g]
        kern = np.log(1.0 / r) if log_case else r ** (-m)
        g_int = np.sum(W * kern, axis=-1) * gn                # [cells, F]
        uy = np.einsum("kfgv,kv->kfg", B, u[mesh.C[idx]])
        own = idx == k0
        g_w = np.where(own, 1.0 if log_case else 1.0 / m, 1.0 / (2.0 * s) if log_case else 1.0 / (2.0 * s * m))
        val = np.sum(np.where(sel, g_int * g_w[:, None], 0.0))
        g_abs = np.sum(np.where(sel, np.abs(np.sum(W * kern, axis=-1) * gn * g_w[:, None]), 0.0))
        u_int = np.sum(W * nd / r ** (d + 2.0 * s) * uy, axis=-1)       # other cells: u(y)
        o_int = np.sum(W * nd / r ** (d + 2.0 * s), axis=-1)            # own cell: times u(x)
        u_abs = np.sum(np.abs(W * nd / r ** (d + 2.0 * s)) * np.where(own[:, None, None], abs(ux), np.abs(uy)), axis=-1)
        g_abs += np.sum(np.where(sel, u_abs, 0.0)) / (2.0 * s)
        return val, np.where(sel & ~own[:, None], u_int, 0.0), np.where(sel & own[:, None], o_int, 0.0), g_abs

    for row, k0 in enumerate(cells):
        # facets of K0, whichever cell's boundary they are part of
        sel_near = np.any(np.all(keys[:, :, None, :] == keys[k0][None, None, :, :], axis=-1), axis=-1)  # [nc, F]
        near_cells = np.nonzero(sel_near.any(axis=1))[0]
        for a in range(q):
            x = X[k0, a]
            if d == 1:
                lam = np.array([1.0 - ref[a, 0], ref[a, 0]])
            else:
                lam = np.array([1.0 - ref[a, 0] - ref[a, 1], ref[a, 0], ref[a, 1]])
            ux = lam @ u[mesh.C[k0]]
            val = 0.0
            size = 0.0
            for arrays, sel, idx in ((far, ~sel_near, all_cells), (near, sel_near, near_cells)):
                v, u_other, own_int, g_abs = terms(x, ux, arrays, sel, k0, idx)
                val += v - np.sum(u_other) / (2.0 * s) - ux / (2.0 * s) * np.sum(own_int)
                size += g_abs
            out[row, a] = C * val
            out_abs[row, a] = abs(C) * size
    return (out, out_abs) if with_abs else out


def cell_diameters(mesh: OracleMesh):
    """h_K: the longest edge (2D) or the length (1D) of every cell."""
    P = mesh.V[mesh.C]
    if mesh.dim == 1:
        return P[:, 1, 0] - P[:, 0, 0]
    e = [np.linalg.norm(P[:, b] - P[:, a], axis=1) for a, b in ((0, 1), (1, 2), (2, 0))]
    return np.maximum(np.maximum(e[0], e[1]), e[2])


def br_indicators(mesh: OracleMesh, s: float, u_dof, f_nodal=None, k_cell: int = 3, k_edge: int = 4,
                  k_near: int = 16, dof_mode: str = "interior"):
    """eta_i for the DOFs of mesh.dofs(): sqrt(sum_{K in S_i} h_K^{2s} ||f - (-Delta)^s u_h||_{L2(K)}^2);
    f = 1 when f_nodal is None, else the P1 interpolant of the nodal values."""
    S = strong_form(mesh, s, u_dof, k_cell, k_edge, k_near, dof_mode)
    X, W, ref = cell_rule_points(mesh, k_cell)
    if f_nodal is None:
        fx = np.ones_like(S)
    else:
        f = np.asarray(f_nodal, dtype=np.float64)
        if mesh.dim == 1:
            lam = np.stack([1.0 - ref[:, 0], ref[:, 0]], axis=1)
        else:
            lam = np.stack([1.0 - ref[:, 0] - ref[:, 1], ref[:, 0], ref[:, 1]], axis=1)
        fx = f[mesh.C] @ lam.T
    cell_err = cell_diameters(mesh) ** (2.0 * s) * np.sum(W * (fx - S) ** 2, axis=1)
    vod, _ = mesh.dofs(s, dof_mode)
    eta2 = np.array([sum(cell_err[k] for k in mesh.cells_of_vertex[v]) for v in vod])
    return np.sqrt(eta2)


def mark_max(eta, theta: float = 0.8):
    """Nodes i with eta_i >= theta max_j eta_j (maximum marking)."""
    eta = np.asarray(eta)
    return eta >= theta * eta.max()


def marked_cells(mesh: OracleMesh, s: float, node_marks, dof_mode: str = "interior"):
    """Cells of the patches S_i of the marked nodes, ascending."""
    vod, _ = mesh.dofs(s, dof_mode)
    cells = set()
    for i in np.nonzero(node_marks)[0]:
        cells.update(mesh.cells_of_vertex[vod[i]])
    return np.array(sorted(cells), dtype=np.int64)


def refine(vertices, cells, cell_marks):
    """Conforming refinement of the marked cells (Section 7: refinement without hanging nodes).

    1D: every marked interval is split at its midpoint.  2D: newest-vertex bisection.  A
    triangle (v0, v1, v2) has newest vertex v0 and refinement edge {v1, v2}; bisecting it at
    the midpoint m of that edge gives (m, v0, v1) and (m, v2, v0).  Written here through the
    set B of edges to be halved: B starts with the refinement edges of the marked cells and is
    closed by adding the refinement edge of every cell that has an edge in B (so no edge is
    halved on one side only); then every cell whose refinement edge is in B is bisected, and
    each child again if its refinement edge (an edge of the parent) is in B.  The result does
    not depend on the order of the cells.  Returns (vertices, cells): old vertices first, then
    the midpoints in order of creation; the children replace their parent in place."""
    V = [tuple(float(c) for c in p) for p in np.asarray(vertices, dtype=np.float64).reshape(len(vertices), -1)]
    T = [tuple(int(c) for c in t) for t in np.asarray(cells)]
    marks = np.asarray(cell_marks, dtype=bool)
    mid = {}

    def midpoint(a, b):
        key = (min(a, b), max(a, b))
        if key not in mid:
            V.append(tuple((x + y) / 2.0 for x, y in zip(V[a], V[b])))
            mid[key] = len(V) - 1
        return mid[key]

    if len(V[0]) == 1:
        out = []
        for t, mk in zip(T, marks):
            if mk:
                m = midpoint(t[0], t[1])
                out += [(t[0], m), (m, t[1])]
            else:
                out.append(t)
        return np.array(V, dtype=np.float64), np.array(out, dtype=np.int64)

    def ekey(a, b):
        return (min(a, b), max(a, b))

    B = {ekey(t[1], t[2]) for t, mk in zip(T, marks) if mk}
    while True:
        grown = False
        for t in T:
            if ekey(t[1], t[2]) in B:
                continue
            if ekey(t[0], t[1]) in B or ekey(t[0], t[2]) in B:
                B.add(ekey(t[1], t[2]))
                grown = True
        if not grown:
            break

    def split(t):
        if ekey(t[1], t[2]) not in B:
            return [t]
        m = midpoint(t[1], t[2])
        return split((m, t[0], t[1])) + split((m, t[2], t[0]))

    out = []
    for t in T:
        out += split(t)
    return np.array(V, dtype=np.float64), np.array(out, dtype=np.int64)
