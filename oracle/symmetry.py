"""Symmetry reduction (Section 7, "Exploiting Symmetry"; oracle, test infrastructure only).

Omega is invariant under the rotation B by 2 pi / K about the origin, B^K = Id, and the data
f (hence u) are too.  Only the sector omega = {r <= 1, 0 <= phi <= 2 pi / K} is meshed; the
whole mesh is its K rotated copies.  The reduced problem is the Galerkin problem on the
periodic subspace of V_h: a degree of freedom of the reduced problem is an orbit
{B^l v} of degrees of freedom of the whole mesh, its basis function the sum of their hat
functions.  With P the (whole DOF) x (orbit) incidence matrix, the whole mesh's A and b,

    A_red = P^T A P / K,   b_red = P^T b / K,

the paper's bilinear form with the effective kernel k_eff(x, y) = sum_l |x - B^l y|^{-d-2s}
over omega x omega divided by K, and the same division for <f, v> = K int_omega f v.  The
reduced solution is the periodic whole-mesh solution restricted to the orbit representatives.
The whole-mesh matrix comes from the element-pair oracle (assemble.py) unchanged: this module
only builds the copies and folds.

Only the rows of the orbit representatives are needed: with exact integrals A is invariant
under the rotation, so P^T A P / K has entries (|O_r| / K) sum_{j in O_c} A[rep_r, j].  The
quadrature is invariant only up to its own error (the singular rules of touching pairs depend
on which cell of the pair comes first, and the copies number the cells differently: 3e-7 of
the entries on the 8-fold sector), so the reduced matrix is read as the symmetric part of that
row formula (reduced_system); fold_system gives P^T A P / K itself.

Orbit numbering: an orbit is represented by the lowest sector vertex id among its copy-0
vertices (a vertex on the ray phi = 0 and its image on phi = 2 pi / K belong to one orbit; the
centre is an orbit of its own); orbits are numbered by that id, ascending.
"""
from __future__ import annotations

import math

import numpy as np

from .assemble import assemble_matrix, load_vector
from .mesh import OracleMesh


def replicate(vertices, cells, K: int, tol: float = 1e-10):
    """The K rotated copies of a sector mesh, coincident vertices merged.

    Returns (V, C, vmap, cell_copy): vmap[l, v] = vertex of the whole mesh that is copy l of
    sector vertex v; cells of copy l follow those of copy l - 1 in the sector's order."""
    Vs = np.asarray(vertices, dtype=np.float64)
    Cs = np.asarray(cells, dtype=np.int64)
    nv = len(Vs)
    V = []
    vmap = np.zeros((K, nv), dtype=np.int64)
    for l in range(K):
        c, s = math.cos(2 * math.pi * l / K), math.sin(2 * math.pi * l / K)
        R = np.array([[c, -s], [s, c]])
        for v in range(nv):
            p = R @ Vs[v]
            # an earlier vertex at the same place (plain search: meshes here are small)
            hit = -1
            for w in range(len(V)):
                if abs(V[w][0] - p[0]) <= tol and abs(V[w][1] - p[1]) <= tol:
                    hit = w
                    break
            if hit < 0:
                V.append(p)
                hit = len(V) - 1
            vmap[l, v] = hit
    C = np.concatenate([vmap[l][Cs] for l in range(K)])
    cell_copy = np.repeat(np.arange(K), len(Cs))
    return np.array(V), C, vmap, cell_copy


def orbits(vertices, cells, K: int, s: float, dof_mode: str = "interior"):
    """Orbits of the whole mesh's degrees of freedom.

    Returns (mesh, P, reps): the whole OracleMesh, P [n_whole, n_red] (0/1 incidence of whole
    DOFs in orbits) and reps[r] = the sector vertex that represents orbit r."""
    V, C, vmap, _ = replicate(vertices, cells, K)
    mesh = OracleMesh(V, C)
    vod, dov = mesh.dofs(s, dof_mode)
    nvs = vmap.shape[1]
    # orbit of a whole vertex: the lowest sector vertex whose copy-0 image shares the orbit
    orbit_of_vertex = {}
    for v in range(nvs):
        members = set(int(vmap[l, v]) for l in range(K))
        key = min(u for u in range(nvs) if int(vmap[0, u]) in members)
        for w in members:
            orbit_of_vertex[w] = key
    reps = sorted({orbit_of_vertex[int(w)] for w in vod})
    col = {r: k for k, r in enumerate(reps)}
    P = np.zeros((len(vod), len(reps)))
    for i, w in enumerate(vod):
        P[i, col[orbit_of_vertex[int(w)]]] = 1.0
    return mesh, P, np.array(reps, dtype=np.int64)


def _whole_f(vertices, cells, K, mesh, f_sector):
    if f_sector is None:
        return None
    _, _, vmap, _ = replicate(vertices, cells, K)
    f = np.zeros(mesh.nv)
    for l in range(K):
        f[vmap[l]] = np.asarray(f_sector, dtype=np.float64)
    return f


def fold_system(vertices, cells, K: int, s: float, f_sector=None, dof_mode: str = "interior", **orders):
    """(P^T A P / K, P^T b / K, reps) from the whole mesh's full matrix."""
    mesh, P, reps = orbits(vertices, cells, K, s, dof_mode)
    A, _ = assemble_matrix(mesh, s, dof_mode=dof_mode, **orders)
    b = load_vector(mesh, s, _whole_f(vertices, cells, K, mesh, f_sector), dof_mode)
    return P.T @ A @ P / K, P.T @ b / K, reps


def reduced_system(vertices, cells, K: int, s: float, f_sector=None, dof_mode: str = "interior", **orders):
    """(A_red, b_red, reps): the reduced matrix, the symmetric part of
    (|O_r| / K) sum_{j in O_c} A[rep_r, j] from the representatives' rows of the whole matrix,
    and the load vector P^T b / K.  f_sector: None (f = 1) or the nodal values of f on the
    sector's vertices (f periodic, so its copies carry the same values)."""
    mesh, P, reps = orbits(vertices, cells, K, s, dof_mode)
    vod, dov = mesh.dofs(s, dof_mode)
    _, _, vmap, _ = replicate(vertices, cells, K)
    rep_rows = dov[vmap[0][reps]]
    A_rows, _ = assemble_matrix(mesh, s, dof_mode=dof_mode, rows=rep_rows, **orders)
    size = P.sum(axis=0)
    R = (size / K)[:, None] * (A_rows @ P)
    b = load_vector(mesh, s, _whole_f(vertices, cells, K, mesh, f_sector), dof_mode)
    return (R + R.T) / 2.0, P.T @ b / K, reps


def reduced_system_keff(vertices, cells, K: int, s: float, f_sector=None, dof_mode: str = "interior", orders=None):
    """(A_red, b_red, reps) in Section 7's effective-kernel form: the sector's cells against the
    K images of the sector's cells, each orbit of element pairs of the whole mesh (under the
    rotation) evaluated once.  With the whole mesh's cells numbered copy by copy (copy l of sector
    cell k is cell l n_s + k), an orbit of unordered pairs is represented by (k, copy l of k') with
    k < k' and any l, or k = k' and 1 <= l <= K / 2 (l = K / 2 is an orbit of K / 2 pairs: weight
    1/2); every cell once for the identical pair and the boundary term.  Each representative's full
    contribution (both off-diagonal blocks and both diagonal-block terms) is added in orbit
    coordinates, so A_red = P^T A P / K exactly for a rotation-invariant quadrature; the oracle's
    touching rules take the lower cell index as K, which rotation does not preserve, so the two
    differ by the quadrature error of those pairs.  b_red = P^T b / K.  2D rotations only."""
    from .assemble import (QuadOrders, boundary_own_edge_2d, boundary_separated, boundary_vertex_2d,
                           common_edge_2d, common_vertex_2d, frac_constant, identical_2d, separated_blocks)

    orders = orders or QuadOrders()
    Cs = np.asarray(cells)
    ns = len(Cs)
    mesh, P, reps = orbits(vertices, cells, K, s, dof_mode)
    if mesh.dim != 2:
        raise ValueError("rotations of a 2D sector only")
    vod, dov = mesh.dofs(s, dof_mode)
    orb = -np.ones(mesh.nv, dtype=np.int64)
    orb[vod] = np.argmax(P, axis=1)
    n_red = P.shape[1]
    A = np.zeros((n_red, n_red))
    C = frac_constant(2, s)
    has_dof = (dov[mesh.C] >= 0).any(axis=1)

    def add(rv, cv, blk, w=1.0):
        for a, vi in enumerate(rv):
            oi = orb[vi]
            if oi < 0:
                continue
            for b, vj in enumerate(cv):
                oj = orb[vj]
                if oj >= 0:
                    A[oi, oj] += w * blk[a, b]

    nc = mesh.nc
    idx = np.arange(nc)
    for k in range(ns):
        kk, ll = idx % ns, idx // ns
        rep = (kk > k) | ((kk == k) & (ll >= 1) & (2 * ll <= K))
        weight = np.where((kk == k) & (2 * ll == K), 0.5, 1.0)
        shared, near = mesh.classify_cells(k)
        partner = rep & (has_dof | has_dof[k])
        for m in np.nonzero(partner & (shared > 0))[0]:
            lo, hi = min(k, m), max(k, m)
            if shared[m] == 2:
                loc, blk = common_edge_2d(mesh, s, C, lo, hi, orders.k_touch)
            else:
                loc, blk = common_vertex_2d(mesh, s, C, lo, hi, orders.k_vertex)
            add(loc, loc, blk, weight[m])
        for sel, order in (((shared == 0) & near, orders.k_near), ((shared == 0) & ~near, orders.k_far)):
            for m in np.nonzero(partner & sel)[0]:
                off, blk_k, blk_m = separated_blocks(mesh, s, C, k, np.array([m]), order)
                w = weight[m]
                add(mesh.C[k], mesh.C[m], off[0], w)
                add(mesh.C[m], mesh.C[k], off[0].T, w)
                add(mesh.C[k], mesh.C[k], blk_k, w)
                add(mesh.C[m], mesh.C[m], blk_m[0], w)
        if has_dof[k]:
            loc, blk = identical_2d(mesh, s, C, k, 2 * orders.k_touch)
            add(loc, loc, blk)
            fsh, fnear = mesh.classify_facets(k)
            for f in np.nonzero(fsh > 0)[0]:
                if fsh[f] == 2:
                    loc, blk = boundary_own_edge_2d(mesh, s, C, k, f, orders.k_bnd)
                else:
                    loc, blk = boundary_vertex_2d(mesh, s, C, k, f, orders.k_bnd)
                add(loc, loc, blk)
            for sel, order in ((fnear & (fsh == 0), orders.k_near), (~fnear & (fsh == 0), orders.k_far)):
                fs = np.nonzero(sel)[0]
                if len(fs):
                    add(mesh.C[k], mesh.C[k], boundary_separated(mesh, s, C, k, fs, order))
    b = load_vector(mesh, s, _whole_f(vertices, cells, K, mesh, f_sector), dof_mode)
    return A, P.T @ b / K, reps
