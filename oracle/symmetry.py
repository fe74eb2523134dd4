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
