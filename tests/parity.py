"""Entry-wise parity measures of a GPU matrix against the oracle's float64 matrix.

An entry a_ij whose DOF supports share no vertex is a sum of single-signed terms
-C ∬ phi_i(x) phi_j(y) |x-y|^{-d-2s} over separated element pairs (Section 5; Section 6
gives the same sign for disjoint supports), so its error is measured relative to the
entry itself.  Entries of touching supports add the singular, identical-element and
boundary terms of both signs; their error is measured relative to sqrt(a_ii a_jj).
"""
import numpy as np
import scipy.sparse as sp


def touching_mask(om, s, dof_mode="interior"):
    """n x n bool: DOF pairs (i, j) such that a cell of supp phi_i shares a vertex with a
    cell of supp phi_j (pure combinatorics on the oracle's mesh)."""
    vod, _ = om.dofs(s, dof_mode)
    nc, k = om.C.shape
    S = sp.csr_matrix((np.ones(nc * k), (np.repeat(np.arange(nc), k), om.C.ravel())), shape=(nc, om.nv))
    N = ((S.T @ S) > 0).astype(np.int64)  # vertices that share a cell
    T = ((N @ N) > 0).tocsr()  # vertices whose stars share a vertex
    return np.asarray(T[vod][:, vod].todense())


def f64_errors(Ag, Ao, touch, diag_rows, diag_all):
    """(max |Ag - Ao| / |Ao| over disjoint-support entries, max |Ag - Ao| / sqrt(a_ii a_jj)
    over touching entries) for rows Ag, Ao [r, n], their touching mask [r, n] and the
    diagonals of those rows [r] and of the whole matrix [n]."""
    Ag = np.asarray(Ag, dtype=np.float64)
    Ao = np.asarray(Ao, dtype=np.float64)
    diff = np.abs(Ag - Ao)
    far = ~touch
    assert np.all(Ao[far] < 0), "disjoint-support entries are negative"
    rel_far = float(np.max(diff[far] / np.abs(Ao[far]))) if far.any() else 0.0
    scale = np.sqrt(np.outer(diag_rows, diag_all))
    rel_touch = float(np.max(diff[touch] / scale[touch])) if touch.any() else 0.0
    return rel_far, rel_touch


def check_f64(Ag, Ao, om, s, tol=1e-12, rows=None, dof_mode="interior", diag=None):
    """Assert the float64 parity bar; Ao holds the oracle's rows `rows` (all when None).
    diag: the whole diagonal (defaults to Ao's, which needs all rows)."""
    touch = touching_mask(om, s, dof_mode)
    if rows is None:
        rows = np.arange(Ao.shape[0])
        diag = np.diag(Ao) if diag is None else diag
        Ag = np.asarray(Ag)
    else:
        Ag = np.asarray(Ag)[rows]
    assert diag is not None
    far, near = f64_errors(Ag, Ao, touch[rows], diag[rows], diag)
    assert far < tol and near < tol, (far, near)
    return far, near
