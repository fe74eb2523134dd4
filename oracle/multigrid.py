"""Galerkin multigrid on nested P1 spaces (oracle; test infrastructure only).

Section 5 of the paper proposes multigrid for the dense systems without giving an
algorithm; the reading implemented here (and by the GPU path) is the textbook
Galerkin V-cycle:

* Nested meshes give nested P1 spaces V_c ⊂ V_f.  The prolongation P (fine DOFs x
  coarse DOFs) has P_ij = φ_j^c(x_i): the coarse hat function j evaluated at fine
  vertex i (exact for nested spaces, since a coarse function is linear on each
  coarse cell and the fine vertices lie in coarse cells).
* Coarse operators A_c = Pᵀ A_f P.
* Smoother: damped Jacobi x <- x + ω D⁻¹ (r - A x), ω = 4 / (3 λ), λ the estimate
  ||D⁻¹A x_K|| / ||x_K|| after K = 10 steps of the power iteration
  x_{k+1} = D⁻¹A x_k / ||D⁻¹A x_k|| from x_0 = (1, ..., 1).
* V-cycle from a zero guess: ν pre-smoothing steps, residual, restriction Pᵀ,
  recursion (exact solve on the coarsest level), prolongation P, ν post-smoothing steps.

Parity status: pinned in ``tests/test_oracle_multigrid.py`` — the Galerkin product
against the matrix assembled directly on the coarse mesh, linear-function
reproduction of P, the projector property of the coarse correction, symmetry and
A-norm contraction of the V-cycle.
"""
from __future__ import annotations

import numpy as np


def prolongation(Vf, dofs_f, Vc, Tc, dofs_c, tol=1e-12):
    """Dense P (len(dofs_f) x len(dofs_c)) by brute-force point location.

    Vf, Vc: vertex coordinates (2D); Tc: coarse cells; dofs_*: vertex index of each DOF."""
    Vf = np.asarray(Vf, dtype=np.float64)
    Vc = np.asarray(Vc, dtype=np.float64)
    col = {int(v): j for j, v in enumerate(dofs_c)}
    P = np.zeros((len(dofs_f), len(dofs_c)))
    for i, v in enumerate(dofs_f):
        x = Vf[v]
        for t in Tc:
            a, b, c = Vc[t[0]], Vc[t[1]], Vc[t[2]]
            m = np.array([[b[0] - a[0], c[0] - a[0]], [b[1] - a[1], c[1] - a[1]]])
            l1, l2 = np.linalg.solve(m, x - a)
            lam = (1.0 - l1 - l2, l1, l2)
            if min(lam) >= -tol:
                for k in range(3):
                    j = col.get(int(t[k]))
                    if j is not None:
                        P[i, j] = lam[k]
                break
        else:
            raise ValueError(f"fine vertex {v} lies in no coarse cell")
    return P


def galerkin(A, P):
    return P.T @ A @ P


def lambda_estimate(A, steps=10):
    """Power-iteration estimate of the largest eigenvalue of D⁻¹A (see module text)."""
    dinv = 1.0 / np.diag(A)
    x = np.ones(A.shape[0])
    for _ in range(steps):
        y = dinv * (A @ x)
        x = y / np.linalg.norm(y)
    return float(np.linalg.norm(dinv * (A @ x)) / np.linalg.norm(x))


def jacobi_weight(A, steps=10):
    return 4.0 / (3.0 * lambda_estimate(A, steps))


def hierarchy(A, Ps):
    """Level operators [A_0 = A, A_1 = P_1ᵀ A_0 P_1, ...] for prolongations Ps (fine to coarse order)."""
    As = [np.asarray(A, dtype=np.float64)]
    for P in Ps:
        As.append(galerkin(As[-1], P))
    return As


def vcycle(As, Ps, r, nu=2, omegas=None, level=0):
    """One V-cycle for A_level x = r from x = 0; exact solve on the last level."""
    A = As[level]
    if level == len(As) - 1:
        return np.linalg.solve(A, r)
    om = omegas[level] if omegas is not None else jacobi_weight(A)
    dinv = 1.0 / np.diag(A)
    x = np.zeros_like(r)
    for _ in range(nu):
        x = x + om * dinv * (r - A @ x)
    rc = Ps[level].T @ (r - A @ x)
    x = x + Ps[level] @ vcycle(As, Ps, rc, nu, omegas, level + 1)
    for _ in range(nu):
        x = x + om * dinv * (r - A @ x)
    return x


def vcycle_matrix(As, Ps, nu=2, omegas=None):
    """The V-cycle as a matrix (columns = V-cycle of unit vectors)."""
    n = As[0].shape[0]
    return np.stack([vcycle(As, Ps, e, nu, omegas) for e in np.eye(n)], axis=1)
