"""Fractional heat equation (oracle; test infrastructure only).

Section 2 poses the fractional heat equation d_t u + (-Delta)^s u = f on [0, T] x Omega,
u = u_0 at t = 0; Section 5 discretises it implicitly in time, which gives in every step a
system (M + dt A^s) u = b with the P1 mass matrix M.  Read here as the implicit Euler step
(M + dt A^s) u^{k+1} = M u^k + dt F, F the load vector of f (Section 5 leaves the scheme
open; implicit Euler is the scheme that produces exactly that matrix).

* mass_matrix: M_ij = int phi_i phi_j, assembled cell by cell from the P1 element mass
  matrix |K| (1 + delta_ab) / ((d + 1)(d + 2)) (exact integral of two barycentric
  coordinates), rows and columns restricted to the DOF set of mesh.dofs().
* implicit_euler: the steps above, each system solved by the oracle's Cholesky solve.
"""
from __future__ import annotations

import numpy as np

from .mesh import OracleMesh
from .solve import cholesky_solve


def mass_matrix(mesh: OracleMesh, s: float, dof_mode: str = "interior"):
    """Dense P1 mass matrix on the DOFs of mesh (float64)."""
    vod, dov = mesh.dofs(s, dof_mode)
    n = len(vod)
    d = mesh.dim
    M = np.zeros((n, n))
    local = (np.ones((d + 1, d + 1)) + np.eye(d + 1)) / ((d + 1) * (d + 2))
    for k in range(mesh.nc):
        cell = mesh.C[k]
        for a, va in enumerate(cell):
            i = dov[va]
            if i < 0:
                continue
            for b, vb in enumerate(cell):
                j = dov[vb]
                if j >= 0:
                    M[i, j] += mesh.vol[k] * local[a, b]
    return M


def heat_matrix(A, M, dt):
    """The implicit-step matrix M + dt A."""
    return M + dt * A


def implicit_euler(A, M, F, u0, dt, steps):
    """u^{k+1} = (M + dt A)^{-1} (M u^k + dt F), k = 0 .. steps - 1; returns all iterates."""
    H = heat_matrix(A, M, dt)
    us = [np.asarray(u0, dtype=np.float64)]
    for _ in range(steps):
        us.append(cholesky_solve(H, M @ us[-1] + dt * F))
    return us
