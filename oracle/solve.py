"""Direct and iterative solves of A u = b (oracle; test infrastructure only).

Section 5: a factorisation costs O(n^3); conjugate gradients with diagonal
scaling need O(n^{s/d}) iterations because κ(D^{-1}A) = O(n^{2s/d}).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def cholesky_solve(A, b):
    """Solve with a Cholesky factorisation (raises LinAlgError if A is not SPD)."""
    c = scipy.linalg.cho_factor(A, lower=True)
    return scipy.linalg.cho_solve(c, b)


def pcg_jacobi(A, b, tol=1e-8, maxit=10000):
    """Conjugate gradients preconditioned by D = diag(A); stop at ||r||/||b|| <= tol.

    Returns (x, iterations, relative residual history)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    dinv = 1.0 / np.diag(A)
    z = dinv * r
    p = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / nb]
    it = 0
    while hist[-1] > tol and it < maxit:
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
        hist.append(np.linalg.norm(r) / nb)
    return x, it, hist
