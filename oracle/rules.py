"""Quadrature rules for the oracle (test infrastructure only).

Section 5 and Appendix B of the paper ask for Gauss-type rules of variable order
on element pairs; the rule family is not fixed there.  The reading used here:

* Gauss-Legendre on [0, 1], k points (numpy's leggauss, mapped affinely);
* on a triangle, the collapsed (Duffy / conical) product rule of order k:
  lambda1 = t_a, lambda2 = t_b (1 - t_a), weight w_a w_b (1 - t_a), q = k^2
  points on the reference triangle {lambda >= 0, lambda1 + lambda2 <= 1}
  (weights sum to 1/2), points ordered a-major.
"""
from __future__ import annotations

import functools

import numpy as np


@functools.lru_cache(maxsize=None)
def gauss01(k: int):
    """k-point Gauss-Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(k)
    return (x + 1.0) / 2.0, w / 2.0


def gauss_on(a: float, b: float, k: int):
    """k-point Gauss-Legendre rule on [a, b]."""
    t, w = gauss01(k)
    return a + (b - a) * t, (b - a) * w


@functools.lru_cache(maxsize=None)
def triangle(k: int):
    """Collapsed Gauss rule on the reference triangle: (lambda [q,2], weights [q])."""
    t, w = gauss01(k)
    lam1 = np.repeat(t, k)
    lam2 = np.tile(t, k) * (1.0 - lam1)
    wt = np.repeat(w, k) * np.tile(w, k) * (1.0 - lam1)
    return np.stack([lam1, lam2], axis=1), wt


def p1_shape(lam):
    """P1 shape functions (phi_0, phi_1, phi_2) = (1 - l1 - l2, l1, l2) at reference points."""
    lam = np.atleast_2d(lam)
    return np.stack([1.0 - lam[:, 0] - lam[:, 1], lam[:, 0], lam[:, 1]], axis=1)
