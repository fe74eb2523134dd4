"""Closed forms that pin the oracle (test infrastructure only).

* ball solutions of Section 7 (f = 1 and the Jacobi-polynomial families) and
  the energies (f, u) used with the Galerkin identity ||u - u_h||^2 = (f,u) - (f,u_h)
  (Section 7.1);
* the exact stiffness matrix of interior hat functions, derived from the
  Fourier form a(u,v) = <|xi|^{2s} u^, v^> of Section 2: writing
  |xi|^{2s} = |xi|^{2s-4} |xi|^4 gives a(u,v) = c_{d,s} ∬ |x-y|^{4-2s-d} dΔu(x) dΔv(y),
  where Δu of a P1 function is a sum of point masses (1D) or line measures on
  edges (2D) and c_{d,s} is the Riesz-potential constant of order 4 - 2s.  Both
  reduce to smooth or explicitly integrable low-dimensional integrals, so they
  are an independent route to every matrix entry (separated, touching and
  boundary parts together).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import gamma

from . import rules
from .assemble import frac_constant
from .mesh import OracleMesh


def ball_solution_scale(d: int, s: float) -> float:
    """u = scale * (1 - |x|^2)_+^s solves (-Δ)^s u = 1 on the unit ball (Section 7, n = 0)."""
    return 2.0 ** (-2 * s) * gamma(d / 2.0) / (gamma(d / 2.0 + s) * gamma(1.0 + s))


def energy_f1(d: int, s: float) -> float:
    """(f, u) for f = 1 on the unit ball: scale * ∫ (1 - |x|^2)^s."""
    if d == 1:
        integral = math.sqrt(math.pi) * gamma(1.0 + s) / gamma(1.5 + s)
    else:
        integral = math.pi / (1.0 + s)
    return ball_solution_scale(d, s) * integral


def energy_sign_1d(s: float) -> float:
    """(f, u) for f = sign(x) on (-1, 1) (Section 7.1)."""
    return 2.0 ** (1 - 2 * s) / ((2 * s + 1) * gamma(1 + s) ** 2)


def riesz_constant_1d(s: float) -> float:
    """c with a(u,v) = c ∬ |x-y|^{3-2s} u''(x) v''(y) in 1D (s != 1/2)."""
    return frac_constant(1, s) / (2 * s * (1 - 2 * s) * (2 - 2 * s) * (3 - 2 * s))


def riesz_constant_2d(s: float) -> float:
    """c with a(u,v) = c ∬ |x-y|^{2-2s} dΔu dΔv in 2D."""
    return -frac_constant(2, s) / (4 * s * s * (2 - 2 * s) ** 2)


def exact_matrix_1d(z, s: float, dps: int = 40):
    """Exact matrix of the interior hats on the 1D mesh with sorted nodes z (mpmath).

    phi_i'' = δ_{z_{i-1}}/h_{i-1} - (1/h_{i-1} + 1/h_i) δ_{z_i} + δ_{z_{i+1}}/h_i;
    the fourth-order differences cancel heavily, hence the extended precision.
    """
    import mpmath as mp

    mp.mp.dps = dps
    zz = [mp.mpf(float(t)) for t in z]
    ss = mp.mpf(s)
    C = (mp.mpf(2) ** (2 * ss) * ss * mp.gamma(ss + mp.mpf(1) / 2)
         / (mp.sqrt(mp.pi) * mp.gamma(1 - ss)))
    c = C / (2 * ss * (1 - 2 * ss) * (2 - 2 * ss) * (3 - 2 * ss))
    n = len(zz) - 2
    W = []
    for i in range(1, n + 1):
        hl, hr = zz[i] - zz[i - 1], zz[i + 1] - zz[i]
        W.append([(i - 1, 1 / hl), (i, -(1 / hl + 1 / hr)), (i + 1, 1 / hr)])
    A = np.zeros((n, n))
    p = 3 - 2 * ss
    for i in range(n):
        for j in range(i, n):
            acc = mp.mpf(0)
            for a, wa in W[i]:
                for b, wb in W[j]:
                    if a != b:
                        acc += wa * wb * abs(zz[a] - zz[b]) ** p
            A[i, j] = A[j, i] = float(c * acc)
    return A


# ---------------------------------------------------------------- 2D -------
def _edge_jumps(mesh: OracleMesh, v: int):
    """Line-measure weights of Δphi_v: {edge (a,b) sorted: J}, with
    Δu = -Σ_K Σ_{e⊂∂K} (∇u|_K · n^out_{K,e}) δ_e."""
    J = {}
    V = mesh.V
    for k in mesh.cells_of_vertex[v]:
        cell = list(mesh.C[k])
        P = V[cell]
        M = np.array([P[1] - P[0], P[2] - P[0]])  # rows
        ghat = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])[cell.index(v)]
        g = np.linalg.solve(M, ghat)  # physical gradient: M g = ghat
        for a, b, c in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
            t = P[b] - P[a]
            nrm = np.array([t[1], -t[0]]) / np.hypot(*t)
            if np.dot(nrm, P[c] - P[a]) > 0:
                nrm = -nrm
            key = (min(cell[a], cell[b]), max(cell[a], cell[b]))
            J[key] = J.get(key, 0.0) - float(np.dot(g, nrm))
    return J


def _edge_pair_integral(V, e, f, s, kq=40):
    """∫_e ∫_f |x-y|^{2-2s} (arc length on both)."""
    p = 2.0 - 2.0 * s
    a0, a1 = V[e[0]], V[e[1]]
    b0, b1 = V[f[0]], V[f[1]]
    La, Lb = np.linalg.norm(a1 - a0), np.linalg.norm(b1 - b0)
    shared = set(e) & set(f)
    if len(shared) == 2:
        return 2.0 * La ** (4 - 2 * s) / ((3 - 2 * s) * (4 - 2 * s))
    t, w = rules.gauss01(kq)
    if len(shared) == 1:
        P = shared.pop()
        ua = V[e[1] if e[0] == P else e[0]] - V[P]
        ub = V[f[1] if f[0] == P else f[0]] - V[P]
        r1 = np.linalg.norm(ua[None, :] - t[:, None] * ub[None, :], axis=1) ** p
        r2 = np.linalg.norm(t[:, None] * ua[None, :] - ub[None, :], axis=1) ** p
        return La * Lb / (4 - 2 * s) * float(np.dot(w, r1 + r2))
    x = a0[None, :] + t[:, None] * (a1 - a0)[None, :]
    y = b0[None, :] + t[:, None] * (b1 - b0)[None, :]
    r = np.linalg.norm(x[:, None, :] - y[None, :, :], axis=2) ** p
    return La * Lb * float(w @ r @ w)


def exact_matrix_2d(mesh: OracleMesh, s: float, pairs=None, kq: int = 40):
    """Exact A_ij = c Σ_{e,e'} J^i_e J^j_e' ∫_e∫_e' |x-y|^{2-2s} for interior-vertex DOFs.

    pairs: iterable of (i, j) DOF index pairs (default: the whole upper triangle).
    Returns a dict {(i, j): value} (or the full matrix when pairs is None).
    """
    vod, dov = mesh.dofs(s, "interior")
    n = len(vod)
    c = riesz_constant_2d(s)
    jumps = [_edge_jumps(mesh, int(v)) for v in vod]
    cache = {}

    def I(e, f):
        key = (e, f) if e <= f else (f, e)
        if key not in cache:
            cache[key] = _edge_pair_integral(mesh.V, key[0], key[1], s, kq)
        return cache[key]

    def entry(i, j):
        acc = 0.0
        for e, Je in jumps[i].items():
            for f, Jf in jumps[j].items():
                acc += Je * Jf * I(e, f)
        return c * acc

    if pairs is None:
        A = np.zeros((n, n))
        for i in range(n):
            for j in range(i, n):
                A[i, j] = A[j, i] = entry(i, j)
        return A
    return {(i, j): entry(i, j) for i, j in pairs}
