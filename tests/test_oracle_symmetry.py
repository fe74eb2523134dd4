"""Pins of the symmetry-reduced problem (Section 7, "Exploiting Symmetry"): the rotated copies
form a conforming mesh of the whole polygon; the reduced system agrees with P^T A P / K and
its solution with the whole mesh's; with f = f_{2,8} (periodic under the rotation by pi/4) the
energy error against the closed form u_{2,8} (Section 7) is positive and falls under
refinement."""
import math

import numpy as np
import pytest
from scipy import special

from oracle import rules, solve
from oracle import symmetry as sym
from paper_1708_03912_gb300 import synth

K = 8


def test_copies_form_a_conforming_polygon():
    V, T = synth.sector(K, 6)
    W, C, vmap, copy = sym.replicate(V, T, K)
    P = W[C]
    area = 0.5 * np.abs((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
                        - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))
    # the polygon inscribed in the unit circle with the outer ring's points: K * (its sector part)
    n_outer = max(1, round(2 * math.pi * 6 / K))
    assert abs(area.sum() - K * n_outer * 0.5 * math.sin(2 * math.pi / (K * n_outer))) < 1e-12
    cnt = {}
    for c in C:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            e = (min(c[a], c[b]), max(c[a], c[b]))
            cnt[e] = cnt.get(e, 0) + 1
    # every edge inside the unit circle is shared, the ones on it are not
    for (a, b), k in cnt.items():
        on_circle = abs(np.hypot(*W[a]) - 1) < 1e-12 and abs(np.hypot(*W[b]) - 1) < 1e-12
        assert k == (1 if on_circle else 2)
    # merged: the centre once, each cut-ray vertex once per ray
    n_ray = sum(1 for v in V if abs(v[1]) < 1e-14 and v[0] > 0)
    assert len(W) == K * (len(V) - 1 - n_ray) + 1


@pytest.mark.parametrize("s", [0.25, 0.5, 0.75])
def test_reduced_system_matches_fold_and_whole_solution(s):
    V, T = synth.sector(K, 5)
    A1, b1, reps = sym.fold_system(V, T, K, s)
    A2, b2, reps2 = sym.reduced_system(V, T, K, s)
    assert np.array_equal(reps, reps2)
    d = np.sqrt(np.outer(np.diag(A1), np.diag(A1)))
    # equal up to the quadrature's own rotation defect (touching-pair rules depend on cell order)
    assert np.max(np.abs(A1 - A2) / d) < 1e-6
    assert np.allclose(b1, b2, rtol=0, atol=1e-15)
    assert np.linalg.eigvalsh(A2).min() > 0
    # the reduced solution is the whole mesh's solution on the representatives
    mesh, P, _ = sym.orbits(V, T, K, s)
    from oracle import assemble_matrix, load_vector
    A, _ = assemble_matrix(mesh, s)
    u = solve.cholesky_solve(A, load_vector(mesh, s))
    ur = solve.cholesky_solve(A2, b2)
    assert np.max(np.abs(P @ ur - u)) < 1e-5 * np.max(np.abs(u))
    # and the whole solution is periodic: constant on every orbit
    spread = max(np.ptp(u[P[:, r] > 0]) for r in range(P.shape[1]))
    assert spread < 1e-5 * np.max(np.abs(u))


def _f28(x, y, s):
    r2 = x * x + y * y
    th = np.arctan2(y, x)
    lam = 2 ** (2 * s) * special.gamma(3 + s) * special.gamma(11 + s) / (special.gamma(3) * special.gamma(11))
    return lam * r2 ** 4 * np.cos(8 * th) * special.eval_jacobi(2, s, 8, 2 * r2 - 1)


def _energy28(s):
    # <f, u> = lam pi / 2 int_0^1 t^8 P(2t-1)^2 (1-t)^s dt, Gauss-Jacobi in x = 2t - 1
    lam = 2 ** (2 * s) * special.gamma(3 + s) * special.gamma(11 + s) / (special.gamma(3) * special.gamma(11))
    x, w = special.roots_jacobi(10, s, 0.0)
    t = (1 + x) / 2
    return lam * math.pi / 2 * 2 ** (-s - 1) * np.sum(w * t ** 8 * special.eval_jacobi(2, s, 8, x) ** 2)


@pytest.mark.parametrize("s", [0.5])
def test_closed_form_f28_energy_error_falls(s):
    errs = []
    for M in (4, 8, 12):
        V, T = synth.sector(K, M)
        A, _, reps = sym.reduced_system(V, T, K, s)
        mesh, P, _ = sym.orbits(V, T, K, s)
        vod, dov = mesh.dofs(s)
        # load vector <f, phi_i> of the whole mesh by an order-10 collapsed Gauss rule (f is a
        # polynomial of degree 12 in x, y), then folded
        lam_, w_ = rules.triangle(10)
        b = np.zeros(len(vod))
        for c in mesh.C:
            Pc = mesh.V[c]
            area2 = abs((Pc[1, 0] - Pc[0, 0]) * (Pc[2, 1] - Pc[0, 1]) - (Pc[1, 1] - Pc[0, 1]) * (Pc[2, 0] - Pc[0, 0]))
            y = Pc[0] + lam_[:, 0:1] * (Pc[1] - Pc[0]) + lam_[:, 1:2] * (Pc[2] - Pc[0])
            fv = _f28(y[:, 0], y[:, 1], s)
            phi = rules.p1_shape(lam_)
            for a in range(3):
                if dov[c[a]] >= 0:
                    b[dov[c[a]]] += area2 * np.sum(w_ * fv * phi[:, a])
        br = P.T @ b / K
        ur = solve.cholesky_solve(A, br)
        errs.append(_energy28(s) - K * br @ ur)
    print("energy error^2", errs)
    assert all(e > 0 for e in errs)
    assert errs[0] > errs[1] > errs[2]
