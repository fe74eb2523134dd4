"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- a closed form, an independent exact route to the matrix, a
library routine on a special case, or an invariant the mathematics fixes."""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import gamma

from oracle import OracleMesh, QuadOrders, assemble_matrix, exact, load_vector, rules, solve
from oracle.assemble import frac_constant
from paper_1708_03912_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
HIGH = QuadOrders(k_far=10, k_near=14, k_touch=20, k_bnd=20, k_vertex=20)


def scaled_err(A, E):
    d = np.sqrt(np.outer(np.diag(E), np.diag(E)))
    return float(np.max(np.abs(A - E) / d))


# ---------------------------------------------------------------- rules ----
def test_gauss_exact_on_polynomials():
    for k in (1, 3, 6):
        t, w = rules.gauss01(k)
        for p in range(2 * k):
            assert abs(np.dot(w, t ** p) - 1.0 / (p + 1)) < 1e-14


def test_triangle_rule_exact_on_monomials():
    # ∫_T λ1^a λ2^b = a! b! / (a+b+2)!
    for k in (2, 4, 6):
        lam, w = rules.triangle(k)
        for a in range(k):
            for b in range(k - a):
                ref = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
                assert abs(np.dot(w, lam[:, 0] ** a * lam[:, 1] ** b) - ref) < 1e-14


def test_constant_special_values():
    # C(d,s) against its definition at s = 1/2: C(1,1/2) = 1/π, C(2,1/2) = 1/(2π)
    assert abs(frac_constant(1, 0.5) - 1 / math.pi) < 1e-15
    assert abs(frac_constant(2, 0.5) - 1 / (2 * math.pi)) < 1e-15


# ----------------------------------------------------------------- mesh ----
def test_mesh_boundary_and_dofs():
    V, T = synth.interval(128)
    m = OracleMesh(V, T)
    assert len(m.dofs(0.25)[0]) == 127
    assert len(m.dofs(0.25, "paper")[0]) == 129
    V, T = synth.disc(25)
    m = OracleMesh(V, T)
    # boundary vertices lie on the unit circle, inward normals point to the centre
    bv = np.nonzero(m.on_boundary)[0]
    assert np.allclose(np.hypot(*m.V[bv].T), 1.0)
    mids = (m.V[m.facets[:, 0]] + m.V[m.facets[:, 1]]) / 2
    assert np.all(np.sum(m.normals * mids, axis=1) < 0)
    assert abs(m.vol.sum() - math.pi) < 1e-2


# ------------------------------------------------------------- 1D exact ----
@pytest.mark.parametrize("s", [0.25, 0.4, 0.75])
def test_1d_matches_exact_matrix(s):
    mp = pytest.importorskip("mpmath")  # noqa: F841
    for V, T in (synth.interval(16), synth.graded_interval(12, 2.0)):
        m = OracleMesh(V, T)
        E = exact.exact_matrix_1d(V[:, 0], s)
        A, _ = assemble_matrix(m, s, HIGH)
        assert scaled_err(A, E) < 1e-12
        A, _ = assemble_matrix(m, s)
        assert scaled_err(A, E) < 5e-6


def test_1d_golden():
    gold = json.load(open(os.path.join(GOLD, "interval16_exact.json")))
    V, T = synth.interval(16)
    m = OracleMesh(V, T)
    for s, E in gold["matrices"].items():
        A, _ = assemble_matrix(m, float(s), HIGH)
        assert scaled_err(A, np.array(E)) < 1e-12


# ------------------------------------------------------------- 2D exact ----
@pytest.mark.parametrize("s", [0.25, 0.75])
def test_2d_matches_exact_matrix_disc(s):
    V, T = synth.disc(3)
    m = OracleMesh(V, T)
    E = exact.exact_matrix_2d(m, s)
    errs = []
    for orders in (QuadOrders(), QuadOrders(6, 8, 12, 12, 10), HIGH):
        A, _ = assemble_matrix(m, s, orders)
        errs.append(scaled_err(A, E))
    assert errs[0] < 5e-5 and errs[1] < errs[0] / 20 and errs[2] < 1e-10


def test_2d_golden_square():
    gold = json.load(open(os.path.join(GOLD, "square4_exact.json")))
    V, T = synth.square(4, 0.2)
    m = OracleMesh(V, T)
    for s, E in gold["matrices"].items():
        A, _ = assemble_matrix(m, float(s), HIGH)
        assert scaled_err(A, np.array(E)) < 1e-10


# ------------------------------------------------------- energy identity ----
def test_1d_energy_rate():
    # ||u-u_h||^2 = (f,u) - b·u_h > 0, O(n^-1) on uniform meshes (Section 7.1)
    for s in (0.25, 0.75):
        E = exact.energy_f1(1, s)
        gaps = []
        for N in (16, 32, 64):
            m = OracleMesh(*synth.interval(N))
            A, _ = assemble_matrix(m, s)
            b = load_vector(m, s)
            gaps.append(E - b @ solve.cholesky_solve(A, b))
        assert all(g > 0 for g in gaps)
        r = [gaps[i] / gaps[i + 1] for i in range(2)]
        assert all(1.7 < x < 2.4 for x in r), r


def test_1d_sign_energy():
    # f = sign(x): (f,u) = 2^{1-2s}/((2s+1)Γ(1+s)^2) (Section 7.1), approached from below
    s = 0.25
    Eex = exact.energy_sign_1d(s)
    m = OracleMesh(*synth.interval(64))
    A, vod = assemble_matrix(m, s)
    cen = m.V[m.C].mean(axis=1)[:, 0]
    b = np.zeros(len(vod))
    dov = -np.ones(m.nv, dtype=int)
    dov[vod] = np.arange(len(vod))
    for k, c in enumerate(m.C):
        for v in c:
            if dov[v] >= 0:
                b[dov[v]] += np.sign(cen[k]) * m.vol[k] / 2
    Eh = b @ solve.cholesky_solve(A, b)
    assert 0 < Eex - Eh < 0.03 * Eex


def test_2d_energy_inscribed_disc():
    # polygons inscribed in the disc: V_h ⊂ H~^s(disc), so the gap is a squared error
    for s in (0.25, 0.75):
        E = exact.energy_f1(2, s)
        gaps = []
        for M in (3, 5, 8):
            m = OracleMesh(*synth.disc(M))
            A, _ = assemble_matrix(m, s)
            b = load_vector(m, s)
            gaps.append(E - b @ solve.cholesky_solve(A, b))
        assert gaps[0] > gaps[1] > gaps[2] > 0, gaps


@pytest.mark.parametrize("s", [0.25, 0.5, 0.75])
def test_1d_solution_converges_to_closed_form(s):
    # f = 1 on (-1, 1): u = c (1 - x^2)^s (Section 2's closed form on the ball).  Per node, the error
    # of the Galerkin solution on uniform meshes of N = 64, 128, 256 cells: its maximum, at the nodes
    # next to the boundary where u behaves like dist^s, falls like h^s (the best any piecewise linear
    # function does there); away from the boundary (|x| <= 1/2) the error falls like h.  Both observed
    # rates must match to a few hundredths: a wrong constant, term or sign leaves an O(1) error that
    # does not fall at all.
    c = exact.ball_solution_scale(1, s)
    e_max, e_in = [], []
    for N in (64, 128, 256):
        m = OracleMesh(*synth.interval(N))
        A, vod = assemble_matrix(m, s)
        u = solve.cholesky_solve(A, load_vector(m, s))
        x = m.V[vod, 0]
        e = np.abs(u - c * (1 - x * x) ** s)
        e_max.append(e.max())
        e_in.append(e[np.abs(x) <= 0.5].max())
    r_max = np.log2(np.array(e_max[:-1]) / np.array(e_max[1:]))
    r_in = np.log2(np.array(e_in[:-1]) / np.array(e_in[1:]))
    assert np.all(np.abs(r_max - s) < 0.03), r_max
    assert np.all((r_in > 0.93) & (r_in < 1.05)), r_in
    assert e_max[-1] < 0.04 * c


# ------------------------------------------------------------- invariants ----
def test_symmetry_spd_scaling_rigid_motion():
    s = 0.6
    V, T = synth.square(3, 0.2)
    m = OracleMesh(V, T)
    A, _ = assemble_matrix(m, s)
    assert np.abs(A - A.T).max() < 1e-14 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0
    lam = 0.37
    A2, _ = assemble_matrix(OracleMesh(lam * V, T), s)
    assert np.abs(A2 - lam ** (2 - 2 * s) * A).max() < 1e-12 * np.abs(A).max()
    th = 0.83
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    A3, _ = assemble_matrix(OracleMesh(V @ R.T + np.array([3.0, -1.5]), T), s)
    assert np.abs(A3 - A).max() < 1e-11 * np.abs(A).max()


def test_regional_rows_sum_to_zero():
    # regional operator on the all-vertex basis: Σ_j phi_j = 1 kills (u(x)-u(y))
    m = OracleMesh(*synth.interval(10))
    A, _ = assemble_matrix(m, 0.3, dof_mode="paper", regional=True)
    assert np.abs(A.sum(axis=1)).max() < 1e-12 * np.abs(A).max()
    m = OracleMesh(*synth.square(3, 0.2))
    A, _ = assemble_matrix(m, 0.3, dof_mode="paper", regional=True)
    assert np.abs(A.sum(axis=1)).max() < 1e-12 * np.abs(A).max()


def test_paper_mode_1d_boundary_dofs():
    # s < 1/2: all vertices are DOFs; exact matrix through the boundary term and
    # pairs is still SPD and reduces to the interior matrix on interior rows? no:
    # rows differ, but the interior block of the paper-mode matrix equals the
    # interior-mode matrix exactly.
    m = OracleMesh(*synth.interval(12))
    Ap, vp = assemble_matrix(m, 0.3, dof_mode="paper")
    Ai, vi = assemble_matrix(m, 0.3)
    sel = np.isin(vp, vi)
    assert np.abs(Ap[np.ix_(sel, sel)] - Ai).max() < 1e-13 * np.abs(Ai).max()
    assert np.linalg.eigvalsh(Ap).min() > 0


def test_row_subset_equals_full():
    m = OracleMesh(*synth.disc(3))
    A, _ = assemble_matrix(m, 0.4)
    rows = np.array([0, 5, 11])
    Ar, _ = assemble_matrix(m, 0.4, rows=rows)
    assert np.abs(Ar - A[rows]).max() < 1e-14 * np.abs(A).max()


def test_jacobi_cg_iteration_growth():
    # κ(D^-1 A) = O(n^{2s/d}) ⇒ iterations grow like n^{s/d} (Section 5)
    s = 0.75
    its = []
    for N in (32, 128, 512):
        m = OracleMesh(*synth.interval(N))
        A, _ = assemble_matrix(m, s)
        b = load_vector(m, s)
        x, it, _ = solve.pcg_jacobi(A, b, tol=1e-8)
        assert np.linalg.norm(A @ x - b) <= 1.01e-8 * np.linalg.norm(b)
        its.append(it)
    r = its[2] / its[0]
    assert 2.0 < r < 16 ** 0.75 * 1.6, its


def test_load_vector_nodal_one_equals_f1():
    m = OracleMesh(*synth.disc(4))
    b1 = load_vector(m, 0.5)
    b2 = load_vector(m, 0.5, np.ones(m.nv))
    assert np.abs(b1 - b2).max() < 1e-15
    # Σ_i ∫phi_i over all vertices is |Ω|
    bp = load_vector(m, 0.3, dof_mode="paper")
    assert abs(bp.sum() - m.vol.sum()) < 1e-13


def test_load_vector_nodal_against_midpoint_rules():
    # b_i = ∫ f_h phi_i with f_h the P1 interpolant: the integrand is quadratic on each cell,
    # so the edge-midpoint rule on triangles (|K|/3 times the sum over the three edge
    # midpoints) and Simpson's rule on intervals integrate it exactly; neither uses the
    # mass-matrix formula of the oracle
    rng = np.random.default_rng(20170813)
    m = OracleMesh(*synth.disc(5))
    f = rng.standard_normal(m.nv)
    vod, dov = m.dofs(0.5)
    b = np.zeros(len(vod))
    for k in range(m.nc):
        cell = m.C[k]
        for a in range(3):
            for c in range(a + 1, 3):
                fm = 0.5 * (f[cell[a]] + f[cell[c]])  # f_h at the midpoint of edge (a, c)
                for v in (cell[a], cell[c]):          # phi_v = 1/2 there, the third hat is 0
                    if dov[v] >= 0:
                        b[dov[v]] += m.vol[k] / 3.0 * fm * 0.5
    assert np.abs(load_vector(m, 0.5, f) - b).max() < 1e-14 * np.abs(b).max()
    # 1D: Simpson on every cell
    V, T = synth.graded_interval(20, 1.5)
    m1 = OracleMesh(V, T)
    f1 = rng.standard_normal(m1.nv)
    vod1, dov1 = m1.dofs(0.5)
    b1 = np.zeros(len(vod1))
    for k in range(m1.nc):
        i, j = m1.C[k]
        h = abs(m1.V[j, 0] - m1.V[i, 0])
        fm = 0.5 * (f1[i] + f1[j])
        for v, fv in ((i, f1[i]), (j, f1[j])):   # phi_v: 1 at v, 1/2 at the midpoint, 0 at the other end
            if dov1[v] >= 0:
                b1[dov1[v]] += h / 6.0 * (fv * 1.0 + 4.0 * fm * 0.5)
    assert np.abs(load_vector(m1, 0.5, f1) - b1).max() < 1e-14 * np.abs(b1).max()
