"""Pins of the oracle's strong form (Lemma 4.1, Appendix A) and indicators (Section 4):
1D against the closed form of (-Delta)^s of a piecewise linear function (sum of jumps of
u' times |x - z|^{1-2s}, a logarithm at s = 1/2); 2D against brute-force evaluations of
the defining integral away from and inside the support; the indicators against the
energy error under refinement."""
import math

import numpy as np
import pytest

from oracle import OracleMesh, assemble_matrix, load_vector, solve
from oracle.adaptive import br_indicators, cell_rule_points, mark_max, marked_cells, strong_form
from oracle.assemble import frac_constant
from oracle.exact import energy_f1
from paper_1708_03912_gb300 import synth


@pytest.mark.parametrize("s", [0.25, 0.4, 0.5, 0.75])
def test_strong_form_1d_closed_form(s):
    # u piecewise linear, u'' = sum_j J_j delta_{z_j}: (-Delta)^s u = C/(2s(1-2s)) sum_j J_j |x-z_j|^{1-2s},
    # and C sum_j J_j log|x - z_j| at s = 1/2 (sum_j J_j = 0)
    V, T = synth.graded_interval(12, 2.0)
    om = OracleMesh(V, T)
    vod, _ = om.dofs(s)
    u = np.random.default_rng(1).standard_normal(len(vod))
    S = strong_form(om, s, u, k_cell=3)
    x = cell_rule_points(om, 3)[0][..., 0]
    un = np.zeros(om.nv)
    un[vod] = u
    order = np.argsort(om.V[:, 0])
    z, uz = om.V[order, 0], un[order]
    sl = np.diff(uz) / np.diff(z)
    J = np.concatenate([[sl[0]], np.diff(sl), [-sl[-1]]])
    C = frac_constant(1, s)
    r = np.abs(x[..., None] - z)
    ref = (C * np.sum(J * np.log(r), axis=-1) if s == 0.5 else
           C / (2 * s * (1 - 2 * s)) * np.sum(J * r ** (1 - 2 * s), axis=-1))
    assert np.max(np.abs(S - ref)) < 1e-13 * np.max(np.abs(ref))


def _hat_2d():
    V, T = synth.disc(3)
    om = OracleMesh(V, T)
    vod, _ = om.dofs(0.5)
    i = int(np.argmin(np.linalg.norm(om.V[vod], axis=1)))  # the DOF nearest the centre
    u = np.zeros(len(vod))
    u[i] = 1.0
    return om, u, vod[i]


def _polar_integral(om, un, x, rho, s, ntheta=24):
    """int_{|y-x| > rho} u(y) |x-y|^{-2-2s} dy for the P1 function u (nodal values un): rays from x,
    u linear between the ray's crossings of mesh edges, radial integrals in closed form, Gauss in the
    angle between the angles of the vertices."""
    edges = set()
    for c in om.C:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            edges.add((min(c[a], c[b]), max(c[a], c[b])))
    edges = np.array(sorted(edges))
    P, Q = om.V[edges[:, 0]], om.V[edges[:, 1]]
    ang = np.sort(np.mod(np.arctan2(om.V[:, 1] - x[1], om.V[:, 0] - x[0]), 2 * np.pi))
    brk = np.concatenate([[0.0], ang, [2 * np.pi]])
    tg, wg = np.polynomial.legendre.leggauss(ntheta)
    total = 0.0
    for a0, a1 in zip(brk[:-1], brk[1:]):
        if a1 - a0 < 1e-14:
            continue
        for tt, ww in zip(tg, wg):
            th = 0.5 * (a0 + a1) + 0.5 * (a1 - a0) * tt
            e = np.array([math.cos(th), math.sin(th)])
            # ray x + t e against the segments P + lam (Q - P), Cramer's rule
            m01, m11 = P[:, 0] - Q[:, 0], P[:, 1] - Q[:, 1]
            det = e[0] * m11 - e[1] * m01
            ok = np.abs(det) > 1e-15
            rx, ry = P[:, 0] - x[0], P[:, 1] - x[1]
            with np.errstate(divide="ignore", invalid="ignore"):
                t = (rx * m11 - ry * m01) / det
                lam = (e[0] * ry - e[1] * rx) / det
            sel = ok & (t > 0) & (lam >= -1e-12) & (lam <= 1 + 1e-12)
            ts = np.concatenate([[0.0], np.sort(t[sel])])
            rad = 0.0
            for t0, t1 in zip(ts[:-1], ts[1:]):
                lo, hi = max(t0, rho), t1
                if hi <= lo:
                    continue
                # u is linear on [t0, t1]: its values at two interior points of the segment
                ta, tb = t0 + 0.25 * (t1 - t0), t0 + 0.75 * (t1 - t0)
                ua, ub = _eval(om, un, x + ta * e), _eval(om, un, x + tb * e)
                beta = (ub - ua) / (tb - ta)
                alpha = ua - beta * ta
                # int alpha r^{-1-2s} + beta r^{-2s} dr
                rad += alpha * (lo ** (-2 * s) - hi ** (-2 * s)) / (2 * s) + beta * (hi ** (1 - 2 * s) - lo ** (1 - 2 * s)) / (1 - 2 * s)
            total += 0.5 * (a1 - a0) * ww * rad
    return total


def _eval(om, un, y):
    P = om.V[om.C]
    d1, d2, r = P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], y - P[:, 0]
    det = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    l1 = (r[:, 0] * d2[:, 1] - r[:, 1] * d2[:, 0]) / det
    l2 = (d1[:, 0] * r[:, 1] - d1[:, 1] * r[:, 0]) / det
    inside = (l1 >= -1e-12) & (l2 >= -1e-12) & (l1 + l2 <= 1 + 1e-12)
    if not inside.any():
        return 0.0
    k = int(np.nonzero(inside)[0][0])
    c = om.C[k]
    return un[c[0]] * (1 - l1[k] - l2[k]) + un[c[1]] * l1[k] + un[c[2]] * l2[k]


@pytest.mark.parametrize("s", [0.25, 0.4, 0.75])
def test_strong_form_2d_brute_force(s):
    # the rule on the edges of the point's own cell has to resolve |x - y|^{-2-2s} next to x:
    # order 64 reaches 1e-13 here
    om, u, v = _hat_2d()
    C = frac_constant(2, s)
    S = strong_form(om, s, u, k_cell=2, k_edge=24, k_near=64)
    X = cell_rule_points(om, 2)[0]
    un = np.zeros(om.nv)
    un[v] = 1.0
    supp = set(om.cells_of_vertex[v])
    checked = inside = 0
    for k in range(om.nc):
        x = X[k, 0]
        if k not in supp:
            # away from the support: -C int phi(y) |x-y|^{-2-2s}, smooth (collapsed Gauss of order 24)
            from oracle import rules
            lam, w = rules.triangle(24)
            ref = 0.0
            for K in supp:
                P = om.V[om.C[K]]
                y = P[0] + lam[:, 0:1] * (P[1] - P[0]) + lam[:, 1:2] * (P[2] - P[0])
                phi = rules.p1_shape(lam)[:, int(np.nonzero(om.C[K] == v)[0][0])]
                ref += np.sum(w * 2 * om.vol[K] * phi * np.sum((x - y) ** 2, axis=1) ** (-1 - s))
            assert abs(S[k, 0] - (-C * ref)) < 1e-9 * abs(C * ref)
            checked += 1
        elif inside < 8:
            inside += 1
            # inside: C [u(x) 2 pi rho^{-2s} / (2s) - int_{|y-x|>rho} u |x-y|^{-2-2s}], the disc of radius
            # rho inside K contributing nothing (u linear there)
            P = om.V[om.C[k]]
            dist = min(abs((P[b, 0] - P[a, 0]) * (x[1] - P[a, 1]) - (P[b, 1] - P[a, 1]) * (x[0] - P[a, 0]))
                       / np.linalg.norm(P[b] - P[a]) for a, b in ((0, 1), (1, 2), (2, 0)))
            rho = 0.5 * dist
            ux = _eval(om, un, x)
            ref = C * (ux * 2 * np.pi * rho ** (-2 * s) / (2 * s) - _polar_integral(om, un, x, rho, s))
            assert abs(S[k, 0] - ref) < 1e-11 * abs(ref), (k, S[k, 0], ref)
    assert checked > 0 and inside > 0


def test_indicators_track_the_energy_error():
    # 1D, f = 1, s = 0.25 on uniform meshes: the estimator sum_i eta_i^2 and the squared energy
    # error (the Galerkin gap E - b.u) fall at the same rate, their ratio stays within a factor 2
    s = 0.25
    ratios = []
    for N in (8, 16, 32):
        V, T = synth.interval(N)
        om = OracleMesh(V, T)
        A, _ = assemble_matrix(om, s)
        b = load_vector(om, s)
        u = solve.cholesky_solve(A, b)
        err2 = energy_f1(1, s) - b @ u
        eta = br_indicators(om, s, u, k_cell=6)
        ratios.append(np.sum(eta ** 2) / err2)
    print("estimator / error^2:", ratios)
    assert max(ratios) < 2 * min(ratios)


def test_marking():
    eta = np.array([0.1, 0.79, 0.8, 1.0, 0.5])
    assert list(mark_max(eta, 0.8)) == [False, False, True, True, False]
    V, T = synth.disc(3)
    om = OracleMesh(V, T)
    marks = np.zeros(len(om.dofs(0.5)[0]), dtype=bool)
    marks[0] = True
    cells = marked_cells(om, 0.5, marks)
    assert set(cells) == set(om.cells_of_vertex[om.dofs(0.5)[0][0]])


def _edges_count(T):
    cnt = {}
    for t in T:
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            k = (min(a, b), max(a, b))
            cnt[k] = cnt.get(k, 0) + 1
    return cnt


def _canonical(V, T):
    """Mesh as a set of triangles (newest vertex, {refinement edge}) by coordinates."""
    key = lambda i: tuple(np.round(V[i], 14))
    return {(key(t[0]), frozenset([key(t[1]), key(t[2])])) for t in T}


def test_refine_conforming_and_minimal():
    from oracle.adaptive import refine
    V, T = synth.lshape(levels=1)
    rng = np.random.default_rng(5)
    marks = rng.random(len(T)) < 0.1
    V2, T2 = refine(V, T, marks)
    P0, P2 = V[T], V2[T2]
    area = lambda P: 0.5 * ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))
    assert abs(np.sum(np.abs(area(P2))) - np.sum(np.abs(area(P0)))) < 1e-13
    # conforming: every edge is shared by two cells or lies on the boundary, and no vertex lies
    # inside an edge
    cnt = _edges_count(T2)
    bnd0 = {k for k, c in _edges_count(T).items() if c == 1}
    for (a, b), c in cnt.items():
        assert c in (1, 2)
        if c == 1:  # a boundary edge is (a half of) an old boundary edge
            assert any(np.allclose(np.cross(np.append(V2[b] - V2[a], 0), np.append(V[q] - V[p], 0))[2], 0) and
                       min(np.linalg.norm(V2[a] - V[p]), np.linalg.norm(V2[a] - V[q])) < 1e-12 or
                       min(np.linalg.norm(V2[b] - V[p]), np.linalg.norm(V2[b] - V[q])) < 1e-12
                       for p, q in bnd0)
    for (a, b) in cnt:
        d = V2[b] - V2[a]
        rel = V2 - V2[a]
        t = rel @ d / (d @ d)
        perp = np.abs(rel[:, 0] * d[1] - rel[:, 1] * d[0])
        inside = (t > 1e-12) & (t < 1 - 1e-12) & (perp < 1e-12 * (d @ d))
        assert not inside.any()
    # every marked cell is bisected at its refinement edge; cells untouched by the closure stay
    old = _canonical(V, T)
    new = _canonical(V2, T2)
    marked = _canonical(V, T[marks])
    assert not (marked & new)
    kept = old & new
    assert len(T2) == len(kept) + sum(1 for t in T2 if (tuple(np.round(V2[t[0]], 14)),
                                                        frozenset([tuple(np.round(V2[t[1]], 14)), tuple(np.round(V2[t[2]], 14))])) not in old)
    # the unique conforming closure: the independent recursive bisection of the mesh generator
    # (which refines cell by cell) reaches the same triangles
    V3, T3 = synth._nvb_refine(V, T, list(np.nonzero(marks)[0]))
    assert _canonical(V3, T3) == new
    # order independence: reversing the cell order gives the same mesh
    V4, T4 = refine(V, T[::-1], marks[::-1])
    assert _canonical(V4, T4) == new


def test_refine_shape_regular_and_1d():
    from oracle.adaptive import refine
    V, T = synth.square(4)
    # newest vertex opposite the longest edge (the right angle): bisection then keeps every
    # triangle similar to the first ones (right isosceles)
    P = V[T]
    longest = np.argmax(np.stack([np.linalg.norm(P[:, 2] - P[:, 1], axis=1), np.linalg.norm(P[:, 0] - P[:, 2], axis=1),
                                  np.linalg.norm(P[:, 1] - P[:, 0], axis=1)], 1), 1)
    T = np.stack([np.roll(t, -int(l)) for t, l in zip(T, longest)])

    def min_angle(V, T):
        P = V[T]
        out = []
        for a, b, c in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
            u, v = P[:, b] - P[:, a], P[:, c] - P[:, a]
            out.append(np.arccos(np.sum(u * v, 1) / np.linalg.norm(u, axis=1) / np.linalg.norm(v, axis=1)))
        return np.min(out)
    a0 = min_angle(V, T)
    for it in range(8):
        P = V[T].mean(axis=1)
        marks = np.hypot(P[:, 0], P[:, 1]) < 0.6 ** it
        V, T = refine(V, T, marks)
    assert abs(a0 - np.pi / 4) < 1e-12
    assert min_angle(V, T) >= a0 - 1e-12
    assert len(T) > 100
    # 1D: halves
    V1, T1 = synth.interval(4)
    V2, T2 = refine(V1, T1, np.array([True, False, False, True]))
    L = np.sort(V2[T2[:, 1], 0] - V2[T2[:, 0], 0])
    assert np.allclose(L, [0.25, 0.25, 0.25, 0.25, 0.5, 0.5])
