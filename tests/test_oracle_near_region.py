"""Pins for the oracle's near-region form of the diagonal blocks (the near-field assembly of the
cluster method, Section 6): the far pairs' diagonal-block terms and the boundary term are
replaced by C/(2s) times an integral over the boundary of N(K) (divergence theorem).  Checked
against closed forms of the exterior integral, against the exact stiffness matrices, and
against the pair-sum assembly of Section 5."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import OracleMesh, QuadOrders, assemble_matrix, exact
from oracle.assemble import cell_points, facet_sum, frac_constant, near_region_facets
from paper_1708_03912_gb300 import synth

HIGH = QuadOrders(k_far=10, k_near=14, k_touch=20, k_bnd=20, k_vertex=20)


def scaled_err(A, E):
    d = np.sqrt(np.outer(np.diag(E), np.diag(E)))
    return float(np.max(np.abs(A - E) / d))


def _exterior_square(x, a, s):
    """∫ over the plane minus [-a, a]^2 of |x - y|^{-2-2s} dy for x inside the square: in polar
    coordinates about x the radial integral is r0^{-2s} / (2s), r0(theta) the distance to the
    square's boundary along theta."""
    def r0(th):
        c, sn = math.cos(th), math.sin(th)
        ts = []
        if c > 0: ts.append((a - x[0]) / c)
        if c < 0: ts.append((-a - x[0]) / c)
        if sn > 0: ts.append((a - x[1]) / sn)
        if sn < 0: ts.append((-a - x[1]) / sn)
        return min(ts)
    corners = sorted(math.atan2(cy - x[1], cx - x[0]) % (2 * math.pi) for cx in (-a, a) for cy in (-a, a))
    cuts = [0.0] + corners + [2 * math.pi]
    tot = 0.0
    for lo, hi in zip(cuts, cuts[1:]):
        if hi > lo:
            tot += integrate.quad(lambda th: r0(th) ** (-2 * s), lo, hi, epsabs=0, epsrel=1e-13, limit=200)[0]
    return tot / (2 * s)


@pytest.mark.parametrize("s", [0.25, 0.5, 0.8])
def test_facet_sum_is_the_exterior_integral_2d(s):
    # a cell K inside the square [-1, 1]^2, the square's four edges with normals into it:
    # sum_ij of the block = C/(2s) * 2s * sum_a w_a ∫_{outside} k(x_a, y) dy (partition of unity)
    V = np.array([[-0.3, -0.2], [0.35, -0.1], [0.05, 0.4]])
    m = OracleMesh(V, [[0, 1, 2]])
    C = frac_constant(2, s)
    a = 1.0
    Y0 = np.array([[-a, -a], [a, -a], [a, a], [-a, a]])
    Y1 = np.roll(Y0, -1, axis=0)
    n = np.array([[0.0, 1.0], [-1.0, 0.0], [0.0, -1.0], [1.0, 0.0]])
    blk = facet_sum(m, s, C, 0, Y0, Y1, n, np.full(4, 2 * a), 40)
    xa, wa, _ = cell_points(m, 0, 40)
    want = C * sum(w * _exterior_square(x, a, s) for x, w in zip(xa[0], wa[0]))
    assert abs(blk.sum() - want) <= 1e-12 * abs(want)


def test_facet_sum_is_the_exterior_integral_1d():
    # N = [-1, 2]: ∫ outside |x - y|^{-1-2s} dy = ((x + 1)^{-2s} + (2 - x)^{-2s}) / (2s)
    s = 0.35
    m = OracleMesh(np.array([[0.0], [0.5]]), [[0, 1]])
    C = frac_constant(1, s)
    blk = facet_sum(m, s, C, 0, np.array([[-1.0], [2.0]]), np.array([[-1.0], [2.0]]),
                    np.array([[1.0], [-1.0]]), np.ones(2), 12)
    xa, wa, pha = cell_points(m, 0, 12)
    x = xa[0, :, 0]
    E = ((x + 1.0) ** (-2 * s) + (2.0 - x) ** (-2 * s)) / (2 * s)
    want = C * np.einsum("ai,aj,a->ij", pha, pha, wa[0] * E)
    assert np.max(np.abs(blk - want)) <= 1e-14 * np.max(np.abs(want))


def test_near_region_boundary_is_closed():
    # the facets of the boundary of N(K) form closed polygons: every vertex is an end of an even
    # number of them, normals are unit and point into a cell of N(K)
    V, T = synth.lshape(0.25, 0)
    m = OracleMesh(V, T)
    for k in (0, 7, len(T) // 2, len(T) - 1):
        Y0, Y1, n, flen, verts, bidx = near_region_facets(m, k)
        cnt = np.bincount(verts.ravel(), minlength=m.nv)
        assert np.all(cnt % 2 == 0) and len(verts) >= 3
        assert np.allclose(np.linalg.norm(n, axis=1), 1.0)
        assert np.allclose(np.linalg.norm(Y1 - Y0, axis=1), flen)
        # boundary facets of Omega keep their stored inward normal
        for q in np.nonzero(bidx >= 0)[0]:
            assert np.array_equal(n[q], m.normals[bidx[q]])


@pytest.mark.parametrize("s", [0.25, 0.4, 0.75])
def test_near_region_1d_matches_exact_matrix(s):
    pytest.importorskip("mpmath")
    for V, T in (synth.interval(16), synth.graded_interval(12, 2.0)):
        m = OracleMesh(V, T)
        E = exact.exact_matrix_1d(V[:, 0], s)
        B, _ = assemble_matrix(m, s, HIGH, self_term="near_region")
        assert scaled_err(B, E) < 1e-12
        B, _ = assemble_matrix(m, s, self_term="near_region")
        assert scaled_err(B, E) < 5e-6


@pytest.mark.parametrize("s", [0.25, 0.75])
def test_near_region_2d_matches_exact_matrix(s):
    V, T = synth.disc(3)
    m = OracleMesh(V, T)
    E = exact.exact_matrix_2d(m, s)
    errs = [scaled_err(assemble_matrix(m, s, o, self_term="near_region")[0], E) for o in (QuadOrders(), HIGH)]
    assert errs[0] < 5e-5 and errs[1] < 1e-10, errs


@pytest.mark.parametrize("s", [0.25, 0.5, 0.75])
def test_near_region_only_changes_the_diagonal_blocks(s):
    # entries of DOFs whose supports share no cell are the pair sums' (the diagonal blocks are the
    # only change), the rest agree within the pair sums' own quadrature error
    V, T = synth.disc(5, 2.0)
    m = OracleMesh(V, T)
    A, vod = assemble_matrix(m, s)
    B, _ = assemble_matrix(m, s, self_term="near_region")
    share = np.zeros((len(vod), len(vod)), dtype=bool)
    for K in range(m.nc):
        ds = [int(np.searchsorted(vod, v)) for v in m.C[K] if v in set(vod)]
        for i in ds:
            share[i, ds] = True
    D = np.sqrt(np.outer(np.diag(A), np.diag(A)))
    far = ~share
    assert np.max(np.abs(A - B)[far] / np.abs(A)[far]) < 1e-13
    assert np.max(np.abs(A - B)[share] / D[share]) < 5e-6
    assert np.array_equal(B, B.T) or np.max(np.abs(B - B.T) / D) < 1e-15


def test_near_region_rejects_regional():
    V, T = synth.interval(8)
    with pytest.raises(ValueError):
        assemble_matrix(OracleMesh(V, T), 0.5, regional=True, self_term="near_region")
