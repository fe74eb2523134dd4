"""Pins of the oracle's near-field part N of A = N + F (F: off-diagonal blocks of the
separated pairs at vertex-graph distance >= 2, the far field of Section 6)."""
import numpy as np
import pytest

from oracle import OracleMesh, QuadOrders, assemble_matrix
from oracle.assemble import frac_constant, nearfield_pattern
from paper_1708_03912_gb300 import synth


@pytest.mark.parametrize("s", [0.3, 0.45])
def test_1d_regional_row_sums_are_far_field_integrals(s):
    # Regional operator, all vertices as DOFs (Section 3 for s < 1/2): every pair's block
    # has zero row sums (the form vanishes on constants), so the row sums of N are the
    # diagonal-block terms of the far pairs alone,
    #   (N 1)_i = C Σ_{K ∋ i} ∫_K phi_i(x) ∫_{far(K)} |x - y|^{-1-2s} dy dx,
    # far(K_k) = [z_0, z_{k-2}] ∪ [z_{k+3}, z_N].  The inner integral is done in closed
    # form here, the outer one by 40-point Gauss-Legendre (smooth integrand).
    V, T = synth.graded_interval(24, 1.6)
    om = OracleMesh(V, T)
    N, vod = assemble_matrix(om, s, QuadOrders(k_far=14, k_near=14), dof_mode="paper", regional=True,
                             far_offdiag=False)
    z = np.sort(V[:, 0])
    assert len(vod) == len(z)
    C = frac_constant(1, s)
    t, w = np.polynomial.legendre.leggauss(40)
    nc = len(z) - 1
    rs = np.zeros(len(z))
    for k in range(nc):
        a, b = z[k], z[k + 1]
        x = a + (b - a) * (t + 1) / 2
        wx = w * (b - a) / 2
        G = np.zeros_like(x)
        if k - 2 >= 1:
            G += ((x - z[k - 2]) ** (-2 * s) - (x - z[0]) ** (-2 * s)) / (2 * s)
        if k + 3 <= nc - 1:
            G += ((z[k + 3] - x) ** (-2 * s) - (z[nc] - x) ** (-2 * s)) / (2 * s)
        phi_a = (b - x) / (b - a)  # hat of z_k on K
        rs[k] += C * np.sum(wx * phi_a * G)
        rs[k + 1] += C * np.sum(wx * (1 - phi_a) * G)
    order = np.argsort(V[vod, 0])
    got = N.sum(axis=1)[order]
    scale = np.abs(np.diag(N)).max()
    assert np.max(np.abs(got - rs)) < 1e-10 * scale
    assert np.max(np.abs(rs)) > 1e-3 * scale  # the far field is not negligible here


def test_pattern_and_agreement_with_full_matrix():
    V, T = synth.disc(4)
    om = OracleMesh(V, T)
    s = 0.6
    A, vod = assemble_matrix(om, s)
    N, _ = assemble_matrix(om, s, far_offdiag=False)
    pat = nearfield_pattern(om, s)
    d = np.sqrt(np.outer(np.diag(A), np.diag(A)))
    assert np.max(np.abs(N - N.T) / d) < 1e-14  # symmetric up to the summation order
    assert not N[~pat].any()  # nothing outside the near-field pattern
    # DOF pairs whose supports have no cell pair at distance >= 2 get no far-field term
    nc = om.nc
    far = np.zeros((nc, nc), dtype=bool)
    for k in range(nc):
        shared, near = om.classify_cells(k)
        far[k] = (shared == 0) & ~near
    S = np.zeros((len(vod), nc), dtype=np.int64)
    for i, v in enumerate(vod):
        S[i, om.cells_of_vertex[v]] = 1
    nofar = (S @ far.astype(np.int64) @ S.T) == 0
    assert nofar.sum() > len(vod)
    assert np.max(np.abs(N - A)[nofar] / d[nofar]) < 1e-14
    # and where far pairs exist, N differs from A (the far field was left out)
    assert np.max(np.abs(N - A)[~nofar] / d[~nofar]) > 1e-6


def test_disjoint_support_entries_are_negative_and_inside_the_far_part():
    # Section 6: for DOFs whose supports share no vertex, a(phi_i, phi_j) = -C ∬ phi_i phi_j k < 0;
    # the entry-wise float64 parity check measures those entries relative to themselves.  Every
    # touching pair is in the near-field pattern (touching cells are near-field pairs).
    import sys
    import os

    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from parity import touching_mask

    for (V, T), s in ((synth.disc(5), 0.3), (synth.graded_interval(30, 2.0), 0.7), (synth.lshape(0.25, 0), 0.5)):
        om = OracleMesh(V, T)
        A, _ = assemble_matrix(om, s)
        M = touching_mask(om, s)
        assert np.all(A[~M] < 0)
        assert np.all(nearfield_pattern(om, s)[M])
        assert np.all(np.diag(M))
