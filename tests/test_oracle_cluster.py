"""Pins of the oracle's cluster method (Section 6): the block partition, the Chebyshev
interpolation pieces against polynomial reproduction and exact integrals, and the
matrix-vector product against the dense matrix with an error that falls geometrically
with the interpolation order."""
import numpy as np
import pytest

from oracle import OracleMesh, assemble_matrix
from oracle.cluster import (ClusterTree, block_partition, cheb_points, kernel_matrix, lagrange, leaf_coefficients,
                            shift_matrix, hmatvec)
from oracle.heat import mass_matrix
from paper_1708_03912_gb300 import synth


@pytest.fixture(scope="module")
def disc():
    V, T = synth.disc(7)
    om = OracleMesh(V, T)
    A, _ = assemble_matrix(om, 0.5)
    return om, A


def test_partition_covers_every_pair_once(disc):
    om, _ = disc
    for leaf, eta in ((1, 1.0), (8, 1.0), (16, 2.0)):
        tree = ClusterTree(om, 0.5, leaf)
        far, near = block_partition(tree, eta)
        cover = np.zeros((tree.n, tree.n), dtype=np.int64)
        for a, b in far + near:
            cover[np.ix_(tree.dofs[a], tree.dofs[b])] += 1
        assert np.all(cover == 1)
        for a, b in far:
            assert eta * tree.dist(a, b) >= max(tree.diam(a), tree.diam(b))
        for a, b in near:
            assert not tree.sons[a] and not tree.sons[b]
            assert eta * tree.dist(a, b) < max(tree.diam(a), tree.diam(b))
        assert any(len(tree.dofs[c]) <= leaf for c in range(len(tree.dofs)))
        for c in range(len(tree.dofs)):
            if tree.sons[c]:
                assert sorted(np.concatenate([tree.dofs[x] for x in tree.sons[c]])) == sorted(tree.dofs[c])
            else:
                assert len(tree.dofs[c]) <= leaf


def test_boxes_contain_supports(disc):
    om, _ = disc
    tree = ClusterTree(om, 0.5, 4)
    for c in range(len(tree.dofs)):
        for i in tree.dofs[c]:
            P = om.V[om.C[om.cells_of_vertex[tree.vod[i]]].ravel()]
            assert np.all(np.abs(P - tree.center[c]) <= tree.side[c] / 2 + 1e-15)


def test_shift_reproduces_father_polynomials(disc):
    # L^father_alpha is a polynomial of degree m-1 per variable, so interpolation at the son's
    # Chebyshev points reproduces it: L^f(x) = sum_beta L^f(xi^son_beta) L^son_beta(x)
    om, _ = disc
    tree = ClusterTree(om, 0.5, 4)
    rng = np.random.default_rng(5)
    for m in (3, 5):
        for c in range(len(tree.dofs)):
            for sn in tree.sons[c]:
                x = tree.center[sn] + (rng.random((7, 2)) - 0.5) * tree.side[sn]
                S = shift_matrix(tree, c, sn, m)
                assert np.allclose(lagrange(tree, sn, m, x) @ S, lagrange(tree, c, m, x), atol=1e-11)
    # Chebyshev points are the interpolation nodes: L_alpha(xi_beta) = delta
    assert np.allclose(lagrange(tree, 0, 4, cheb_points(tree, 0, 4)), np.eye(16), atol=1e-13)


def test_leaf_coefficients_exact_integrals():
    # sum_alpha p(xi_alpha) int phi_i L_alpha = int phi_i p for polynomials p of degree < m per
    # variable; for p = x (linear) the integrals are M x with the P1 mass matrix on all
    # vertices (x is interpolated exactly), for p = 1 they are int phi_i = M 1
    V, T = synth.square(5, 0.2)
    om = OracleMesh(V, T)
    s = 0.3  # all vertices are DOFs in paper mode
    tree = ClusterTree(om, s, 3, "paper")
    M = mass_matrix(om, s, "paper")
    X = om.V[tree.vod]
    for c in range(len(tree.dofs)):
        if tree.sons[c]:
            continue
        coef = leaf_coefficients(tree, c, 4)
        xi = cheb_points(tree, c, 4)
        rows = tree.dofs[c]
        assert np.allclose(coef @ np.ones(16), (M @ np.ones(tree.n))[rows], rtol=1e-13, atol=1e-16)
        assert np.allclose(coef @ xi[:, 0], (M @ X[:, 0])[rows], rtol=1e-12, atol=1e-15)
        assert np.allclose(coef @ (2 * xi[:, 0] - 3 * xi[:, 1]), (M @ (2 * X[:, 0] - 3 * X[:, 1]))[rows],
                           rtol=1e-12, atol=1e-15)


def test_hmatvec_converges_to_dense_product(disc):
    om, A = disc
    x = np.random.default_rng(2).standard_normal(A.shape[0])
    ref = A @ x
    errs = [np.linalg.norm(hmatvec(A, om, 0.5, x, m=m, eta=1.0, leaf=4) - ref) / np.linalg.norm(ref)
            for m in (2, 3, 4, 5, 6)]
    print("relative error by Chebyshev order 2..6:", errs)
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6
    # no admissible pair (eta = 0): the product is the dense one
    assert np.allclose(hmatvec(A, om, 0.5, x, m=2, eta=0.0, leaf=4), ref, rtol=1e-13, atol=1e-13)


def test_hmatvec_1d():
    V, T = synth.graded_interval(48, 2.0)
    om = OracleMesh(V, T)
    A, _ = assemble_matrix(om, 0.25)
    x = np.cos(np.arange(A.shape[0]))
    ref = A @ x
    errs = [np.linalg.norm(hmatvec(A, om, 0.25, x, m=m, leaf=2) - ref) / np.linalg.norm(ref) for m in (2, 4, 6, 8)]
    assert all(b < a for a, b in zip(errs, errs[1:])) and errs[-1] < 1e-7
    assert kernel_matrix(ClusterTree(om, 0.25, 2), 1, 2, 3, 0.25).shape == (3, 3)
