"""Pins of the multigrid oracle (oracle/multigrid.py).  No GPU."""
import numpy as np
import pytest

from oracle import OracleMesh, QuadOrders, assemble_matrix
from oracle.multigrid import galerkin, hierarchy, jacobi_weight, prolongation, vcycle, vcycle_matrix
from paper_1708_03912_gb300 import synth

HIGH = QuadOrders(8, 10, 12, 12, k_vertex=10)


@pytest.fixture(scope="module")
def nested():
    Vc, Tc = synth.square(3, 0.15)
    Vf, Tf = synth.bisect_all(Vc, Tc, 2)
    return Vc, Tc, Vf, Tf


def test_galerkin_product_equals_coarse_assembly(nested):
    # nested spaces: the coarse bilinear form restricted from the fine one (exact up to quadrature)
    Vc, Tc, Vf, Tf = nested
    s = 0.6
    oc, of = OracleMesh(Vc, Tc), OracleMesh(Vf, Tf)
    Ac, _ = assemble_matrix(oc, s, HIGH)
    Af, _ = assemble_matrix(of, s, HIGH)
    P = prolongation(Vf, of.dofs(s)[0], Vc, Tc, oc.dofs(s)[0])
    assert np.abs(galerkin(Af, P) - Ac).max() < 2e-6 * np.abs(Ac).max()


def test_prolongation_reproduces_linear_functions(nested):
    Vc, Tc, Vf, Tf = nested
    f = lambda X: 0.3 + 1.7 * X[:, 0] - 0.9 * X[:, 1]  # noqa: E731
    P = prolongation(Vf, np.arange(len(Vf)), Vc, Tc, np.arange(len(Vc)))
    assert np.allclose(P @ f(Vc), f(Vf), rtol=0, atol=1e-13)
    assert np.allclose(P.sum(axis=1), 1.0, atol=1e-13)  # partition of unity
    assert (P >= -1e-14).all() and (P.max(axis=1) <= 1 + 1e-14).all()


def test_coarse_correction_is_a_projector_and_vcycle_contracts(nested):
    Vc, Tc, Vf, Tf = nested
    s = 0.5
    oc, of = OracleMesh(Vc, Tc), OracleMesh(Vf, Tf)
    Af, _ = assemble_matrix(of, s)
    Af = 0.5 * (Af + Af.T)
    P = prolongation(Vf, of.dofs(s)[0], Vc, Tc, oc.dofs(s)[0])
    As = hierarchy(Af, [P])
    Q = P @ np.linalg.solve(As[1], P.T @ Af)
    assert np.allclose(Q @ Q, Q, atol=1e-10)  # A-orthogonal projection onto the coarse space
    M = vcycle_matrix(As, [P], nu=2)
    assert np.allclose(M, M.T, atol=1e-12 * np.abs(M).max())  # symmetric V-cycle
    ev = np.linalg.eigvals(np.eye(len(Af)) - M @ Af)
    assert np.max(np.abs(ev)) < 0.9  # error propagation contracts
    # without smoothing the V-cycle is exactly the coarse correction
    assert np.allclose(vcycle_matrix(As, [P], nu=0), P @ np.linalg.solve(As[1], P.T), atol=1e-12)
    # and the weight follows its definition
    om = jacobi_weight(Af)
    x = np.ones(len(Af))
    d = 1 / np.diag(Af)
    for _ in range(10):
        y = d * (Af @ x)
        x = y / np.linalg.norm(y)
    assert om == pytest.approx(4 / (3 * np.linalg.norm(d * (Af @ x))), rel=1e-14)


def test_vcycle_beats_jacobi_as_preconditioner(nested):
    Vc, Tc, Vf, Tf = nested
    s = 0.5
    oc, of = OracleMesh(Vc, Tc), OracleMesh(Vf, Tf)
    Af, _ = assemble_matrix(of, s)
    Af = 0.5 * (Af + Af.T)
    P = prolongation(Vf, of.dofs(s)[0], Vc, Tc, oc.dofs(s)[0])
    M = vcycle_matrix(hierarchy(Af, [P]), [P], nu=2)
    d = np.diag(Af)

    def cond(B):
        ev = np.linalg.eigvals(B @ Af).real
        return ev.max() / ev.min()

    assert cond(M) < 0.5 * cond(np.diag(1 / d))
    r = np.random.default_rng(0).standard_normal(len(Af))
    assert np.allclose(vcycle(hierarchy(Af, [P]), [P], r), M @ r, atol=1e-12)
