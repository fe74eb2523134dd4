"""Pins of the oracle's fractional heat equation pieces (Sections 2 and 5): the P1 mass
matrix against exact integrals, the implicit Euler step against the generalised
eigen-decomposition of (A, M) and against the steady state."""
import numpy as np
import scipy.linalg

from oracle import OracleMesh, assemble_matrix, load_vector
from oracle.heat import heat_matrix, implicit_euler, mass_matrix
from paper_1708_03912_gb300 import synth


def test_mass_matrix_exact_integrals():
    # all vertices as DOFs (paper mode, s < 1/2): 1^T M 1 = |Omega|, M 1 = int phi_i (the load
    # vector of f = 1, pinned separately by the midpoint rule), and u^T M u = int u^2 for the
    # linear function u = 1 + 2x - y, interpolated exactly by P1 (int over [-1,1]^2 by hand:
    # int (1 + 2x - y)^2 = 4 + 4 * 4/3 + 4/3 = 4 + 20/3)
    V, T = synth.square(6, 0.2)
    om = OracleMesh(V, T)
    M = mass_matrix(om, 0.3, "paper")
    one = np.ones(om.nv)
    assert abs(one @ M @ one - 4.0) < 1e-13
    assert np.allclose(M @ one, load_vector(om, 0.3, dof_mode="paper"), rtol=1e-13, atol=0)
    u = 1 + 2 * om.V[:, 0] - om.V[:, 1]
    assert abs(u @ M @ u - (4.0 + 20.0 / 3.0)) < 1e-12
    # 1D: int_{-1}^{1} x^2 = 2/3 for u = x
    V1, T1 = synth.graded_interval(17, 2.0)
    o1 = OracleMesh(V1, T1)
    M1 = mass_matrix(o1, 0.2, "paper")
    x = o1.V[:, 0]
    assert abs(x @ M1 @ x - 2.0 / 3.0) < 1e-13
    # interior DOFs: the principal submatrix, symmetric positive definite
    Mi = mass_matrix(om, 0.7)
    vod, _ = om.dofs(0.7)
    assert np.array_equal(Mi, M[np.ix_(vod, vod)])
    assert np.all(np.linalg.eigvalsh(Mi) > 0)


def test_implicit_euler_against_eigenpairs_and_steady_state():
    V, T = synth.disc(4)
    om = OracleMesh(V, T)
    s = 0.6
    A, _ = assemble_matrix(om, s)
    A = 0.5 * (A + A.T)
    M = mass_matrix(om, s)
    F = load_vector(om, s)
    lam, W = scipy.linalg.eigh(A, M)  # A w = lam M w, W^T M W = I
    dt = 0.05
    # f = 0, u0 = sum c_k w_k: after m steps u = sum c_k w_k / (1 + dt lam_k)^m
    c = np.linspace(1.0, -1.0, len(lam))
    u0 = W @ c
    us = implicit_euler(A, M, np.zeros_like(F), u0, dt, 3)
    for m in range(4):
        assert np.allclose(us[m], W @ (c / (1 + dt * lam) ** m), rtol=1e-10, atol=1e-12)
    # f = 1 from u0 = 0: the iterates approach the steady state A^{-1} F geometrically with the
    # slowest factor 1 / (1 + dt lam_min)
    u_inf = np.linalg.solve(A, F)
    us = implicit_euler(A, M, F, np.zeros_like(F), 1.0, 40)
    rate = 1.0 / (1.0 + lam.min())
    err = [np.linalg.norm(u - u_inf) for u in us]
    assert err[-1] < 1e-6 * err[0]
    assert err[20] / err[19] < rate * 1.001
    assert np.allclose(heat_matrix(A, M, 0.0), M)
