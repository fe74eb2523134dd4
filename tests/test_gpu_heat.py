"""GPU parity of the fractional heat equation pieces (Sections 2 and 5) through the C ABI:
the implicit-step matrix M + dt A and the mass product against the oracle, implicit Euler
steps against the oracle's, and the conditioning statement of Section 5 (with dt of order
h^{2s} the diagonally preconditioned CG needs a bounded number of iterations)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import OracleMesh, assemble_matrix, load_vector  # noqa: E402
from oracle.heat import heat_matrix, implicit_euler, mass_matrix  # noqa: E402
from paper_1708_03912_gb300 import fraclap as F  # noqa: E402
from paper_1708_03912_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["disc", "interval"])
def test_heat_matrix_and_mass_apply(case):
    (V, T), s = {"disc": (synth.disc(8), 0.5), "interval": (synth.graded_interval(40, 2.0), 0.3)}[case]
    om = OracleMesh(V, T)
    Ao, _ = assemble_matrix(om, s)
    Mo = mass_matrix(om, s)
    m = F.Mesh(V, T)
    A = m.assemble(s, "fp64")
    n = A.shape[0]
    dt = 0.037
    H = torch.empty_like(A)
    F.fl_heat_matrix(m.h, s, dt, A, H)
    Ho = heat_matrix(Ao, Mo, dt)
    d = np.sqrt(np.outer(np.diag(Ho), np.diag(Ho)))
    assert float(np.max(np.abs(H.cpu().numpy() - Ho) / d)) < 1e-12
    # in place, and dt = 0 gives M exactly as the oracle sums it (up to the summation order)
    A2 = A.clone()
    F.fl_heat_matrix(m.h, s, 0.0, A2, A2)
    assert np.allclose(A2.cpu().numpy(), Mo, rtol=1e-15, atol=1e-17)
    g = torch.Generator().manual_seed(3)
    X = torch.randn(n, 3, generator=g, dtype=torch.float64).cuda()
    B = torch.randn(n, 3, generator=g, dtype=torch.float64).cuda()
    Y = torch.empty_like(X)
    F.fl_mass_apply(m.h, s, 2.0, X, -0.5, B, Y)
    ref = 2.0 * Mo @ X.cpu().numpy() - 0.5 * B.cpu().numpy()
    assert np.allclose(Y.cpu().numpy(), ref, rtol=1e-13, atol=1e-15)
    with pytest.raises(F.FlError):
        F.fl_mass_apply(m.h, s, 1.0, X, 0.0, None, X)  # Y = X
    with pytest.raises(F.FlError):
        F.fl_heat_matrix(m.h, s, -1.0, A, H)
    m.close()


def test_implicit_euler_steps_match_oracle():
    V, T = synth.disc(6)
    s = 0.75
    om = OracleMesh(V, T)
    Ao, _ = assemble_matrix(om, s)
    Ao = 0.5 * (Ao + Ao.T)
    Mo = mass_matrix(om, s)
    Fo = load_vector(om, s)
    m = F.Mesh(V, T)
    A = m.assemble(s, "fp64")
    b = m.load_vector(s)
    u0 = torch.zeros_like(b)
    u, infos = m.heat_steps(A, s, 0.02, u0, b, 4, tol=1e-13)
    uo = implicit_euler(Ao, Mo, Fo, np.zeros_like(Fo), 0.02, 4)[-1]
    assert all(i.status == F.FL_OK for i in infos)
    assert float(np.max(np.abs(u.cpu().numpy() - uo)) / np.max(np.abs(uo))) < 1e-10
    m.close()


def test_heat_conditioning_bounded_iterations():
    # Section 5: with dt = h^{2s} the Jacobi-preconditioned system M + dt A has a condition
    # number bounded independently of h, so CG iterations stay flat under refinement while
    # those of A itself grow like n^{s/d}
    s = 0.75
    its_heat, its_a = [], []
    for M_rings in (8, 16, 32):
        V, T = synth.disc(M_rings)
        m = F.Mesh(V, T)
        A = m.assemble(s, "fp64")
        b = m.load_vector(s)
        h = 1.0 / M_rings
        u, infos = m.heat_steps(A, s, h ** (2 * s), torch.zeros_like(b), b, 1, tol=1e-8)
        its_heat.append(infos[0].iterations)
        _, ia = m.solve(A, b, tol=1e-8)
        its_a.append(ia.iterations)
        m.close()
    print("iterations M + h^2s A:", its_heat, " A:", its_a)
    assert max(its_heat) <= 1.3 * min(its_heat) + 2
    assert its_a[-1] > 1.5 * its_a[0]
