"""GPU parity of the cluster method (Section 6) through the C ABI: the H-matrix product
against the oracle's restatement (same tree, partition and Chebyshev data, near entries
from the float64 matrices), and against the dense product with an error that falls
geometrically with the Chebyshev order."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import OracleMesh, assemble_matrix  # noqa: E402
from oracle.cluster import hmatvec  # noqa: E402
from paper_1708_03912_gb300 import fraclap as F  # noqa: E402
from paper_1708_03912_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["disc", "interval"])
def test_hmatrix_product_matches_oracle(case):
    (V, T), s, leaf, m, eta = {"disc": (synth.disc(7, 2.0), 0.5, 4, 4, 1.0),
                               "interval": (synth.graded_interval(60, 2.0), 0.25, 2, 5, 1.0)}[case]
    om = OracleMesh(V, T)
    Ao, _ = assemble_matrix(om, s)
    x = np.sin(np.arange(Ao.shape[0]) * 0.37)
    yo = hmatvec(Ao, om, s, x, m=m, eta=eta, leaf=leaf)
    mesh = F.Mesh(V, T)
    A = mesh.assemble(s, "fp64")
    H = F.HMatrix(mesh.h, s, m=m, eta=eta, leaf=leaf)
    H.set_near(A)
    xd = torch.tensor(x, device="cuda")
    y = torch.full_like(xd, float("nan"))
    H.matvec(xd, y)
    y2 = torch.empty_like(y)
    H.matvec(xd, y2)
    torch.cuda.synchronize()
    assert torch.equal(y, y2)  # fixed summation order
    yg = y.cpu().numpy()
    err = np.linalg.norm(yg - yo) / np.linalg.norm(yo)
    print(f"{case}: GPU H-matrix product vs oracle: {err:.2e}; info {H.info()}")
    assert err < 1e-12
    H.close()
    mesh.close()


def test_hmatrix_converges_to_dense_product():
    V, T = synth.lshape(0.25, 3)  # 19188 triangles, n = 9083
    s = 0.5
    mesh = F.Mesh(V, T)
    A = mesh.assemble(s, "fp64")
    n = A.shape[0]
    g = torch.Generator().manual_seed(7)
    x = torch.randn(n, generator=g, dtype=torch.float64).cuda()
    ref = A @ x
    errs = []
    for m in (2, 3, 4, 5, 6):
        H = F.HMatrix(mesh.h, s, m=m, eta=1.0, leaf=32)
        H.set_near(A)
        y = torch.empty_like(x)
        H.matvec(x, y)
        errs.append(float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref)))
        info = H.info()
        H.close()
    print("H-matrix relative error by Chebyshev order 2..6:", errs, info)
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6
    assert info["near_entries"] < 0.25 * n * n  # the near field is a small part of the matrix
    mesh.close()


def test_hmatrix_errors():
    V, T = synth.disc(5)
    mesh = F.Mesh(V, T)
    H = F.HMatrix(mesh.h, 0.5, m=3, leaf=4)
    x = torch.ones(mesh.num_dofs(0.5), dtype=torch.float64, device="cuda")
    with pytest.raises(F.FlError):
        H.matvec(x, torch.empty_like(x))  # no near field yet
    H.set_near(mesh.assemble(0.5, "fp64"))
    with pytest.raises(F.FlError):
        H.matvec(x, x)
    with pytest.raises(F.FlError):
        F.HMatrix(mesh.h, 0.5, m=0)
    H.close()
    mesh.close()


def test_hmatrix_solve():
    # Jacobi-PCG with the H-matrix product (Section 5's solver, Section 6's operator): the
    # returned u satisfies the stated residual with the oracle's H-matrix product, and it is
    # the dense solution up to the far field's interpolation error
    from oracle import load_vector, solve

    V, T = synth.disc(7, 2.0)
    s, m, leaf = 0.5, 6, 4
    om = OracleMesh(V, T)
    Ao, _ = assemble_matrix(om, s)
    bo = load_vector(om, s)
    mesh = F.Mesh(V, T)
    A = mesh.assemble(s, "fp64")
    H = F.HMatrix(mesh.h, s, m=m, eta=1.0, leaf=leaf)
    H.set_near(A)
    b = torch.tensor(bo, device="cuda")
    u, info = H.solve(b, tol=1e-10)
    assert info.status == F.FL_OK and info.rel_residual <= 1e-10
    ug = u.cpu().numpy()
    res = np.linalg.norm(bo - hmatvec(Ao, om, s, ug, m=m, eta=1.0, leaf=leaf)) / np.linalg.norm(bo)
    assert res <= 2e-10, res
    uo = solve.cholesky_solve(Ao, bo)
    err = np.max(np.abs(ug - uo)) / np.max(np.abs(uo))
    _, idense = mesh.solve(A, b, tol=1e-10)
    print(f"H-matrix solve: {info.iterations} steps (dense {idense.iterations}), residual {res:.1e}, "
          f"error vs dense {err:.1e}")
    assert err < 1e-6
    assert abs(info.iterations - idense.iterations) <= 3
    # a limit of one step reports that it did not converge
    _, i1 = H.solve(b, tol=1e-12, maxit=1)
    assert i1.status == F.FL_ENOTCONV and i1.iterations == 1
    H.close()
    mesh.close()
