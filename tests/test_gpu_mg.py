"""GPU parity of the Galerkin multigrid (fl_prolongation, fl_mg_*) against the oracle
(oracle/multigrid.py) on nested meshes, and its use as a CG preconditioner."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import OracleMesh, assemble_matrix  # noqa: E402
from oracle.multigrid import galerkin, hierarchy, jacobi_weight, prolongation, vcycle  # noqa: E402
from oracle.solve import cholesky_solve  # noqa: E402
from paper_1708_03912_gb300 import fraclap as F  # noqa: E402
from paper_1708_03912_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
S = 0.5


@pytest.fixture(scope="module")
def three_levels():
    V0, T0 = synth.square(4, 0.1)
    V1, T1 = synth.bisect_all(V0, T0, 2)
    V2, T2 = synth.bisect_all(V1, T1, 1)
    meshes = [(V2, T2), (V1, T1), (V0, T0)]  # fine to coarse
    om = [OracleMesh(V, T) for V, T in meshes]
    A, _ = assemble_matrix(om[0], S)
    A = 0.5 * (A + A.T)
    Ps = [prolongation(meshes[k][0], om[k].dofs(S)[0], meshes[k + 1][0], meshes[k + 1][1], om[k + 1].dofs(S)[0])
          for k in range(2)]
    return meshes, A, Ps


def build_mg(meshes, A_dev):
    hs = [F.fl_create(V, T) for V, T in meshes]
    mg = F.Multigrid(A_dev)
    for k in range(len(meshes) - 1):
        ptr, col, val = F.fl_prolongation(hs[k], hs[k + 1], S)
        mg.add_level(ptr, col, val, F.fl_num_dofs(hs[k + 1], S))
    for h in hs:
        F.fl_destroy(h)
    return mg


def test_galerkin_levels_and_weights(three_levels):
    meshes, A, Ps = three_levels
    Ad = torch.tensor(A, device="cuda")
    mg = build_mg(meshes, Ad)
    mg.setup(nu=2)
    As = hierarchy(A, Ps)
    for k in (1, 2):
        Ak = mg.level_matrix(k).cpu().numpy()
        assert Ak.shape == As[k].shape
        assert np.abs(Ak - As[k]).max() <= 1e-12 * np.abs(As[k]).max()
    for k in (0, 1):
        assert mg.omega(k) == pytest.approx(jacobi_weight(As[k]), rel=1e-5)
    mg.close()


def test_vcycle_parity(three_levels):
    meshes, A, Ps = three_levels
    Ad = torch.tensor(A, device="cuda")
    mg = build_mg(meshes, Ad)
    mg.setup(nu=2)
    As = hierarchy(A, Ps)
    rng = np.random.default_rng(3)
    for _ in range(3):
        r = rng.standard_normal(A.shape[0]).astype(np.float32)
        z = torch.zeros(A.shape[0], dtype=torch.float32, device="cuda")
        mg.vcycle(torch.tensor(r, device="cuda"), z)
        zo = vcycle(As, Ps, r.astype(np.float64), nu=2)
        err = np.abs(z.cpu().numpy() - zo).max() / np.abs(zo).max()
        print(f"V-cycle float32 vs oracle float64: {err:.2e}")
        assert err < 2e-4
    mg.close()


def test_mg_preconditioned_cg_solves(three_levels):
    meshes, A, Ps = three_levels
    Ad = torch.tensor(A, device="cuda")
    mg = build_mg(meshes, Ad)
    mg.setup(nu=2)
    b = np.random.default_rng(5).standard_normal(A.shape[0])
    u = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    info = mg.solve(torch.tensor(b, device="cuda"), u, tol=1e-12, maxit=200)
    assert info.status == F.FL_OK
    uo = cholesky_solve(A, b)
    assert np.abs(u.cpu().numpy() - uo).max() <= 1e-8 * np.abs(uo).max()
    mg.close()


def test_mg_beats_jacobi_on_the_lshape():
    # nested L-shape levels (refined towards the corner and the boundary), GPU-assembled
    meshes = [synth.lshape(0.25, 2), synth.lshape(0.25, 1)]
    m = F.Mesh(*meshes[0])
    A = m.assemble(S, "fp64")
    b = m.load_vector(S)
    mg = build_mg(meshes, A)
    mg.setup(nu=2)
    u = torch.empty_like(b)
    imf = mg.solve(b, u, tol=1e-8, maxit=500)
    _, ij = m.solve(A, b, tol=1e-8)
    print(f"L-shape n = {A.shape[0]}: MG-PCG {imf.iterations} iterations, Jacobi-PCG {ij.iterations}")
    assert imf.status == F.FL_OK and imf.iterations * 3 < ij.iterations
    mg.close()
    m.close()
