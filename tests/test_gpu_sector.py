"""GPU parity of the symmetry-reduced problem (Section 7, "Exploiting Symmetry") against the
oracle: the reduced matrix (representatives' rows of the whole matrix, folded over the orbits,
symmetric part), the folded load vector and the reduced solution, on K-fold sectors."""
import numpy as np
import pytest

from oracle import solve
from oracle import symmetry as sym
from paper_1708_03912_gb300 import synth

pytestmark = pytest.mark.gpu


def _f(V, s):
    # f_{2,8} of Section 7 (periodic under the rotation by pi/4), at the vertices
    from scipy import special

    r2 = np.sum(V ** 2, axis=1)
    th = np.arctan2(V[:, 1], V[:, 0])
    lam = 2 ** (2 * s) * special.gamma(3 + s) * special.gamma(11 + s) / (special.gamma(3) * special.gamma(11))
    return lam * r2 ** 4 * np.cos(8 * th) * special.eval_jacobi(2, s, 8, 2 * r2 - 1)


@pytest.mark.parametrize("K,M,s", [(8, 5, 0.25), (8, 5, 0.5), (8, 8, 0.75), (4, 6, 0.5), (6, 6, 0.3)])
def test_reduced_matrix_load_and_solution(K, M, s):
    import torch
    from paper_1708_03912_gb300.fraclap import Mesh

    V, T = synth.sector(K, M)
    Ao, bo, reps = sym.reduced_system(V, T, K, s)
    m = Mesh.sector(V, T, K)
    assert m.num_dofs(s) == len(reps)
    A = m.assemble(s).cpu().numpy()
    assert np.array_equal(A, A.T)
    d = np.sqrt(np.outer(np.diag(Ao), np.diag(Ao)))
    err = np.max(np.abs(A - Ao) / d)
    print(K, M, s, "matrix", err)
    assert err < 1e-12
    b = m.load_vector(s).cpu().numpy()
    assert np.max(np.abs(b - bo)) <= 1e-14 * np.max(np.abs(bo))
    # nodal f on the sector's vertices
    f = _f(V, s) if K == 8 else np.cos(K * np.arctan2(V[:, 1], V[:, 0])) * np.sum(V ** 2, axis=1)
    _, bf, _ = sym.reduced_system(V, T, K, s, f_sector=f)
    bg = m.load_vector(s, torch.tensor(f, device="cuda")).cpu().numpy()
    assert np.max(np.abs(bg - bf)) <= 1e-13 * np.max(np.abs(bf))
    # the reduced solution
    u, info = m.solve(m.assemble(s), torch.tensor(bf, device="cuda"), tol=1e-12)
    uo = solve.cholesky_solve(Ao, bf)
    assert np.max(np.abs(u.cpu().numpy() - uo)) <= 1e-8 * np.max(np.abs(uo))
    m.close()


def test_mixed_precision_and_far_pipe():
    import torch
    from paper_1708_03912_gb300.fraclap import Mesh

    K, s = 8, 0.5
    V, T = synth.sector(K, 8)
    Ao, _, _ = sym.reduced_system(V, T, K, s)
    d = np.sqrt(np.outer(np.diag(Ao), np.diag(Ao)))
    am = Mesh.sector(V, T, K).assemble(s, "mixed").cpu().numpy()
    assert np.max(np.abs(am - Ao) / d) < 2e-5
    af = Mesh.sector(V, T, K, far_f64_pipe=True).assemble(s).cpu().numpy()
    assert np.max(np.abs(af - Ao) / d) < 1e-12


def test_reduced_against_whole_mesh_on_gpu():
    # the reduced solution equals the whole mesh's GPU solution on every orbit (to the
    # quadrature's rotation defect); the reduced assembly evaluates fewer element pairs
    import torch
    from paper_1708_03912_gb300 import fraclap as F
    from paper_1708_03912_gb300.fraclap import Mesh

    K, s = 8, 0.5
    V, T = synth.sector(K, 16)
    W, C, vmap, _ = sym.replicate(V, T, K)
    mw = Mesh(W, C)
    Aw = mw.assemble(s)
    uw, _ = mw.solve(Aw, mw.load_vector(s), tol=1e-12)
    ms = Mesh.sector(V, T, K)
    ur, _ = ms.solve(ms.assemble(s), ms.load_vector(s), tol=1e-12)
    vod_w = F.fl_dof_vertices(mw.h, s)
    dov_w = -np.ones(len(W), dtype=np.int64)
    dov_w[vod_w] = np.arange(len(vod_w))
    reps = F.fl_dof_vertices(ms.h, s)
    uwn = uw.cpu().numpy()
    got = ur.cpu().numpy()
    want = uwn[dov_w[vmap[0][reps]]]
    assert np.max(np.abs(got - want)) < 1e-5 * np.max(np.abs(want))
    tw = F.fl_get_stats(mw.h, s)["n_tiles"]
    tr = F.fl_get_stats(ms.h, s)["n_tiles"]
    print("tiles reduced / whole", tr, tw)
    assert tr < 0.5 * tw
