"""GPU parity of the learned patch preconditioner (sample rows, float16 stencil table,
symmetric apply, gradients of the training loss) against the oracle (oracle/mlp.py),
and flexible CG with it and with the fallback."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import OracleMesh, assemble_matrix  # noqa: E402
from oracle.mlp import apply as o_apply  # noqa: E402
from oracle.mlp import coefficients, geometry, loss_grad, patches, residual_patch  # noqa: E402
from oracle.solve import cholesky_solve  # noqa: E402
from paper_1708_03912_gb300 import fraclap as F  # noqa: E402
from paper_1708_03912_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
K, H, KO = 12, 64, 13
FG = 2 * K + 3


def unpack(w):
    o = 0
    out = []
    for shape in ((FG, H), (H,), (H, H), (H,), (H, KO), (KO,)):
        size = int(np.prod(shape))
        out.append(np.asarray(w[o:o + size], dtype=np.float64).reshape(shape))
        o += size
    return out


def randomised(lp, seed, scale):
    rng = np.random.default_rng(seed)
    w = lp.params()
    tail = H * KO + KO
    w[-tail:] = rng.standard_normal(tail).astype(np.float32) * scale
    lp.set_params(w)
    return w


@pytest.fixture(scope="module")
def small():
    V, T = synth.square(7, 0.2)
    s = 0.6
    m = OracleMesh(V, T)
    A, _ = assemble_matrix(m, s)
    return V, T, s, m, 0.5 * (A + A.T)


def test_samples_stencil_and_apply(small):
    V, T, s, om, A = small
    h = F.fl_create(V, T)
    lp = F.LearnedPreconditioner(h, s, seed=3)
    w = randomised(lp, 8, 0.05)
    Ad = torch.tensor(A, device="cuda")
    lp.bind(Ad)
    r = np.random.default_rng(8).standard_normal(A.shape[0])
    X, sig = lp.features(torch.tensor(r, device="cuda"))
    nbr, hl, hop = patches(om, s, K)
    G = geometry(om, s, nbr, hl, hop)
    xr, so = residual_patch(r, nbr)
    assert np.allclose(X.cpu().numpy(), np.concatenate([G, xr], axis=1), rtol=2e-6, atol=2e-6)
    assert np.allclose(sig.cpu().numpy(), so, rtol=1e-6)
    w16 = unpack(w.astype(np.float16).astype(np.float64))  # the stencil is computed with float16 weights
    C, _ = coefficients(w16, G)
    assert np.abs(lp.stencil() - C).max() < 1e-5
    z = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    lp.apply(torch.tensor(r, device="cuda"), z)
    zo = o_apply(w16, G, nbr, np.diag(A), r)
    err = np.abs(z.cpu().numpy() - zo).max() / np.abs(zo).max()
    print(f"stencil apply vs oracle: {err:.2e}")
    assert err < 1e-5
    lp.close()
    F.fl_destroy(h)


def test_gradients_against_oracle(small):
    V, T, s, om, A = small
    h = F.fl_create(V, T)
    lp = F.LearnedPreconditioner(h, s, seed=5)
    w = randomised(lp, 9, 0.3)
    rng = np.random.default_rng(9)
    B = 777  # not a multiple of the block size
    X = rng.standard_normal((B, lp.F)).astype(np.float32)
    Tt = rng.standard_normal(B).astype(np.float32)
    loss, g = lp.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(Tt, device="cuda"))
    lo, go = loss_grad(unpack(w), X[:, :FG].astype(np.float64), X[:, FG:].astype(np.float64), Tt.astype(np.float64))
    assert loss == pytest.approx(lo, rel=1e-4)
    gflat = np.concatenate([np.ravel(x) for x in go])
    err = np.abs(g - gflat).max() / np.abs(gflat).max()
    print(f"gradient float32 vs oracle float64: {err:.2e}")
    assert err < 1e-4
    lp.close()
    F.fl_destroy(h)


def test_fcg_fallback_and_exactness(small):
    V, T, s, om, A = small
    h = F.fl_create(V, T)
    lp = F.LearnedPreconditioner(h, s, seed=5)
    Ad = torch.tensor(A, device="cuda")
    b = np.random.default_rng(11).standard_normal(A.shape[0])
    bd = torch.tensor(b, device="cuda")
    u = torch.empty_like(bd)
    uo = cholesky_solve(A, b)
    # untrained network = Jacobi: converges, no fallback
    info = F.fl_fcg_solve(h, Ad, bd, u, lp=lp, tol=1e-12)
    assert info.status == F.FL_OK and info.fallback_at == -1 and info.rel_residual <= 1e-12
    assert np.abs(u.cpu().numpy() - uo).max() <= 1e-8 * np.abs(uo).max()
    # a stencil that is not positive: flexible CG hands over to Jacobi and still converges
    w = lp.params()
    w[-KO] = -3.0  # b3[0]: diagonal coefficient 1 - 3 < 0
    lp.set_params(w)
    info = F.fl_fcg_solve(h, Ad, bd, u, lp=lp, tol=1e-10)
    assert info.status == F.FL_OK and info.fallback_at >= 1 and info.final_preconditioner == 0
    assert np.abs(u.cpu().numpy() - uo).max() <= 1e-6 * np.abs(uo).max()
    lp.close()
    F.fl_destroy(h)


def test_training_gains_over_jacobi():
    # trained on the method's own CG pairs (noise-started Jacobi-PCG iterates on A x = 0),
    # the learned stencil takes fewer flexible-CG steps than Jacobi-PCG, and the answer is
    # the float64 one
    V, T = synth.lshape(0.25, 2)
    s = 0.5
    m = F.Mesh(V, T)
    A = m.assemble(s, "fp64")
    b = m.load_vector(s)
    lp = F.LearnedPreconditioner(m.h, s, seed=1)
    lp.collect_noise(A, 8, [0, 1, 2, 4])
    first = lp.train(1, batch=8192, lr=1e-9)
    loss = lp.train(2000, batch=8192, lr=1e-3)
    assert loss < 0.5 * first
    u = torch.empty_like(b)
    uj, ij = m.solve(A, b, tol=1e-10)
    info = F.fl_fcg_solve(m.h, A, b, u, lp=lp, tol=1e-10)
    print(f"L-shape n = {A.shape[0]}: Jacobi-PCG {ij.iterations} steps, learned flexible CG {info.iterations}")
    assert info.status == F.FL_OK and info.fallback_at == -1 and info.rel_residual <= 1e-10
    assert info.iterations <= 0.9 * ij.iterations
    assert torch.allclose(u, uj, rtol=0, atol=1e-7 * float(uj.abs().max()))
    lp.close()
    m.close()
