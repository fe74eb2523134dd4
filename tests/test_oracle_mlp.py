"""Pins of the learned-preconditioner oracle (oracle/mlp.py).  No GPU."""
import numpy as np
import pytest

from oracle import OracleMesh, assemble_matrix
from oracle.mlp import apply, coefficients, geometry, loss_grad, patches, residual_patch, stencil_matrix
from paper_1708_03912_gb300 import synth


def weights(Fg, H, Ko, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((Fg, H)) * scale, rng.standard_normal(H) * scale,
            rng.standard_normal((H, H)) * scale, rng.standard_normal(H) * scale,
            rng.standard_normal((H, Ko)) * scale, rng.standard_normal(Ko) * scale]


def test_gradient_matches_finite_differences():
    Fg, H, Ko, B = 5, 4, 3, 9
    rng = np.random.default_rng(1)
    G = rng.standard_normal((B, Fg))
    X = rng.standard_normal((B, Ko))
    t = rng.standard_normal(B)
    W = weights(Fg, H, Ko, 2)
    _, grads = loss_grad(W, G, X, t)
    eps = 1e-6
    for p in range(6):
        gflat = np.asarray(grads[p]).reshape(-1)
        for idx in range(W[p].size):
            Wp = [w.copy() for w in W]
            Wm = [w.copy() for w in W]
            Wp[p].reshape(-1)[idx] += eps
            Wm[p].reshape(-1)[idx] -= eps
            fd = (loss_grad(Wp, G, X, t)[0] - loss_grad(Wm, G, X, t)[0]) / (2 * eps)
            assert abs(fd - gflat[idx]) <= 1e-7 * max(1.0, abs(fd))


def test_patches_geometry_and_residual_patch():
    V, T = synth.square(5, 0.2)
    m = OracleMesh(V, T)
    s = 0.4
    nbr, h, hop = patches(m, s, K=6)
    dofs, _ = m.dofs(s)
    X = V[dofs]
    for i in range(len(dofs)):
        ks = nbr[i][nbr[i] >= 0]
        d = np.linalg.norm(X[ks] - X[i], axis=1)
        assert np.all(np.diff(d) >= -1e-15) and i not in ks  # ordered by distance, centre excluded
    assert hop.min() >= 1 and hop.max() <= 8
    G = geometry(m, s, nbr, h, hop)
    i = 7
    j = nbr[i, 0]
    assert G[i, 0] * h[i] == pytest.approx(X[j, 0] - X[i, 0])
    assert G[i, -1] == s and G[i, -2] == hop[i] / 8 and G[i, -3] == pytest.approx(np.log(h[i]))
    r = np.random.default_rng(4).standard_normal(len(dofs))
    x, sig = residual_patch(r, nbr)
    ks = nbr[i][nbr[i] >= 0]
    assert sig[i] == pytest.approx(np.sqrt((r[i] ** 2 + np.sum(r[ks] ** 2)) / (1 + len(ks))), rel=1e-12)
    assert x[i, 0] * sig[i] == pytest.approx(r[i]) and x[i, 1] * sig[i] == pytest.approx(r[ks[0]])


def test_jacobi_limit_and_symmetric_apply():
    V, T = synth.square(5, 0.2)
    m = OracleMesh(V, T)
    s = 0.6
    A, _ = assemble_matrix(m, s)
    nbr, h, hop = patches(m, s, K=12)
    G = geometry(m, s, nbr, h, hop)
    d = np.diag(A)
    r = np.random.default_rng(5).standard_normal(A.shape[0])
    W = weights(G.shape[1], 8, 13, 6)
    W[4] = np.zeros((8, 13))
    W[5] = np.zeros(13)
    assert np.allclose(apply(W, G, nbr, d, r), r / d, rtol=1e-14, atol=0)
    W = weights(G.shape[1], 8, 13, 7)
    C, _ = coefficients(W, G)
    M = stencil_matrix(C, nbr, d)
    assert np.allclose(apply(W, G, nbr, d, r), 0.5 * (M + M.T) @ r)
    # the prediction of a sample is the normalised i-th entry of M r
    x, sig = residual_patch(r, nbr)
    assert np.allclose(np.sum(C * x, axis=1) * sig / d, M @ r)
