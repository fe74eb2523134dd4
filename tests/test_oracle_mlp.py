"""Pins of the learned-preconditioner oracle (oracle/mlp.py).  No GPU."""
import numpy as np
import pytest

from oracle import OracleMesh, assemble_matrix
from oracle.mlp import apply, features, forward, loss_grad, patches
from paper_1708_03912_gb300 import synth


def weights(F, H, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((F, H)) * scale, rng.standard_normal(H) * scale,
            rng.standard_normal((H, H)) * scale, rng.standard_normal(H) * scale,
            rng.standard_normal(H) * scale, np.array(rng.standard_normal() * scale)]


def test_gradient_matches_finite_differences():
    F, H, B = 7, 5, 11
    rng = np.random.default_rng(1)
    X = rng.standard_normal((B, F))
    t = rng.standard_normal(B)
    W = weights(F, H, 2)
    L, G = loss_grad(W, X, t)
    eps = 1e-6
    for p in range(6):
        flat = W[p].reshape(-1)
        gflat = np.asarray(G[p]).reshape(-1)
        for idx in range(flat.size):
            Wp = [w.copy() for w in W]
            Wm = [w.copy() for w in W]
            Wp[p].reshape(-1)[idx] += eps
            Wm[p].reshape(-1)[idx] -= eps
            fd = (loss_grad(Wp, X, t)[0] - loss_grad(Wm, X, t)[0]) / (2 * eps)
            assert abs(fd - gflat[idx]) <= 1e-7 * max(1.0, abs(fd))


def test_patches_and_features():
    V, T = synth.square(5, 0.2)
    m = OracleMesh(V, T)
    s = 0.4
    nbr, h, hop = patches(m, s, K=6)
    dofs, dov = m.dofs(s)
    X = V[dofs]
    for i in range(len(dofs)):
        ks = nbr[i][nbr[i] >= 0]
        d = np.linalg.norm(X[ks] - X[i], axis=1)
        assert np.all(np.diff(d) >= -1e-15) and i not in ks  # ordered by distance, centre excluded
    assert hop.min() >= 1 and hop.max() <= 8
    r = np.random.default_rng(4).standard_normal(len(dofs))
    Fx, sig = features(m, s, r, nbr, h, hop)
    i = 7
    ks = nbr[i][nbr[i] >= 0]
    assert sig[i] == pytest.approx(np.sqrt((r[i] ** 2 + np.sum(r[ks] ** 2)) / (1 + len(ks))), rel=1e-12)
    assert Fx[i, 0] * sig[i] == pytest.approx(r[i], rel=1e-14)
    assert Fx[i, 1] * sig[i] == pytest.approx(r[ks[0]], rel=1e-14)
    assert Fx[i, -1] == s and Fx[i, -2] == hop[i] / 8 and Fx[i, -3] == pytest.approx(np.log(h[i]))


def test_zero_output_layer_is_jacobi():
    V, T = synth.square(5, 0.2)
    m = OracleMesh(V, T)
    s = 0.6
    A, _ = assemble_matrix(m, s)
    nbr, h, hop = patches(m, s, K=12)
    r = np.random.default_rng(5).standard_normal(A.shape[0])
    Fx, sig = features(m, s, r, nbr, h, hop)
    W = weights(Fx.shape[1], 8, 6)
    W[4] = np.zeros(8)
    W[5] = np.array(0.0)
    assert np.allclose(apply(W, Fx, sig, np.diag(A)), r / np.diag(A), rtol=1e-14, atol=0)
    y, _ = forward(W, Fx)
    assert np.allclose(y, Fx[:, 0])
