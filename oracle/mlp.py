"""Learned patch preconditioner (oracle; test infrastructure only).

No part of this is in the paper.  The preconditioner is linear in the residual, with
coefficients that a small network computes from the mesh geometry around each DOF:

* Patch of DOF i: the K nearest other DOFs among the vertices within two mesh edges
  of vertex i, ordered by (distance, vertex index); missing entries padded with -1.
* h_i: mean length of the mesh edges at vertex i; hop_i: mesh edges from vertex i to
  the nearest boundary vertex, capped at 8.
* Geometry features g_i (2K + 3): ((x_{j_k} - x_i)/h_i, (y_{j_k} - y_i)/h_i) for k < K
  (zeros where padded), log h_i, hop_i/8, s.
* Network: o_i = W3ᵀ tanh(W2ᵀ tanh(W1ᵀ g_i + b1) + b2) + b3 (K + 1 outputs, hidden
  widths H, H); stencil c_i = o_i + (1, 0, ..., 0).
* M r: (M r)_i = (c_i0 r_i + Σ_k c_ik r_{j_k}) / A_ii; the preconditioner applied is the
  symmetric part ½ (M + Mᵀ) r.  With W3 = 0, b3 = 0 it is the Jacobi preconditioner.
* Training samples pair the normalised residual patch of one DOF,
  x_i = (r_i, r_{j_0}, ..., r_{j_{K-1}}) / σ_i (zeros where padded),
  σ_i = sqrt((r_i² + Σ_k r_{j_k}²) / (1 + K_i) + 1e-30), with the target t_i = e_i A_ii / σ_i
  of an error/residual pair (r = A e); prediction y = c_i · x_i; loss mean (y - t)².
  For white-noise errors this is the least-squares (Frobenius) fit of M to A⁻¹ on the
  patch pattern.

Parity status: gradients pinned against central finite differences
(tests/test_oracle_mlp.py); patch table against brute-force distances; the Jacobi
limit and the symmetric apply against their definitions.
"""
from __future__ import annotations

import numpy as np


def patches(mesh, s, K=12):
    """(nbr [n, K] DOF indices or -1, h [n], hop [n]) for the oracle mesh's DOFs at order s."""
    dofs, dov = mesh.dofs(s)
    V = mesh.V
    nv = len(V)
    adj = [set() for _ in range(nv)]
    for c in mesh.C:
        for a in range(3):
            for b in range(3):
                if a != b:
                    adj[c[a]].add(int(c[b]))
    h = np.array([np.mean([np.linalg.norm(V[v] - V[w]) for w in adj[v]]) for v in range(nv)])
    onb = mesh.on_boundary
    hop = np.full(nv, 8, dtype=np.int64)
    frontier = [v for v in range(nv) if onb[v]]
    for v in frontier:
        hop[v] = 0
    d = 0
    while frontier and d < 8:
        d += 1
        nxt = []
        for v in frontier:
            for w in adj[v]:
                if hop[w] > d:
                    hop[w] = d
                    nxt.append(w)
        frontier = nxt
    n = len(dofs)
    nbr = -np.ones((n, K), dtype=np.int64)
    for i, v in enumerate(dofs):
        ring = set(adj[v])
        for w in list(ring):
            ring |= adj[w]
        ring.discard(v)
        cand = [(float(np.linalg.norm(V[w] - V[v])), int(w)) for w in ring if dov[w] >= 0]
        cand.sort()
        for k, (_, w) in enumerate(cand[:K]):
            nbr[i, k] = dov[w]
    return nbr, h[dofs], hop[dofs]


def geometry(mesh, s, nbr, h, hop):
    dofs, _ = mesh.dofs(s)
    X = mesh.V[dofs]
    n, K = nbr.shape
    G = np.zeros((n, 2 * K + 3))
    for i in range(n):
        for k in range(K):
            j = nbr[i, k]
            if j >= 0:
                G[i, 2 * k] = (X[j, 0] - X[i, 0]) / h[i]
                G[i, 2 * k + 1] = (X[j, 1] - X[i, 1]) / h[i]
        G[i, 2 * K] = np.log(h[i])
        G[i, 2 * K + 1] = hop[i] / 8.0
        G[i, 2 * K + 2] = s
    return G


def residual_patch(r, nbr):
    """(x [n, K+1], sigma [n]) of a residual."""
    n, K = nbr.shape
    x = np.zeros((n, K + 1))
    sig = np.zeros(n)
    for i in range(n):
        present = nbr[i][nbr[i] >= 0]
        sig[i] = np.sqrt((r[i] ** 2 + np.sum(r[present] ** 2)) / (1 + len(present)) + 1e-30)
        x[i, 0] = r[i] / sig[i]
        for k in range(K):
            if nbr[i, k] >= 0:
                x[i, 1 + k] = r[nbr[i, k]] / sig[i]
    return x, sig


def coefficients(Wts, G):
    W1, b1, W2, b2, W3, b3 = Wts
    H1 = np.tanh(G @ W1 + b1)
    H2 = np.tanh(H1 @ W2 + b2)
    C = H2 @ W3 + b3
    C[:, 0] += 1.0
    return C, (H1, H2)


def loss_grad(Wts, G, X, t):
    """Loss mean (c(g) · x - t)² and its gradient with respect to (W1, b1, W2, b2, W3, b3)."""
    W1, b1, W2, b2, W3, b3 = Wts
    C, (H1, H2) = coefficients(Wts, G)
    y = np.sum(C * X, axis=1)
    B = G.shape[0]
    dy = 2.0 * (y - t) / B
    dO = dy[:, None] * X
    gW3 = H2.T @ dO
    gb3 = dO.sum(axis=0)
    dA2 = (dO @ W3.T) * (1.0 - H2 ** 2)
    gW2 = H1.T @ dA2
    gb2 = dA2.sum(axis=0)
    dA1 = (dA2 @ W2.T) * (1.0 - H1 ** 2)
    gW1 = G.T @ dA1
    gb1 = dA1.sum(axis=0)
    return float(np.mean((y - t) ** 2)), (gW1, gb1, gW2, gb2, gW3, gb3)


def stencil_matrix(C, nbr, diag):
    """M with M_ii = c_i0 / A_ii, M_{i j_k} = c_ik / A_ii."""
    n, K = nbr.shape
    M = np.zeros((n, n))
    for i in range(n):
        M[i, i] += C[i, 0] / diag[i]
        for k in range(K):
            if nbr[i, k] >= 0:
                M[i, nbr[i, k]] += C[i, 1 + k] / diag[i]
    return M


def apply(Wts, G, nbr, diag, r):
    """½ (M + Mᵀ) r."""
    C, _ = coefficients(Wts, G)
    M = stencil_matrix(C, nbr, diag)
    return 0.5 * (M @ r + M.T @ r)
