"""Learned patch preconditioner (oracle; test infrastructure only).

No part of this is in the paper: the preconditioner M(r) maps the residual r of a
conjugate-gradient iterate to an estimate of its error e = A⁻¹ r, one DOF at a time,
from the residual on a small patch of nearby DOFs.  Definitions (the GPU path states
the same ones):

* Patch of DOF i: the K nearest other DOFs among the vertices within two mesh edges
  of vertex i, ordered by (distance, vertex index); missing entries padded with -1.
* h_i: mean length of the mesh edges at vertex i; hop_i: number of mesh edges from
  vertex i to the nearest boundary vertex, capped at 8.
* Features x_i (length 1 + 3K + 3):
  σ_i = sqrt((r_i² + Σ_k r_{j_k}²) / (1 + K_i) + 1e-30) over the K_i present neighbours,
  x = [r_i/σ_i, (r_{j_k}/σ_i, (x_{j_k} - x_i)/h_i, (y_{j_k} - y_i)/h_i) for k < K
  (zeros where padded), log(h_i), hop_i/8, s].
* Network: y = x_0 + w3·tanh(W2ᵀ tanh(W1ᵀ x + b1) + b2) + b3 (hidden widths H, H);
  M(r)_i = σ_i y_i / A_ii.  With w3 = b3 = 0 this is the Jacobi preconditioner.
* Training loss on samples (x_n, t_n) with t_n = e_i A_ii / σ_i:  mean_n (y_n - t_n)².

Parity status: the gradients are pinned against central finite differences of the
loss (tests/test_oracle_mlp.py); the patch table against brute-force distances; the
features against their definition on a hand-checked mesh.
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
    # h: mean incident edge length
    h = np.array([np.mean([np.linalg.norm(V[v] - V[w]) for w in adj[v]]) for v in range(nv)])
    # hops to the boundary (breadth-first from the boundary vertices)
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


def features(mesh, s, r, nbr, h, hop):
    dofs, _ = mesh.dofs(s)
    X = mesh.V[dofs]
    n, K = nbr.shape
    F = np.zeros((n, 1 + 3 * K + 3))
    sig = np.zeros(n)
    for i in range(n):
        present = nbr[i][nbr[i] >= 0]
        ss = r[i] ** 2 + np.sum(r[present] ** 2)
        sig[i] = np.sqrt(ss / (1 + len(present)) + 1e-30)
        F[i, 0] = r[i] / sig[i]
        for k in range(K):
            j = nbr[i, k]
            if j < 0:
                continue
            F[i, 1 + 3 * k] = r[j] / sig[i]
            F[i, 2 + 3 * k] = (X[j, 0] - X[i, 0]) / h[i]
            F[i, 3 + 3 * k] = (X[j, 1] - X[i, 1]) / h[i]
        F[i, 1 + 3 * K] = np.log(h[i])
        F[i, 2 + 3 * K] = hop[i] / 8.0
        F[i, 3 + 3 * K] = s
    return F, sig


def forward(Wts, X):
    W1, b1, W2, b2, w3, b3 = Wts
    H1 = np.tanh(X @ W1 + b1)
    H2 = np.tanh(H1 @ W2 + b2)
    return X[:, 0] + H2 @ w3 + b3, (H1, H2)


def loss_grad(Wts, X, t):
    """Loss mean (y - t)² and its gradient with respect to (W1, b1, W2, b2, w3, b3)."""
    W1, b1, W2, b2, w3, b3 = Wts
    y, (H1, H2) = forward(Wts, X)
    B = X.shape[0]
    dy = 2.0 * (y - t) / B
    gw3 = H2.T @ dy
    gb3 = np.sum(dy)
    dA2 = np.outer(dy, w3) * (1.0 - H2 ** 2)
    gW2 = H1.T @ dA2
    gb2 = dA2.sum(axis=0)
    dA1 = (dA2 @ W2.T) * (1.0 - H1 ** 2)
    gW1 = X.T @ dA1
    gb1 = dA1.sum(axis=0)
    return float(np.mean((y - t) ** 2)), (gW1, gb1, gW2, gb2, gw3, np.array(gb3))


def apply(Wts, F, sig, diag):
    y, _ = forward(Wts, F)
    return sig * y / diag
