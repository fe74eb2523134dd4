"""Seeded synthetic inputs: meshes and right-hand sides.

This module holds no arithmetic of the finite element method itself; it only
produces vertex coordinates, cell connectivity and nodal data.  Both the CPU
oracle and the GPU path take their inputs from here, so it must stay free of
any assembly, quadrature or solver code.

Mesh shapes follow the paper's numerical examples (Section 7): the interval
(-1, 1), the unit disc (quasi-uniform, or graded towards the boundary with
radii r_i = 1 - (1 - i/M)^mu as in Section 3), and the L-shaped domain
[0,2]^2 minus [1,2]^2 refined towards the re-entrant corner and the boundary.
The paper's adaptively refined meshes are not available, so these stand in
for them.  The sector mesh serves the symmetry-reduced problem (Section 7).
"""
from __future__ import annotations

import math

import numpy as np

SEED = 20170813


def interval(n_el: int, a: float = -1.0, b: float = 1.0):
    """Uniform mesh of (a, b) with n_el elements: z_k = a + (b - a) k / n_el."""
    k = np.arange(n_el + 1, dtype=np.float64)
    z = a + (b - a) * k / n_el
    cells = np.stack([np.arange(n_el), np.arange(1, n_el + 1)], axis=1)
    return z[:, None].copy(), cells.astype(np.int32)


def graded_interval(n_el: int, mu: float = 2.0):
    """Mesh of (-1, 1) graded symmetrically towards both ends: z = sign(t)(1-(1-|t|)^mu)."""
    t = np.linspace(-1.0, 1.0, n_el + 1)
    z = np.sign(t) * (1.0 - (1.0 - np.abs(t)) ** mu)
    z[0], z[-1] = -1.0, 1.0
    cells = np.stack([np.arange(n_el), np.arange(1, n_el + 1)], axis=1)
    return z[:, None].copy(), cells.astype(np.int32)


def _zipper(inner, inner_ang, outer, outer_ang, pts):
    """Triangulate the annulus between two closed rings, walking both rings and
    closing each step with the shorter of the two candidate diagonals."""
    na, nb = len(inner), len(outer)
    tris = []
    i = j = 0

    def d2(p, q):
        return (pts[p][0] - pts[q][0]) ** 2 + (pts[p][1] - pts[q][1]) ** 2

    while i < na or j < nb:
        if j == nb:
            adv_inner = True
        elif i == na:
            adv_inner = False
        else:
            adv_inner = d2(inner[(i + 1) % na], outer[j % nb]) < d2(inner[i % na], outer[(j + 1) % nb])
        if adv_inner:
            tris.append((inner[i % na], outer[j % nb], inner[(i + 1) % na]))
            i += 1
        else:
            tris.append((inner[i % na], outer[j % nb], outer[(j + 1) % nb]))
            j += 1
    return tris


def disc(M: int, mu: float = 1.0):
    """Unit-disc mesh of M concentric rings with radii r_i = 1 - (1 - i/M)^mu.

    Ring i carries round(2*pi*r_i/h_i) equally spaced points (h_i = r_i - r_{i-1}),
    odd rings shifted by half a step; consecutive rings are joined by a walk that
    closes each step with the shorter diagonal, the first ring by a fan around the
    centre.  mu = 1 gives the
    quasi-uniform disc, mu = 2 the boundary-graded disc.  All boundary vertices lie
    on the unit circle, so the polygon is inscribed in the disc.
    """
    r = [1.0 - (1.0 - i / M) ** mu for i in range(M + 1)]
    pts = [(0.0, 0.0)]
    rings = []
    for i in range(1, M + 1):
        h = r[i] - r[i - 1]
        n = max(6, int(round(2 * math.pi * r[i] / h)))
        off = math.pi / n if i % 2 == 1 else 0.0
        ang = [off + 2 * math.pi * k / n for k in range(n)]
        idx = list(range(len(pts), len(pts) + n))
        pts.extend((r[i] * math.cos(t), r[i] * math.sin(t)) for t in ang)
        rings.append((idx, ang))
    tris = []
    idx0, _ = rings[0]
    for k in range(len(idx0)):
        tris.append((0, idx0[k], idx0[(k + 1) % len(idx0)]))
    for (ia, aa), (ib, ab) in zip(rings[:-1], rings[1:]):
        tris.extend(_zipper(ia, aa, ib, ab, pts))
    return np.array(pts, dtype=np.float64), np.array(tris, dtype=np.int32)


def _zipper_open(inner, outer, pts):
    """Triangulate the strip between two open polylines (first and last points on the two
    cut rays), closing each step with the shorter diagonal."""
    na, nb = len(inner) - 1, len(outer) - 1
    tris = []
    i = j = 0

    def d2(p, q):
        return (pts[p][0] - pts[q][0]) ** 2 + (pts[p][1] - pts[q][1]) ** 2

    while i < na or j < nb:
        if j == nb:
            adv_inner = True
        elif i == na:
            adv_inner = False
        else:
            adv_inner = d2(inner[i + 1], outer[j]) < d2(inner[i], outer[j + 1])
        if adv_inner:
            tris.append((inner[i], outer[j], inner[i + 1]))
            i += 1
        else:
            tris.append((inner[i], outer[j], outer[j + 1]))
            j += 1
    return tris


def sector(K: int, M: int):
    """Uniform mesh of the circular sector {r <= 1, 0 <= phi <= 2 pi / K} (Section 7's
    periodic example with K = 8): M rings at radii j/M, ring j carrying
    max(1, round(2 pi j / K)) + 1 equally spaced points from phi = 0 to phi = 2 pi / K, so the
    vertices on the two cut rays sit at the same radii (the rotation by 2 pi / K maps one ray's
    vertices onto the other's).  Rings are joined by the shorter-diagonal walk, the first by a
    fan around the centre."""
    pts = [(0.0, 0.0)]
    rings = [[0]]
    for j in range(1, M + 1):
        r = j / M
        n = max(1, int(round(2 * math.pi * j / K)))
        idx = list(range(len(pts), len(pts) + n + 1))
        pts.extend((r * math.cos(2 * math.pi * t / (K * n)), r * math.sin(2 * math.pi * t / (K * n)))
                   for t in range(n + 1))
        rings.append(idx)
    tris = [(0, rings[1][t], rings[1][t + 1]) for t in range(len(rings[1]) - 1)]
    for a, b in zip(rings[1:-1], rings[2:]):
        tris.extend(_zipper_open(a, b, pts))
    return np.array(pts, dtype=np.float64), np.array(tris, dtype=np.int32)


def rotated_copies(V, T, K: int):
    """The K copies of a sector mesh rotated by 2 pi l / K about the origin, coincident
    vertices (the cut rays, the centre) merged: the whole mesh the sector stands for."""
    V = np.asarray(V, dtype=np.float64)
    pts, idx = [], {}
    cells = []
    for l in range(K):
        c, s_ = math.cos(2 * math.pi * l / K), math.sin(2 * math.pi * l / K)
        vid = []
        for x, y in V:
            p = (c * x - s_ * y, s_ * x + c * y)
            key = (round(p[0], 9), round(p[1], 9))
            if key not in idx:
                idx[key] = len(pts)
                pts.append(p)
            vid.append(idx[key])
        cells.extend([vid[a], vid[b], vid[d]] for a, b, d in np.asarray(T))
    return np.array(pts, dtype=np.float64), np.array(cells, dtype=np.int32)


def square(m: int, jitter: float = 0.0, seed: int = SEED, lo: float = -1.0, hi: float = 1.0):
    """Structured triangulation of [lo,hi]^2 with m x m cells, interior vertices jittered.

    Each cell is split along alternating diagonals; interior vertices move by up to
    jitter * h in each coordinate (uniform, seeded).
    """
    g = np.linspace(lo, hi, m + 1)
    X, Y = np.meshgrid(g, g, indexing="ij")
    V = np.stack([X.ravel(), Y.ravel()], axis=1)
    h = (hi - lo) / m
    if jitter > 0:
        rng = np.random.default_rng(seed)
        inner = np.array([(i > 0 and i < m and j > 0 and j < m) for i in range(m + 1) for j in range(m + 1)])
        V[inner] += rng.uniform(-jitter * h, jitter * h, size=(inner.sum(), 2))
    vid = lambda i, j: i * (m + 1) + j  # noqa: E731
    tris = []
    for i in range(m):
        for j in range(m):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            if (i + j) % 2 == 0:
                tris += [(a, b, c), (a, c, d)]
            else:
                tris += [(a, b, d), (b, c, d)]
    return V, np.array(tris, dtype=np.int32)


def _nvb_refine(V, T, marked):
    """Newest-vertex bisection with conforming closure (no hanging nodes).

    T[k] = (v0, v1, v2) with the refinement edge (v1, v2) opposite the newest
    vertex v0.  A marked triangle is bisected at the midpoint of its refinement
    edge; neighbours whose refinement edge is not that edge are bisected first
    (recursively), so the result stays conforming.
    """
    V = [tuple(p) for p in V]
    T = [tuple(t) for t in T]
    mid = {}

    def midpoint(a, b):
        key = (min(a, b), max(a, b))
        if key not in mid:
            V.append(((V[a][0] + V[b][0]) / 2, (V[a][1] + V[b][1]) / 2))
            mid[key] = len(V) - 1
        return mid[key]

    edge_owner = {}

    def rebuild():
        edge_owner.clear()
        for k, t in enumerate(T):
            if t is None:
                continue
            for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
                edge_owner.setdefault((min(a, b), max(a, b)), []).append(k)

    rebuild()
    alive = [True] * len(T)

    def bisect(k):
        v0, v1, v2 = T[k]
        key = (min(v1, v2), max(v1, v2))
        nbrs = [j for j in edge_owner.get(key, []) if j != k and alive[j]]
        if nbrs:
            j = nbrs[0]
            w0, w1, w2 = T[j]
            if (min(w1, w2), max(w1, w2)) != key:
                bisect(j)
                # after bisecting j, the neighbour across key is one of its children
                nb = [x for x in edge_owner.get(key, []) if x != k and alive[x]]
                j = nb[0]
            m_ = midpoint(v1, v2)
            _split(k, m_)
            _split(j, m_)
        else:
            m_ = midpoint(v1, v2)
            _split(k, m_)

    def _split(k, m_):
        v0, v1, v2 = T[k]
        alive[k] = False
        for a, b in ((v0, v1), (v1, v2), (v2, v0)):
            lst = edge_owner.get((min(a, b), max(a, b)), [])
            if k in lst:
                lst.remove(k)
        for child in ((m_, v0, v1), (m_, v2, v0)):
            T.append(child)
            alive.append(True)
            c = len(T) - 1
            for a, b in ((child[0], child[1]), (child[1], child[2]), (child[2], child[0])):
                edge_owner.setdefault((min(a, b), max(a, b)), []).append(c)

    for k in marked:
        if alive[k]:
            bisect(k)
    T2 = [t for t, al in zip(T, alive) if al]
    return np.array(V, dtype=np.float64), np.array(T2, dtype=np.int64)


def bisect_all(V, T, rounds: int = 1):
    """Nested refinement: every triangle bisected by newest-vertex bisection, `rounds` times
    (two rounds halve the mesh size)."""
    V = np.asarray(V, dtype=np.float64)
    T = np.asarray(T)
    for _ in range(rounds):
        V, T = _nvb_refine(V, T, list(range(len(T))))
        V = np.asarray(V, dtype=np.float64)
        T = np.asarray(T)
    return V, T.astype(np.int32)


def lshape(h0: float = 0.25, levels: int = 0):
    """L-shaped domain [0,2]^2 minus [1,2]^2 (Section 7.3), refined towards the
    re-entrant corner (1,1) and the boundary by newest-vertex bisection.

    Level 0 is a uniform mesh of 96 triangles.  At level l every triangle with
    diameter above max(h_l/8, h_l * min(1, (dist(x_K, boundary)/0.5)^(1/2),
    (|x_K - (1,1)|/0.5)^(2/3))) is bisected (h_l = h0 / 2^(l/2), repeated until no
    triangle is marked), which yields a nested, conforming sequence whose number of
    vertices roughly doubles per level.
    """
    n = 4
    pts = {}
    V = []
    for i in range(2 * n + 1):
        for j in range(2 * n + 1):
            x, y = i / n, j / n
            if x > 1 and y > 1:
                continue
            pts[(i, j)] = len(V)
            V.append((x, y))
    T = []
    for i in range(2 * n):
        for j in range(2 * n):
            if i >= n and j >= n:
                continue
            a, b, c, d = pts[(i, j)], pts[(i + 1, j)], pts[(i + 1, j + 1)], pts[(i, j + 1)]
            # newest vertex first: refinement edge is the diagonal
            T += [(b, c, a), (d, a, c)]
    V = np.array(V, dtype=np.float64)
    T = np.array(T, dtype=np.int64)
    for lev in range(levels):
        h_l = h0 / 2 ** ((lev + 1) / 2)
        while True:
            P = V[T]
            cen = P.mean(axis=1)
            diam = np.max(np.stack([np.linalg.norm(P[:, 0] - P[:, 1], axis=1),
                                    np.linalg.norm(P[:, 1] - P[:, 2], axis=1),
                                    np.linalg.norm(P[:, 2] - P[:, 0], axis=1)]), axis=0)
            dist_b = np.minimum.reduce([cen[:, 0], cen[:, 1], 2 - cen[:, 0], 2 - cen[:, 1],
                                        np.where((cen[:, 0] > 1) | (cen[:, 1] > 1),
                                                 np.minimum(np.abs(cen[:, 0] - 1), np.abs(cen[:, 1] - 1)), 9.0)])
            dist_c = np.hypot(cen[:, 0] - 1, cen[:, 1] - 1)
            target = h_l * np.minimum.reduce([np.ones(len(T)), np.sqrt(np.maximum(dist_b, 1e-12) / 0.5),
                                               (np.maximum(dist_c, 1e-12) / 0.5) ** (2.0 / 3.0)])
            marked = np.nonzero(diam > np.maximum(target, h_l / 8))[0]
            if len(marked) == 0:
                break
            V, T = _nvb_refine(V, T, marked.tolist())
    return V, T.astype(np.int32)


def gaussian_nodal(n_vertices: int, nrhs: int, seed: int = SEED):
    """Nodal right-hand-side values f_i ~ N(0,1), column r seeded with seed + r."""
    out = np.empty((n_vertices, nrhs), dtype=np.float64)
    for r in range(nrhs):
        out[:, r] = np.random.default_rng(seed + r).standard_normal(n_vertices)
    return out


def random_rows(n: int, count: int, seed: int = SEED):
    """Seeded sample of distinct row indices in [0, n), sorted."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(count, n), replace=False))
