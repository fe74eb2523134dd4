"""Mesh bookkeeping for the oracle (test infrastructure only).

Follows Section 3 of the paper: a conforming triangulation P_h of a polygon
(d = 2) or a partition of an interval (d = 1), its boundary facets dP_h, P1
Lagrange basis functions phi_i and the degree-of-freedom set I_h.

Readings (the paper fixes no data layout):
* triangles are re-oriented counter-clockwise, intervals left-to-right;
* a boundary facet is an edge (2D) or vertex (1D) that belongs to exactly one
  cell; its unit normal points into that cell, i.e. into Omega (the paper's
  "inward normal" n_y of the boundary term);
* DOFs: "interior" mode (the default) uses the interior vertices for every s;
  "paper" mode uses all vertices when s < 1/2 and the interior ones otherwise,
  as in Section 3.  Either way DOFs are numbered by increasing vertex index;
* element pairs are classed combinatorially: touching (at least one shared
  vertex; identical / common edge / common vertex), near (no shared vertex, but
  a vertex of one is joined by a mesh edge to a vertex of the other) and far
  (everything else).  Element/facet pairs use the same three classes.
"""
from __future__ import annotations

import numpy as np


class OracleMesh:
    def __init__(self, vertices, cells):
        V = np.asarray(vertices, dtype=np.float64)
        if V.ndim == 1:
            V = V[:, None]
        self.V = V.copy()
        self.dim = V.shape[1]
        if self.dim not in (1, 2):
            raise ValueError("dimension must be 1 or 2")
        C = np.array(cells, dtype=np.int64).copy()
        if C.shape[1] != self.dim + 1:
            raise ValueError("cells must have dim+1 vertices")
        if self.dim == 1:
            swap = V[C[:, 0], 0] > V[C[:, 1], 0]
            C[swap] = C[swap][:, ::-1]
            vol = V[C[:, 1], 0] - V[C[:, 0], 0]
            if np.any(vol <= 0):
                raise ValueError("degenerate interval")
        else:
            P = V[C]
            det = ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
                   - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))
            neg = det < 0
            C[neg] = C[neg][:, [0, 2, 1]]
            vol = np.abs(det) / 2.0
            scale = np.max(np.abs(V)) if len(V) else 1.0
            if np.any(vol <= 1e-14 * scale * scale):
                raise ValueError("degenerate triangle")
        self.C = C
        self.vol = vol
        self.nv = len(V)
        self.nc = len(C)
        self._facets()
        self._adjacency()

    # -- boundary facets and inward normals -------------------------------
    def _facets(self):
        C, V = self.C, self.V
        if self.dim == 1:
            cnt = np.bincount(C.ravel(), minlength=self.nv)
            bverts = np.nonzero(cnt == 1)[0]
            fac, nrm, fcell = [], [], []
            for v in bverts:
                k = int(np.nonzero((C == v).any(axis=1))[0][0])
                fac.append([v])
                fcell.append(k)
                nrm.append([1.0 if C[k, 0] == v else -1.0])
            self.facets = np.array(fac, dtype=np.int64).reshape(-1, 1)
            self.normals = np.array(nrm, dtype=np.float64).reshape(-1, 1)
            self.facet_cell = np.array(fcell, dtype=np.int64)
        else:
            edges = {}
            for k, (a, b, c) in enumerate(C):
                for p, q, r in ((a, b, c), (b, c, a), (c, a, b)):
                    key = (min(p, q), max(p, q))
                    edges.setdefault(key, []).append((k, r))
            fac, nrm, fcell = [], [], []
            for (p, q), owners in sorted(edges.items()):
                if len(owners) == 1:
                    k, r = owners[0]
                    t = V[q] - V[p]
                    n = np.array([-t[1], t[0]]) / np.hypot(t[0], t[1])
                    if np.dot(n, V[r] - V[p]) < 0:
                        n = -n
                    fac.append([p, q])
                    nrm.append(n)
                    fcell.append(k)
                elif len(owners) > 2:
                    raise ValueError("non-manifold edge")
            self.facets = np.array(fac, dtype=np.int64).reshape(-1, 2)
            self.normals = np.array(nrm, dtype=np.float64).reshape(-1, 2)
            self.facet_cell = np.array(fcell, dtype=np.int64)
            # edge (sorted vertex pair) -> [(cell, opposite vertex)], and boundary edge -> facet index
            self.edge_owners = edges
            self.facet_of_edge = {(int(p), int(q)): f for f, (p, q) in enumerate(self.facets)}
        self.on_boundary = np.zeros(self.nv, dtype=bool)
        self.on_boundary[self.facets.ravel()] = True
        self.facet_len = (np.ones(len(self.facets)) if self.dim == 1 else
                          np.linalg.norm(V[self.facets[:, 1]] - V[self.facets[:, 0]], axis=1))

    # -- vertex adjacency through mesh edges -------------------------------
    def _adjacency(self):
        nbr = [set() for _ in range(self.nv)]
        for cell in self.C:
            for a in cell:
                for b in cell:
                    if a != b:
                        nbr[a].add(int(b))
        self.vertex_nbrs = [np.array(sorted(s), dtype=np.int64) for s in nbr]
        self.cells_of_vertex = [[] for _ in range(self.nv)]
        for k, cell in enumerate(self.C):
            for a in cell:
                self.cells_of_vertex[a].append(k)

    # -- degrees of freedom ---------------------------------------------------
    def dofs(self, s: float, mode: str = "interior"):
        """Return (vertex_of_dof, dof_of_vertex) for fractional order s (Section 3)."""
        if mode not in ("interior", "paper"):
            raise ValueError(mode)
        if mode == "paper" and s < 0.5:
            vod = np.arange(self.nv, dtype=np.int64)
        else:
            vod = np.nonzero(~self.on_boundary)[0].astype(np.int64)
        dov = -np.ones(self.nv, dtype=np.int64)
        dov[vod] = np.arange(len(vod))
        return vod, dov

    # -- pair classes -------------------------------------------------------------
    def rings(self, k: int):
        """Boolean vertex masks: vertices of cell k, and those plus their mesh-edge neighbours."""
        m0 = np.zeros(self.nv, dtype=bool)
        m0[self.C[k]] = True
        m1 = m0.copy()
        for a in self.C[k]:
            m1[self.vertex_nbrs[a]] = True
        return m0, m1

    def classify_cells(self, k: int):
        """For all cells: number of vertices shared with cell k, and the near flag."""
        m0, m1 = self.rings(k)
        shared = m0[self.C].sum(axis=1)
        near = (shared == 0) & m1[self.C].any(axis=1)
        return shared, near

    def classify_facets(self, k: int):
        m0, m1 = self.rings(k)
        shared = m0[self.facets].sum(axis=1)
        near = (shared == 0) & m1[self.facets].any(axis=1)
        return shared, near
