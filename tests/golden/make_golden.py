"""Writes the stored expected values under tests/golden/ (calls only oracle/).

interval16_exact.json : exact stiffness matrix of the 15 interior hats of the
    uniform 16-element mesh of (-1,1), from the closed form
    a(u,v) = c ∬ |x-y|^{3-2s} u'' v'' (Section 2 Fourier form; 1D, s != 1/2),
    evaluated with 40-digit arithmetic.
square4_exact.json : exact matrix of the interior hats of the jittered 4x4
    square mesh (paper_1708_03912_gb300.synth.square(4, 0.2)), from the
    edge-pair form a(u,v) = c ∬ |x-y|^{2-2s} dΔu dΔv (2D).
strong_form_cluster_lshape5.json : the oracle's strong form by the cluster
    method (Section 6 with Lemma 4.1; oracle.cluster.strong_form_cluster) at
    the cell-rule points of seeded cells of the L-shape level 5 (73,432 cells,
    s = 1/2, m = 4, eta = 1, leaves of 32), for the smooth nodal function
    u = cos(1.3 x) (1 - 0.4 y^2) + 0.2 x y; with each point's closest DOF, the
    relative gap to the second closest, and the size of the direct form's
    terms.  A stored copy because the oracle needs minutes at this size.

Run:  python tests/golden/make_golden.py [name ...]   (default: all)
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import OracleMesh, exact  # noqa: E402
from paper_1708_03912_gb300 import synth  # noqa: E402

HSF = {"level": 5, "s": 0.5, "m": 4, "eta": 1.0, "leaf": 32, "k_cell": 3, "k_edge": 4, "k_near": 16,
       "seed": 20, "cells": 6}


def mesh_hash(V, T):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(V, dtype="<f8").tobytes())
    h.update(np.ascontiguousarray(T, dtype="<i8").tobytes())
    return h.hexdigest()


def smooth_u(X):
    """The nodal function of the strong-form values: u = cos(1.3 x) (1 - 0.4 y^2) + 0.2 x y."""
    return np.cos(1.3 * X[:, 0]) * (1.0 - 0.4 * X[:, 1] ** 2) + 0.2 * X[:, 0] * X[:, 1]


def strong_form_cluster_cells(V, T, p=HSF):
    """The oracle's cluster strong form at the points of p["cells"] seeded cells, the cell at the
    re-entrant corner (1, 1) and the cell at the convex corner (2, 0)."""
    from oracle import adaptive as oad
    from oracle.adaptive import cell_rule_points
    from oracle.cluster import strong_form_cluster

    om = OracleMesh(V, T)
    s = p["s"]
    vod, dov = om.dofs(s)
    u = smooth_u(om.V[vod])
    cen = om.V[om.C].mean(axis=1)
    cells = list(np.random.default_rng(p["seed"]).choice(om.nc, p["cells"], replace=False))
    for corner in ((1.0, 1.0), (2.0, 0.0)):
        cells.append(int(np.argmin(np.sum((cen - np.array(corner)) ** 2, axis=1))))
    cells = np.array(sorted(set(int(c) for c in cells)), dtype=np.int64)
    opts = dict(k_cell=p["k_cell"], k_edge=p["k_edge"], k_near=p["k_near"])
    S = strong_form_cluster(om, s, u, m=p["m"], eta=p["eta"], leaf=p["leaf"], cells=cells, **opts)
    _, size = oad.strong_form(om, s, u, cells=cells, with_abs=True, **opts)
    X, _, _ = cell_rule_points(om, p["k_cell"])
    closest, gap = [], []
    for k in cells:
        dofs = [int(dov[v]) for v in om.C[k] if dov[v] >= 0]
        ck, gk = [], []
        for x0 in X[k]:
            d2 = sorted((float(np.sum((om.V[vod[i]] - x0) ** 2)), i) for i in dofs)
            ck.append(d2[0][1])
            gk.append((d2[1][0] - d2[0][0]) / d2[0][0] if len(d2) > 1 else float("inf"))
        closest.append(ck)
        gap.append(gk)
    return {"cells": cells.tolist(), "values": S.tolist(), "size": size.tolist(), "closest_dof": closest,
            "gap": gap, "vod_hash": hashlib.sha256(np.ascontiguousarray(vod, dtype="<i8").tobytes()).hexdigest()}


def write_strong_form_cluster():
    p = HSF
    V, T = synth.lshape(0.25, p["level"])
    out = {"citation": "Section 6 (cluster method: near part by Lemma 4.1, far part by Chebyshev "
                       "interpolation of the kernel); oracle.cluster.strong_form_cluster",
           "mesh": f"synth.lshape(0.25, {p['level']})", "mesh_hash": mesh_hash(V, T), "params": p,
           "u": "cos(1.3 x) (1 - 0.4 y^2) + 0.2 x y at the DOF vertices"}
    out.update(strong_form_cluster_cells(V, T, p))
    with open(os.path.join(HERE, "strong_form_cluster_lshape5.json"), "w") as f:
        json.dump(out, f, indent=0)


def write_exact():
    V, T = synth.interval(16)
    out = {"citation": "Section 2 (Fourier form of a(u,v)); 1D closed form through phi''",
           "mesh": "synth.interval(16)", "matrices": {}}
    for s in (0.25, 0.75):
        out["matrices"][str(s)] = exact.exact_matrix_1d(V[:, 0], s).tolist()
    with open(os.path.join(HERE, "interval16_exact.json"), "w") as f:
        json.dump(out, f, indent=0)
    V, T = synth.square(4, 0.2)
    m = OracleMesh(V, T)
    out = {"citation": "Section 2 (Fourier form of a(u,v)); 2D edge-pair form through Δphi",
           "mesh": "synth.square(4, 0.2)", "matrices": {}}
    for s in (0.25, 0.5, 0.75):
        out["matrices"][str(s)] = exact.exact_matrix_2d(m, s).tolist()
    with open(os.path.join(HERE, "square4_exact.json"), "w") as f:
        json.dump(out, f, indent=0)


WRITERS = {"exact": write_exact, "strong_form_cluster": write_strong_form_cluster}


def main(names=None):
    for name in names or sorted(WRITERS):
        WRITERS[name]()


if __name__ == "__main__":
    main(sys.argv[1:])
