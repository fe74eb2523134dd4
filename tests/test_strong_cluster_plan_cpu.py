"""Host planner of the cluster strong form (Section 6), checked on the CPU: every cell-rule point
belongs to the leaf of its cell's closest DOF (ties: the lower DOF; cells without a DOF vertex to
the group without a far part), and each group lists exactly the edges of the cells touching a DOF
of its leaf's inadmissible partners."""
import numpy as np
import pytest

from oracle import OracleMesh
from oracle.adaptive import cell_rule_points
from paper_1708_03912_gb300 import fraclap as F
from paper_1708_03912_gb300 import synth


@pytest.mark.parametrize("case", ["lshape", "disc"])
def test_strong_form_cluster_plan(case):
    V, T = synth.lshape(0.25, 0) if case == "lshape" else synth.disc(5, 2.0)
    s, eta, leaf, kc = 0.5, 1.0, 8, 3
    h = F.fl_create(V, T)
    try:
        plan = F.fl_strong_form_cluster_plan(h, s, eta, leaf, kc)
        cp = F.fl_cluster_plan(h, s, eta, leaf)
        perm = F.fl_near_region_plan(h, s, 2, eta, leaf)["cell_perm"]
        vod = np.asarray(F.fl_dof_vertices(h, s))
    finally:
        F.fl_destroy(h)
    om = OracleMesh(V, T)
    dov = -np.ones(om.nv, dtype=np.int64)
    dov[vod] = np.arange(len(vod))
    node = cp["node"]
    leaf_of = np.full(len(vod), -1)
    for c in range(len(node)):
        if node[c, 2] < 0:
            leaf_of[cp["perm"][node[c, 0]:node[c, 1]]] = c
    X, _, _ = cell_rule_points(om, kc)
    q = X.shape[1]
    assert len(plan["pgroup"]) == om.nc * q
    free = 0
    for k in range(om.nc):
        K = int(perm[k])
        dofs = [int(dov[v]) for v in om.C[K] if dov[v] >= 0]
        for a in range(q):
            got = plan["gnode"][plan["pgroup"][k * q + a]]
            if not dofs:
                assert got == -1
                free += 1
                continue
            d2 = [float(np.sum((om.V[vod[i]] - X[K, a]) ** 2)) for i in dofs]
            i0 = min(zip(d2, dofs))[1]
            assert got == leaf_of[i0], (K, a)
    assert (free > 0) == (case == "lshape")
    partners = {}
    for a, b in cp["near"]:
        partners.setdefault(int(a), []).append(int(b))
    for g, sigma in enumerate(plan["gnode"]):
        lst = plan["gf_fac"][plan["gf_ptr"][g]:plan["gf_ptr"][g + 1]]
        assert np.all(np.diff(lst) > 0)
        got = {tuple(sorted(plan["fac_vert"][e])) for e in lst}
        if sigma < 0:
            want = {tuple(sorted(e)) for e in plan["fac_vert"]}
        else:
            near_dofs = [int(i) for tau in partners[int(sigma)] for i in cp["perm"][node[tau, 0]:node[tau, 1]]]
            cells = {c for i in near_dofs for c in om.cells_of_vertex[vod[i]]}
            want = set()
            for c in cells:
                a_, b_, c_ = om.C[c]
                for p_, q_ in ((a_, b_), (b_, c_), (c_, a_)):
                    want.add((min(p_, q_), max(p_, q_)))
        assert got == want, (g, sigma)


def test_strong_form_cluster_grouping_with_ties():
    # L-shape level 3 (19,188 cells, 172,692 points): the bisection meshes' right isosceles cells put
    # many rule points at equal (or, after rounding, nearly equal) distance from two DOF vertices;
    # every point's group is still the leaf of the closest DOF with ties to the lower DOF
    V, T = synth.lshape(0.25, 3)
    s, eta, leaf, kc = 0.5, 1.0, 32, 3
    h = F.fl_create(V, T)
    try:
        plan = F.fl_strong_form_cluster_plan(h, s, eta, leaf, kc)
        cp = F.fl_cluster_plan(h, s, eta, leaf)
        perm = F.fl_near_region_plan(h, s, 2, eta, leaf)["cell_perm"]
        vod = np.asarray(F.fl_dof_vertices(h, s))
    finally:
        F.fl_destroy(h)
    om = OracleMesh(V, T)
    dov = -np.ones(om.nv, dtype=np.int64)
    dov[vod] = np.arange(len(vod))
    node = cp["node"]
    leaf_of = np.full(len(vod), -1)
    for c in range(len(node)):
        if node[c, 2] < 0:
            leaf_of[cp["perm"][node[c, 0]:node[c, 1]]] = c
    X, _, _ = cell_rule_points(om, kc)
    q = X.shape[1]
    D = om.V[om.C][:, None, :, :] - X[:, :, None, :]   # [cells, q, 3, 2]
    d2 = D[..., 0] ** 2 + D[..., 1] ** 2
    dof = dov[om.C]
    best_d = np.full((om.nc, q), np.inf)
    best_i = np.full((om.nc, q), len(vod))
    for j in range(3):
        dj = np.where(dof[:, j] >= 0, 1.0, np.inf)[:, None] * d2[:, :, j]
        ij = np.where(dof[:, j] >= 0, dof[:, j], len(vod))[:, None]
        take = (dj < best_d) | ((dj == best_d) & (ij < best_i))
        best_d = np.where(take, dj, best_d)
        best_i = np.where(take, ij, best_i)
    assert np.all(best_i < len(vod))  # every cell of this mesh has a DOF vertex
    second = np.sort(np.where((dof >= 0)[:, None, :], d2, np.inf), axis=2)[:, :, 1]
    ties = np.sum(second == best_d)
    assert ties > 1000  # the tie rule decides many points
    pos = np.empty(om.nc, dtype=np.int64)
    pos[perm] = np.arange(om.nc)
    got = np.asarray(plan["gnode"])[plan["pgroup"].reshape(om.nc, q)[pos]]
    assert np.array_equal(got, leaf_of[best_i])
