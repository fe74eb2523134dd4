"""Host planner of the direct near-field assembly (Section 6), checked on the CPU against the
oracle: for every cell with DOFs, the facets of the boundary of N(K) (K, its touching cells
and those at vertex-graph distance 1), their normals pointing into N(K) and their classes."""
import numpy as np
import pytest

from oracle import OracleMesh
from oracle.assemble import near_region_facets
from paper_1708_03912_gb300 import fraclap as F
from paper_1708_03912_gb300 import synth


def _oracle_sets(om, k):
    Y0, Y1, n, flen, verts, bidx = near_region_facets(om, k)
    m0, m1 = om.rings(k)
    sh = m0[verts].sum(axis=1)
    near = (sh == 0) & m1[verts].any(axis=1)
    cls = np.where(sh > 0, np.where((om.dim == 1) | (sh == 2), 2, 3), np.where(near, 1, 0))
    return {(tuple(sorted(int(v) for v in verts[q])), int(cls[q])): n[q] for q in range(len(verts))}


@pytest.mark.parametrize("case", ["lshape", "disc", "interval"])
def test_near_region_facets_match_oracle(case):
    V, T = {"lshape": synth.lshape(0.25, 0), "disc": synth.disc(5, 2.0),
            "interval": synth.graded_interval(40, 2.0)}[case]
    dim = 1 if np.asarray(V).ndim == 1 or np.asarray(V).shape[1] == 1 else 2
    s = 0.5
    h = F.fl_create(V, T)
    try:
        plan = F.fl_near_region_plan(h, s, dim, eta=1.0, leaf=8)
    finally:
        F.fl_destroy(h)
    om = OracleMesh(V, T)
    _, dov = om.dofs(s)
    has_dof = (dov[om.C] >= 0).any(axis=1)
    checked = 0
    for k in range(len(plan["cell_perm"])):
        K = int(plan["cell_perm"][k])
        lo, hi = plan["ef_ptr"][k], plan["ef_ptr"][k + 1]
        if not has_dof[K]:
            assert hi == lo
            continue
        got = {}
        for q in range(lo, hi):
            f = plan["ef_fac"][q]
            key = (tuple(sorted(int(v) for v in plan["fac_vert"][f])), int(plan["ef_cls"][q]))
            assert key not in got
            got[key] = plan["fac_normal"][f]
        want = _oracle_sets(om, K)
        assert set(got) == set(want), (K, set(got) ^ set(want))
        for key in want:
            assert np.allclose(got[key], want[key], rtol=0, atol=1e-14)
        assert np.all(np.diff(plan["ef_fac"][lo:hi]) > 0)  # ascending facet ids
        checked += 1
    assert checked == int(has_dof.sum())
    assert plan["tiles"] > 0


def _blocks_and_leaves(h, s, eta, leaf, V, T):
    perm = F.fl_near_region_plan(h, s, 1 if np.asarray(V).ndim == 1 or np.asarray(V).shape[1] == 1 else 2,
                                 eta=eta, leaf=leaf)["cell_perm"]
    cp = F.fl_cluster_plan(h, s, eta, leaf)
    vod = np.asarray(F.fl_dof_vertices(h, s))
    return perm, cp, vod


@pytest.mark.parametrize("case", ["lshape", "disc", "interval"])
def test_near_region_tiles(case):
    # the tiles of the direct near field and their row masks against a plain restatement of their
    # definition, and the property the assembly needs: every separated pair of a cell of supp phi_i
    # and a cell of supp phi_j, (i, j) a near-field entry, lies in a listed tile whose row bit for its
    # cell in the lower block (the lower cell within one block) is set
    V, T = {"lshape": synth.lshape(0.25, 1), "disc": synth.disc(8, 2.0),
            "interval": synth.graded_interval(300, 2.0)}[case]
    s, eta, leaf = 0.5, 1.0, 8
    h = F.fl_create(V, T)
    try:
        tiles, rowmask = F.fl_near_region_tiles(h, s, eta, leaf)
        perm, cp, vod = _blocks_and_leaves(h, s, eta, leaf, V, T)
    finally:
        F.fl_destroy(h)
    om = OracleMesh(V, T)
    nc = om.nc
    dov = -np.ones(om.nv, dtype=np.int64)
    dov[vod] = np.arange(len(vod))
    pos = np.empty(nc, dtype=np.int64)
    pos[perm] = np.arange(nc)               # original cell -> internal position
    node = cp["node"]
    leaf_of = np.full(len(vod), -1)
    for c in range(len(node)):
        if node[c, 2] < 0:
            leaf_of[cp["perm"][node[c, 0]:node[c, 1]]] = c
    near = {(int(a), int(b)) for a, b in cp["near"]}
    # per internal cell, the leaves of its DOFs; per block, the leaves of its cells' DOFs
    cell_leaves = [set() for _ in range(nc)]
    for K in range(nc):
        for v in om.C[K]:
            if dov[v] >= 0:
                cell_leaves[pos[K]].add(int(leaf_of[dov[v]]))
    nblk = (nc + 31) // 32
    blk_leaves = [set() for _ in range(nblk)]
    for k in range(nc):
        blk_leaves[k // 32] |= cell_leaves[k]
    want = {}
    for I in range(nblk):
        for J in range(I, nblk):
            if any((a, b) in near or (b, a) in near for a in blk_leaves[I] for b in blk_leaves[J]):
                mask = 0
                for kk in range(32):
                    k = 32 * I + kk
                    if k < nc and any((a, b) in near for a in cell_leaves[k] for b in blk_leaves[J]):
                        mask |= 1 << kk
                want[(I, J)] = mask
    got = {(int(I), int(J)): int(mk) for (I, J), mk in zip(tiles, rowmask)}
    assert list(got) == sorted(got)          # ordered by (I, J)
    assert got == want
    assert len(got) < nblk * (nblk + 1) // 2  # a proper subset of the dense tiles
    assert any(mk != 0xFFFFFFFF for mk in got.values())  # and some rows skipped
    # coverage from the mesh: every separated pair feeding a near-field entry
    checked = 0
    for a, b in near:
        da = cp["perm"][node[a, 0]:node[a, 1]]
        db = cp["perm"][node[b, 0]:node[b, 1]]
        ca = {int(K) for i in da for K in om.cells_of_vertex[vod[i]]}
        cb = {int(K) for j in db for K in om.cells_of_vertex[vod[j]]}
        for K in ca:
            far = _far_partners(om, K)
            for M in cb & far:
                lo, hi = sorted((int(pos[K]), int(pos[M])))
                key = (lo // 32, hi // 32)
                assert key in got, (K, M)
                assert (got[key] >> (lo % 32)) & 1, (K, M)
                checked += 1
    assert checked > 0


_FAR_CACHE = {}


def _far_partners(om, K):
    """Cells at vertex-graph distance >= 2 from cell K (no shared vertex and no mesh edge between
    their vertices)."""
    key = (id(om), K)
    if key not in _FAR_CACHE:
        shared, near = om.classify_cells(K)
        _FAR_CACHE[key] = set(np.nonzero((shared == 0) & ~near)[0].tolist()) - {K}
    return _FAR_CACHE[key]


def test_near_region_plans_reject_bad_arguments():
    V, T = synth.disc(4)
    h = F.fl_create(V, T)
    try:
        for call in (lambda: F.fl_near_region_tiles(h, 0.5, 1.0, 0),       # leaf < 1
                     lambda: F.fl_near_region_tiles(h, 0.5, -1.0, 8),      # eta < 0
                     lambda: F.fl_near_region_plan(h, 0.5, 2, 1.0, 0),
                     lambda: F.fl_strong_form_cluster_plan(h, 0.5, 1.0, 8, 0)):  # k_cell < 1
            with pytest.raises(F.FlError) as e:
                call()
            assert e.value.code == F.FL_EINVAL
    finally:
        F.fl_destroy(h)
    # a sector handle (symmetry reduction) has no cluster plans
    Vs, Ts = synth.sector(8, 3)
    hs = F.fl_create_sector(Vs, Ts, 8)
    try:
        for call in (lambda: F.fl_near_region_tiles(hs, 0.5, 1.0, 8),
                     lambda: F.fl_near_region_plan(hs, 0.5, 2, 1.0, 8)):
            with pytest.raises(F.FlError):
                call()
    finally:
        F.fl_destroy(hs)
