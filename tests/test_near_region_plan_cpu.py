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
