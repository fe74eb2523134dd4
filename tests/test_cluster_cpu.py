"""The host planner's cluster tree and block partition (Section 6) equal the oracle's: the
same nodes (DOF sets, in creation order, sons), the same admissible and near-field pairs in
the same order.  Host only; no GPU."""
import numpy as np
import pytest

from oracle import OracleMesh
from oracle.cluster import ClusterTree, block_partition
from paper_1708_03912_gb300 import fraclap as F
from paper_1708_03912_gb300 import synth


@pytest.mark.parametrize("case", ["disc", "graded_disc", "lshape", "interval"])
def test_cluster_plan_matches_oracle(case):
    (V, T), s, leaf, eta = {"disc": (synth.disc(9), 0.5, 8, 1.0),
                            "graded_disc": (synth.disc(8, 2.0), 0.25, 16, 2.0),
                            "lshape": (synth.lshape(0.25, 2), 0.5, 32, 1.0),
                            "interval": (synth.graded_interval(90, 2.0), 0.75, 4, 1.0)}[case]
    om = OracleMesh(V, T)
    tree = ClusterTree(om, s, leaf)
    far, near = block_partition(tree, eta)
    h = F.fl_create(V, T)
    try:
        plan = F.fl_cluster_plan(h, s, eta, leaf)
    finally:
        F.fl_destroy(h)
    node, perm = plan["node"], plan["perm"]
    assert len(node) == len(tree.dofs)
    for c in range(len(node)):
        lo, hi, s0, s1 = node[c]
        assert [x for x in (s0, s1) if x >= 0] == tree.sons[c]
        if tree.sons[c]:  # the DOF set (its order in perm is the sons' order)
            assert np.array_equal(np.sort(perm[lo:hi]), np.sort(tree.dofs[c])), c
        else:  # leaves: the same DOFs in the same order
            assert np.array_equal(perm[lo:hi], tree.dofs[c]), c
    assert [tuple(p) for p in plan["far"]] == far
    assert [tuple(p) for p in plan["near"]] == near


def test_cluster_plan_rejects_bad_parameters():
    V, T = synth.disc(4)
    h = F.fl_create(V, T)
    try:
        with pytest.raises(F.FlError):
            F.fl_cluster_plan(h, 0.5, 1.0, 0)
        with pytest.raises(F.FlError):
            F.fl_cluster_plan(h, 0.5, -1.0, 4)
    finally:
        F.fl_destroy(h)
