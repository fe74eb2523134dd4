"""GPU parity of the strong form by the cluster method (Section 6) against the oracle's
restatement (oracle.cluster.strong_form_cluster: near partners by Lemma 4.1, admissible ones by
Chebyshev interpolation at the point), and against the direct evaluation as the order grows."""
import hashlib
import importlib.util
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import OracleMesh  # noqa: E402
from oracle import adaptive as oad  # noqa: E402
from oracle.cluster import strong_form_cluster  # noqa: E402
from paper_1708_03912_gb300 import fraclap as F  # noqa: E402
from paper_1708_03912_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

# the near part is Lemma 4.1's sum (double-word far facets, float64 near ones: 2^-40 of the sum
# of the terms' absolute values, as for the direct form); the far part is a float64 sum of m^4
# products per point on both sides
TOL = 2.0 ** -40


def _u(mesh_or_n, s):
    om = mesh_or_n
    vod, _ = om.dofs(s)
    X = om.V[vod]
    return np.cos(1.3 * X[:, 0]) * (1.0 - 0.4 * X[:, 1] ** 2) + 0.2 * X[:, 0] * X[:, 1]


@pytest.mark.parametrize("s,case", [(0.25, "disc"), (0.75, "disc"), (0.5, "lshape")])
def test_cluster_strong_form_matches_oracle(s, case):
    # the L-shape's 96-cell mesh has two corner cells without a DOF vertex (their points take the
    # strong form of u itself)
    V, T = synth.disc(5, 2.0) if case == "disc" else synth.lshape(0.25, 0)
    om = OracleMesh(V, T)
    u = _u(om, s)
    m, eta, leaf = 3, 1.0, 8
    So = strong_form_cluster(om, s, u, m=m, eta=eta, leaf=leaf)
    _, size = oad.strong_form(om, s, u, with_abs=True)
    mesh = F.Mesh(V, T)
    H = F.HMatrix(mesh.h, s, m=m, eta=eta, leaf=leaf)
    Sg = H.strong_form(torch.tensor(u, device="cuda")).cpu().numpy()
    err = float(np.max(np.abs(Sg - So) / size))
    print(f"s {s}: cluster strong form vs oracle {err:.2e} of the terms' size")
    assert err <= TOL
    # the same u again: the same bits (fixed summation orders)
    Sg2 = H.strong_form(torch.tensor(u, device="cuda")).cpu().numpy()
    assert np.array_equal(Sg, Sg2)
    H.close()
    mesh.close()


def test_cluster_strong_form_converges_to_direct():
    # L-shape level 3 (19188 cells): the cluster form against the direct one (fl_strong_form) for
    # Chebyshev orders 2..6, leaves of 32, eta = 1; the indicators from it against the direct ones
    V, T = synth.lshape(0.25, 3)
    s = 0.5
    mesh = F.Mesh(V, T)
    A = mesh.assemble(s, "fp64")
    b = mesh.load_vector(s)
    u, _ = mesh.solve(A, b, tol=1e-10)
    Sd = mesh.strong_form(s, u)
    scale = float(Sd.abs().max())
    errs = []
    for m in (2, 3, 4, 5, 6):
        H = F.HMatrix(mesh.h, s, m=m, eta=1.0, leaf=32)
        Sc = H.strong_form(u)
        errs.append(float((Sc - Sd).abs().max()) / scale)
        if m == 6:
            eta_c, _ = H.br_indicators(u)
        H.close()
    print("cluster strong form vs direct, m = 2..6:", errs)
    assert all(b_ < a for a, b_ in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6
    eta_d = mesh.br_indicators(s, u)
    rel = float(((eta_c - eta_d).abs() / eta_d.abs().max()).max())
    print(f"indicators m = 6 vs direct: {rel:.2e}")
    assert rel < 1e-5
    mesh.close()


def test_cluster_strong_form_errors():
    V, T = synth.interval(16)
    mesh = F.Mesh(V, T)
    H = F.HMatrix(mesh.h, 0.5, m=3, leaf=4)
    u = torch.ones(mesh.num_dofs(0.5), dtype=torch.float64, device="cuda")
    with pytest.raises(F.FlError):
        H.strong_form(u)  # 1D
    H.close()
    mesh.close()
    V, T = synth.disc(4)
    mesh = F.Mesh(V, T)
    H = F.HMatrix(mesh.h, 0.3, m=3, leaf=4)
    with pytest.raises(F.FlError):
        H.strong_form(torch.ones(mesh.num_dofs(0.3), dtype=torch.float64, device="cuda"))  # s not a quarter
    H.close()
    mesh.close()


def test_adaptive_loop_with_the_cluster_method():
    # Section 7's loop on the L-shape from 96 cells with the cluster method throughout (near field by
    # local computations, H-matrix PCG, cluster strong form; m = 6) against the dense loop: the same
    # meshes while the indicators' difference stays below the marking threshold's margin, and the
    # estimator at the last common size within a few per cent
    from paper_1708_03912_gb300.fraclap import adaptive_loop

    V, T = synth.lshape(0.25, 0)
    dense = adaptive_loop(V, T, 0.5, 9, theta=0.8)
    clus = adaptive_loop(V, T, 0.5, 9, theta=0.8, cluster={"m": 6, "eta": 1.0, "leaf": 32})
    nd = [r["n"] for r in dense]
    nc = [r["n"] for r in clus]
    print("dense n", nd, "cluster n", nc)
    same = 0
    while same < min(len(nd), len(nc)) and nd[same] == nc[same] and np.array_equal(dense[same]["cells"], clus[same]["cells"]):
        same += 1
    assert same >= 4
    for k in range(same):
        ed = np.sqrt(np.sum(dense[k]["eta"] ** 2))
        ec = np.sqrt(np.sum(clus[k]["eta"] ** 2))
        assert abs(ec - ed) <= 1e-4 * ed, (k, ec, ed)
        assert np.max(np.abs(clus[k]["u"] - dense[k]["u"])) <= 1e-5 * np.max(np.abs(dense[k]["u"]))
    assert all(b >= a for a, b in zip(nc, nc[1:]))


def _golden_module():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "make_golden.py")
    spec = importlib.util.spec_from_file_location("make_golden", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _point_leaves(h, p, cells):
    """The leaf each cell-rule point of `cells` is grouped with by the host plan [cells, q], and the
    leaf of every DOF."""
    plan = F.fl_strong_form_cluster_plan(h, p["s"], p["eta"], p["leaf"], p["k_cell"])
    cp = F.fl_cluster_plan(h, p["s"], p["eta"], p["leaf"])
    perm = F.fl_near_region_plan(h, p["s"], 2, p["eta"], p["leaf"])["cell_perm"]
    q = p["k_cell"] ** 2
    pos = np.empty(len(perm), dtype=np.int64)
    pos[perm] = np.arange(len(perm))
    gnode = np.asarray(plan["gnode"])
    got = gnode[plan["pgroup"][(pos[cells][:, None] * q + np.arange(q)[None, :])]]
    node = cp["node"]
    leaf_of = np.full(len(cp["perm"]), -1)
    for c in range(len(node)):
        if node[c, 2] < 0:
            leaf_of[cp["perm"][node[c, 0]:node[c, 1]]] = c
    return got, leaf_of


def _sampled_cells_error(G, S_cells, point_leaf, leaf_of):
    """(error of the points grouped as the oracle grouped them, share of such points).  A point
    grouped otherwise must be a near-tie of its two closest DOFs (the rule's nodes may differ in the
    last bit between machines): its value belongs to the other leaf's split and is not compared."""
    size = np.asarray(G["size"])
    same = point_leaf == leaf_of[np.asarray(G["closest_dof"])]
    assert np.all(same | (np.asarray(G["gap"]) < 1e-12))
    err = float(np.max(np.abs(S_cells - np.asarray(G["values"]))[same] / size[same]))
    return err, float(same.mean())


def test_cluster_strong_form_full_size_sampled_cells():
    # L-shape level 5 (73,432 cells), the strong-form workload the benchmark times (m = 4, eta = 1,
    # leaves of 32): the cluster strong form at the points of seeded cells, the re-entrant corner's
    # and a convex corner's cell against the oracle's values, stored by tests/golden/make_golden.py
    # (minutes of oracle work at this size) and recomputed here should the mesh generator give
    # another mesh on this machine
    mg = _golden_module()
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "strong_form_cluster_lshape5.json")) as f:
        G = json.load(f)
    p = G["params"]
    V, T = synth.lshape(0.25, p["level"])
    if mg.mesh_hash(V, T) != G["mesh_hash"]:
        G.update(mg.strong_form_cluster_cells(V, T, p))
    s = p["s"]
    mesh = F.Mesh(V, T)
    vod = np.asarray(mesh.dof_vertices(s))
    assert hashlib.sha256(np.ascontiguousarray(vod, dtype="<i8").tobytes()).hexdigest() == G["vod_hash"]
    u = mg.smooth_u(np.asarray(V, dtype=np.float64)[vod])
    cells = np.asarray(G["cells"])
    point_leaf, leaf_of = _point_leaves(mesh.h, p, cells)
    H = F.HMatrix(mesh.h, s, m=p["m"], eta=p["eta"], leaf=p["leaf"])
    Sg = H.strong_form(torch.tensor(u, device="cuda"), p["k_cell"], p["k_edge"], p["k_near"]).cpu().numpy()
    H.close()
    mesh.close()
    err, share = _sampled_cells_error(G, Sg[cells], point_leaf, leaf_of)
    print(f"level 5 cluster strong form, {len(cells)} cells: {err:.2e} of the terms' size "
          f"({share:.0%} of the points grouped as the oracle grouped them)")
    assert share >= 0.5
    assert err <= TOL
