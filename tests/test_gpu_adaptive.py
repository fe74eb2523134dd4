"""GPU parity of the adaptive loop (Section 4, Appendix A, Section 7) against the oracle: the
strong form (-Delta)^s u_h at the cell-rule points, the BR indicators, maximum marking and the
refined meshes of whole loops."""
import numpy as np
import pytest

from oracle import OracleMesh
from oracle import adaptive as oad
from paper_1708_03912_gb300 import synth

pytestmark = pytest.mark.gpu

# Strong form: float64 on both sides, the GPU's far sum in double-word arithmetic for
# s in {1/4, 1/2, 3/4}.  The sum cancels: at each point its terms add up, in absolute value,
# to 10-400 times the field (largest for smooth u, where (-Delta)^s u_h is close to f).  Any
# evaluation of it errs by a few rounding units of each term: the oracle's float64 sum to
# ~2.4e-14 of that size (against a long-double evaluation), a double-word term to about
# 2^-44.  So per point |S_gpu - S_oracle| <= 2^-40 * size, size = C sum |terms| as the
# oracle reports it (with_abs); the field-relative error is printed beside it.
TOL = 2.0 ** -40


def _u(n, seed=3):
    return np.random.default_rng(seed).standard_normal(n)


def _check(Sg, So, size, tol=TOL):
    """max |S_gpu - S_oracle| / size (asserted <= tol) and the field-relative error."""
    err = float(np.max(np.abs(Sg - So) / size))
    field = float(np.max(np.abs(Sg - So) / (np.abs(So) + np.sqrt(np.mean(So ** 2)))))
    assert err <= tol, (err, field)
    return err, field


def test_strong_form_smooth_solution():
    # u the discrete solution for f = 1: the strong form is close to 1 inside while its terms
    # are not (the cancellation is largest); bounded by 2^-40 of the oracle's sum of absolute terms
    import torch
    from oracle import assemble_matrix, load_vector, solve
    from paper_1708_03912_gb300.fraclap import Mesh

    V, T = synth.disc(4)
    om = OracleMesh(V, T)
    for s in (0.25, 0.5, 0.75):
        A, _ = assemble_matrix(om, s)
        u = solve.cholesky_solve(A, load_vector(om, s))
        Sg = Mesh(V, T).strong_form(s, torch.tensor(u, device="cuda")).cpu().numpy()
        So, size = oad.strong_form(om, s, u, with_abs=True)
        print("smooth", s, _check(Sg, So, size))


def _mesh(case):
    if case == "disc":
        return synth.disc(4, 2.0)
    if case == "lshape":
        return synth.bisect_all(*synth.lshape(levels=0), rounds=1)
    if case == "square":
        return synth.square(5, jitter=0.15)
    raise ValueError(case)


@pytest.mark.parametrize("case,s", [("disc", 0.25), ("disc", 0.5), ("disc", 0.75), ("lshape", 0.5),
                                    ("square", 0.75), ("disc", 0.6), ("lshape", 0.3)])
def test_strong_form_2d(case, s):
    import torch
    from paper_1708_03912_gb300.fraclap import Mesh

    V, T = _mesh(case)
    om = OracleMesh(V, T)
    n = len(om.dofs(s)[0])
    u = _u(n)
    m = Mesh(V, T)
    Sg = m.strong_form(s, torch.tensor(u, device="cuda"), k_cell=3, k_edge=4, k_near=16).cpu().numpy()
    So, size = oad.strong_form(om, s, u, k_cell=3, k_edge=4, k_near=16, with_abs=True)
    print(case, s, _check(Sg, So, size))
    # deterministic: a second call gives the same bits
    Sg2 = m.strong_form(s, torch.tensor(u, device="cuda"), k_cell=3, k_edge=4, k_near=16).cpu().numpy()
    assert np.array_equal(Sg, Sg2)
    m.close()


@pytest.mark.parametrize("s", [0.25, 0.5, 0.75])
def test_strong_form_float64_pipe_and_orders(s):
    import torch
    from paper_1708_03912_gb300.fraclap import Mesh

    V, T = synth.disc(4)
    om = OracleMesh(V, T)
    u = _u(len(om.dofs(s)[0]), 5)
    ut = torch.tensor(u, device="cuda")
    a = Mesh(V, T).strong_form(s, ut, k_cell=2, k_edge=6, k_near=24).cpu().numpy()
    b = Mesh(V, T, far_f64_pipe=True).strong_form(s, ut, k_cell=2, k_edge=6, k_near=24).cpu().numpy()
    So, size = oad.strong_form(om, s, u, k_cell=2, k_edge=6, k_near=24, with_abs=True)
    print("dw", s, _check(a, So, size), "f64 pipe", _check(b, So, size))


def test_strong_form_paper_dofs():
    # s < 1/2 with boundary vertices as degrees of freedom: the boundary facets' u(y) term
    import torch
    from paper_1708_03912_gb300.fraclap import Mesh

    V, T = synth.disc(4, 2.0)
    om = OracleMesh(V, T)
    for s in (0.25, 0.3):
        n = len(om.dofs(s, "paper")[0])
        u = _u(n, 7)
        Sg = Mesh(V, T, dof_mode="paper").strong_form(s, torch.tensor(u, device="cuda")).cpu().numpy()
        So, size = oad.strong_form(om, s, u, dof_mode="paper", with_abs=True)
        print("paper", s, _check(Sg, So, size))


@pytest.mark.parametrize("s", [0.25, 0.5, 0.75, 0.4])
def test_strong_form_1d(s):
    import torch
    from paper_1708_03912_gb300.fraclap import Mesh

    V, T = synth.graded_interval(40, 2.0)
    om = OracleMesh(V, T)
    u = _u(len(om.dofs(s)[0]), 9)
    Sg = Mesh(V[:, 0], T).strong_form(s, torch.tensor(u, device="cuda"), k_cell=4).cpu().numpy()
    So, size = oad.strong_form(om, s, u, k_cell=4, with_abs=True)
    print("1d", s, _check(Sg, So, size))


@pytest.mark.parametrize("case,s,fnodal", [("lshape", 0.5, False), ("disc", 0.25, True), ("disc", 0.75, False)])
def test_indicators_and_marking(case, s, fnodal):
    import torch
    from paper_1708_03912_gb300.fraclap import Mesh

    V, T = _mesh(case)
    om = OracleMesh(V, T)
    m = Mesh(V, T)
    A = m.assemble(s)
    f = np.cos(V[:, 0]) + V[:, 1] ** 2 if fnodal else None
    ft = torch.tensor(f, device="cuda") if fnodal else None
    b = m.load_vector(s, ft)
    u, info = m.solve(A, b, tol=1e-12)
    eta, S = m.br_indicators(s, u, ft, return_S=True)
    eta = eta.cpu().numpy()
    ref = oad.br_indicators(om, s, u.cpu().numpy(), f)
    assert np.max(np.abs(eta - ref) / np.max(ref)) < 1e-10
    # marking: the oracle's decision taken on the GPU's indicators, bit for bit
    dm, cm = m.mark_max(s, torch.tensor(eta, device="cuda"), 0.8)
    want = oad.mark_max(eta, 0.8)
    assert np.array_equal(dm.cpu().numpy().astype(bool), want)
    cells = oad.marked_cells(om, s, want)
    got = np.nonzero(cm.cpu().numpy())[0]
    assert np.array_equal(got, cells)
    m.close()


def test_adaptive_loop_lshape():
    # the loop of Section 7 on the L-shape from its 96-cell start, s = 1/2: every refined mesh
    # is the oracle's refinement of the marked patches; the estimator falls
    from paper_1708_03912_gb300.fraclap import adaptive_loop

    V, T = synth.lshape(levels=0)
    steps = adaptive_loop(V, T, 0.5, steps=5, theta=0.8)
    assert len(steps) == 5
    est = [float(np.sqrt(np.sum(st["eta"] ** 2))) for st in steps]
    ns = [st["n"] for st in steps]
    print("n", ns, "estimator", est)
    assert all(b > a for a, b in zip(ns, ns[1:]))
    assert est[-1] < est[0]
    for a, b in zip(steps, steps[1:]):
        om = OracleMesh(a["vertices"], a["cells"])
        marks = oad.marked_cells(om, 0.5, a["dof_marks"].astype(bool))
        cm = np.zeros(len(a["cells"]), bool)
        cm[marks] = True
        assert np.array_equal(cm, a["cell_marks"].astype(bool))
        V2, T2 = oad.refine(a["vertices"], a["cells"], cm)
        assert np.array_equal(V2, b["vertices"]) and np.array_equal(T2.astype(np.int32), b["cells"])
    # the last step's indicators against the oracle's on the same solution
    last = steps[-1]
    om = OracleMesh(last["vertices"], last["cells"])
    ref = oad.br_indicators(om, 0.5, last["u"])
    assert np.max(np.abs(last["eta"] - ref) / np.max(ref)) < 1e-10


def test_strong_form_full_size_sampled():
    # the L-shape at level 5 (73432 cells, s = 1/2), the launch configuration of the benchmark:
    # sampled cells against the oracle point by point
    import torch
    from paper_1708_03912_gb300.fraclap import Mesh

    V, T = synth.lshape(levels=5)
    om = OracleMesh(V, T)
    s = 0.5
    n = len(om.dofs(s)[0])
    u = _u(n, 13)
    Sg = Mesh(V, T).strong_form(s, torch.tensor(u, device="cuda")).cpu().numpy()
    rng = np.random.default_rng(17)
    cells = np.concatenate([[0, len(T) - 1], rng.choice(len(T), 4, replace=False)])
    So, size = oad.strong_form(om, s, u, cells=cells, with_abs=True)
    err = float(np.max(np.abs(Sg[cells] - So) / size))
    field = float(np.max(np.abs(Sg[cells] - So) / (np.abs(So) + np.sqrt(np.mean(Sg ** 2)))))
    print("L5 sampled", err, field)
    assert err <= TOL
