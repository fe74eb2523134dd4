"""GPU parity: the CUDA assembly through the C ABI against the CPU oracle, element by
element, on the same seeded meshes.  Tolerances: float64 mode |ΔA_ij| <= 1e-12 |A_ij|
for entries whose supports share no vertex (single-signed sums) and <= 1e-12
sqrt(A_ii A_jj) for touching supports (quadrature sums in a different order only);
mixed mode (float32 separated pairs) stated, bounded by 2e-5 of the scaled form."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import OracleMesh, QuadOrders, assemble_matrix, load_vector  # noqa: E402
from paper_1708_03912_gb300 import fraclap as F  # noqa: E402
from paper_1708_03912_gb300 import synth  # noqa: E402
from parity import check_f64  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
TOL64 = 1e-12


def scaled(A, E):
    d = np.sqrt(np.outer(np.diag(E), np.diag(E)))
    return float(np.max(np.abs(A - E) / d))


def gpu_matrix(V, T, s, precision="fp64", **kw):
    m = F.Mesh(V, T, **kw)
    A = m.assemble(s, precision)
    torch.cuda.synchronize()
    out = A.cpu().numpy()
    m.close()
    return out


@pytest.mark.parametrize("s", [0.25, 0.5, 0.75, 0.6])
def test_1d_parity(s):
    for V, T in (synth.interval(16), synth.interval(128), synth.graded_interval(70, 2.0)):
        om = OracleMesh(V, T)
        Ao, _ = assemble_matrix(om, s)
        Ag = gpu_matrix(V, T, s)
        check_f64(Ag, Ao, om, s, TOL64)


@pytest.mark.parametrize("s", [0.25, 0.5, 0.75, 0.6])
def test_2d_parity_disc(s):
    V, T = synth.disc(10)  # 629 cells: 20 tiles of 32 and a ragged tail
    om = OracleMesh(V, T)
    Ao, _ = assemble_matrix(om, s)
    Ag = gpu_matrix(V, T, s)
    check_f64(Ag, Ao, om, s, TOL64)


def test_2d_parity_lshape_and_square():
    for (V, T), s in ((synth.lshape(0.25, 0), 0.5), (synth.square(7, 0.25), 0.35)):
        om = OracleMesh(V, T)
        Ao, _ = assemble_matrix(om, s)
        Ag = gpu_matrix(V, T, s)
        check_f64(Ag, Ao, om, s, TOL64)


def test_orders_and_regional():
    V, T = synth.square(5, 0.2)
    om = OracleMesh(V, T)
    o = QuadOrders(k_far=3, k_near=5, k_touch=6, k_bnd=5, k_vertex=4)
    Ao, _ = assemble_matrix(om, 0.4, o)
    Ag = gpu_matrix(V, T, 0.4, k_far=3, k_near=5, k_touch=6, k_bnd=5, k_vertex=4)
    check_f64(Ag, Ao, om, 0.4, TOL64)
    Ao, _ = assemble_matrix(om, 0.4, dof_mode="paper", regional=True)
    Ag = gpu_matrix(V, T, 0.4, dof_mode="paper", regional=True)
    check_f64(Ag, Ao, om, 0.4, TOL64, dof_mode="paper")
    V1, T1 = synth.interval(40)
    om1 = OracleMesh(V1, T1)
    Ao, _ = assemble_matrix(om1, 0.3, dof_mode="paper")
    Ag = gpu_matrix(V1, T1, 0.3, dof_mode="paper")
    check_f64(Ag, Ao, om1, 0.3, TOL64, dof_mode="paper")


def test_exact_golden_high_orders():
    gold = json.load(open(os.path.join(GOLD, "square4_exact.json")))
    V, T = synth.square(4, 0.2)
    for s, E in gold["matrices"].items():
        Ag = gpu_matrix(V, T, float(s), k_far=6, k_near=12, k_touch=20, k_bnd=20, k_vertex=16)
        assert scaled(Ag, np.array(E)) < 1e-8
    gold = json.load(open(os.path.join(GOLD, "interval16_exact.json")))
    V, T = synth.interval(16)
    for s, E in gold["matrices"].items():
        Ag = gpu_matrix(V, T, float(s), k_far=8, k_near=12, k_touch=16, k_bnd=16)
        assert scaled(Ag, np.array(E)) < 1e-10


def test_mixed_precision_error_stated():
    V, T = synth.disc(10)
    s = 0.75
    Ao, _ = assemble_matrix(OracleMesh(V, T), s)
    Am = gpu_matrix(V, T, s, "mixed")
    err = scaled(Am, Ao)
    print(f"mixed-mode scaled error vs float64 oracle: {err:.3e}")
    assert err < 2e-5


def test_deterministic_and_symmetric():
    V, T = synth.disc(8)
    m = F.Mesh(V, T)
    for prec in ("fp64", "mixed"):
        A1 = m.assemble(0.6, prec).cpu()
        A2 = m.assemble(0.6, prec).cpu()
        assert torch.equal(A1, A2)
        assert torch.equal(A1, A1.T)
    m.close()


def test_concurrent_stages_match_serial_schedule():
    # without profiling the near / touching / boundary stages run on the handle's second stream,
    # concurrently with the far-field stage; with profiling every stage runs on the caller's
    # stream in turn.  Both schedules, and a CUDA graph captured from the concurrent one on a
    # side stream of the caller, give the same bits.
    V, T = synth.disc(10)
    m = F.Mesh(V, T)
    for prec in ("fp64", "mixed"):
        A_conc = m.assemble(0.75, prec).clone()
        F.fl_set_profiling(m.h, True)
        A_ser = m.assemble(0.75, prec).clone()
        F.fl_set_profiling(m.h, False)
        assert torch.equal(A_conc, A_ser)
        A_g = torch.full_like(A_conc, float("nan"))
        cap = torch.cuda.Stream()
        cap.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cap):
            m.assemble(0.75, prec, out=A_g)  # warm (tables already resident)
            g = torch.cuda.CUDAGraph()
            A_g.fill_(float("nan"))
            with torch.cuda.graph(g, stream=cap):
                m.assemble(0.75, prec, out=A_g)
        torch.cuda.current_stream().wait_stream(cap)
        A_g.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(A_g, A_conc)
    m.close()


@pytest.mark.parametrize("case", ["disc", "interval", "lshape"])
def test_nearfield_csr_parity(case):
    # N of A = N + F (far off-diagonal blocks left out) as CSR, against the oracle's N:
    # same pattern (bit-exact), values within the float64 parity tolerance; the mixed mode
    # within its stated bound
    from oracle.assemble import nearfield_pattern

    (V, T), s = {"disc": (synth.disc(10), 0.75), "interval": (synth.graded_interval(70, 2.0), 0.4),
                 "lshape": (synth.lshape(0.25, 0), 0.5)}[case]
    om = OracleMesh(V, T)
    No, _ = assemble_matrix(om, s, far_offdiag=False)
    pat = nearfield_pattern(om, s)
    d = np.sqrt(np.outer(np.diag(No), np.diag(No)))
    m = F.Mesh(V, T)
    for prec, tol in (("fp64", TOL64), ("mixed", 2e-5)):
        rowptr, col, val = m.nearfield_csr(s, prec)
        torch.cuda.synchronize()
        rp, cl, vl = rowptr.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
        n = len(rp) - 1
        assert n == No.shape[0] and rp[0] == 0 and rp[-1] == len(cl)
        G = np.zeros_like(No)
        Gp = np.zeros(No.shape, dtype=bool)
        for i in range(n):
            cols = cl[rp[i]:rp[i + 1]]
            assert np.all(np.diff(cols) > 0)  # ascending, no duplicates
            G[i, cols] = vl[rp[i]:rp[i + 1]]
            Gp[i, cols] = True
        assert np.array_equal(Gp, pat)
        assert np.array_equal(G, G.T)  # symmetric values
        assert float(np.max(np.abs(G - No) / d)) < tol, prec
    m.close()


def test_edge_cases():
    # one DOF in 1D, a single interior vertex in 2D, s close to 0 and 1
    V, T = synth.interval(2)
    for s in (0.05, 0.95):
        om = OracleMesh(V, T)
        Ao, _ = assemble_matrix(om, s)
        check_f64(gpu_matrix(V, T, s), Ao, om, s, TOL64)
    V = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1]], dtype=float)
    T = np.array([[0, 1, 2], [0, 2, 3], [0, 3, 4], [0, 4, 1]])
    for s in (0.05, 0.5, 0.95):
        om = OracleMesh(V, T)
        Ao, _ = assemble_matrix(om, s)
        check_f64(gpu_matrix(V, T, s), Ao, om, s, TOL64)
    # padded leading dimension
    V, T = synth.disc(4)
    m = F.Mesh(V, T)
    n = m.num_dofs(0.5)
    buf = torch.full((n, n + 7), 7.0, dtype=torch.float64, device="cuda")
    F.fl_assemble(m.h, 0.5, F.FL_FP64, buf)
    A = m.assemble(0.5)
    assert torch.equal(buf[:, :n], A) and torch.all(buf[:, n:] == 7.0)
    with pytest.raises(F.FlError):
        F.fl_assemble(m.h, 1.5, F.FL_FP64, A)
    m.close()


def test_load_vector_parity():
    V, T = synth.disc(6)
    om = OracleMesh(V, T)
    m = F.Mesh(V, T)
    b = m.load_vector(0.5).cpu().numpy()
    assert np.allclose(b, load_vector(om, 0.5), rtol=1e-14, atol=0)
    f = synth.gaussian_nodal(om.nv, 3)
    B = m.load_vector(0.5, torch.tensor(f, device="cuda")).cpu().numpy()
    assert np.allclose(B, load_vector(om, 0.5, f), rtol=1e-12, atol=1e-15)
    m.close()


def test_full_size_disc_sampled_rows():
    # the quasi-uniform disc of the benchmark (about 3.9k triangles), 12 seeded rows
    V, T = synth.disc(25)
    s = 0.75
    om = OracleMesh(V, T)
    m = F.Mesh(V, T)
    A = m.assemble(s, "fp64").cpu().numpy()
    Am = m.assemble(s, "mixed").cpu().numpy()
    m.close()
    n = A.shape[0]
    rows = synth.random_rows(n, 12)
    Ar, _ = assemble_matrix(om, s, rows=rows)
    check_f64(A, Ar, om, s, TOL64, rows=rows, diag=np.diag(A))
    d = np.sqrt(np.outer(np.diag(A)[rows], np.diag(A)))
    assert float(np.max(np.abs(Am[rows] - Ar) / d)) < 2e-5
    assert np.array_equal(A, A.T)


def test_full_size_graded_disc_sampled_rows():
    # the disc graded toward the boundary (30 rings, mu = 2: 22043 triangles, 8195 DOFs),
    # 3 seeded rows against the oracle, float64 and mixed modes
    V, T = synth.disc(30, 2.0)
    s = 0.5
    m = F.Mesh(V, T)
    A = m.assemble(s, "fp64").cpu().numpy()
    Am = m.assemble(s, "mixed").cpu().numpy()
    m.close()
    n = A.shape[0]
    assert n == 8195
    rows = synth.random_rows(n, 3)
    om = OracleMesh(V, T)
    Ar, _ = assemble_matrix(om, s, rows=rows)
    check_f64(A, Ar, om, s, TOL64, rows=rows, diag=np.diag(A))
    d = np.sqrt(np.outer(np.diag(A)[rows], np.diag(A)))
    assert float(np.max(np.abs(Am[rows] - Ar) / d)) < 2e-5


@pytest.mark.parametrize("s", [0.25, 0.5, 0.75])
def test_double_word_far_field_matches_float64_pipe(s):
    # the float64 mode evaluates the separated pairs at distance >= 2 in double-word arithmetic
    # (2D, k_far = 4, s in {1/4, 1/2, 3/4}); the same pairs on the float64 pipe give the same
    # matrix to well inside the 1e-12 entry tolerance, and both pass it against the oracle
    V, T = synth.disc(7, 2.0)  # graded toward the boundary: far pairs of very different sizes
    om = OracleMesh(V, T)
    Ao, _ = assemble_matrix(om, s)
    A_dw = gpu_matrix(V, T, s)
    A_64 = gpu_matrix(V, T, s, far_f64_pipe=True)
    check_f64(A_dw, Ao, om, s, TOL64)
    check_f64(A_64, Ao, om, s, TOL64)
    far, near = check_f64(A_dw, A_64, om, s, 1e-13)
    print(f"s {s}: double-word vs float64 pipe: {far:.1e} (disjoint supports), {near:.1e} (touching)")


def test_far_variants_and_autotuner():
    # every launch variant of the double-word far kernel gives the same bits; the autotuner
    # records its winner under (kernel, cell count) and later assemblies of a new handle on the
    # same mesh use it (same bits again)
    V, T = synth.disc(10)
    s = 0.75
    m = F.Mesh(V, T)
    ref = m.assemble(s, "fp64").clone()
    for v in (1, 2, 3, 4):
        F.fl_set_far_variant(m.h, v)
        assert torch.equal(m.assemble(s, "fp64"), ref), v
    F.fl_set_far_variant(m.h, 0)
    F.fl_tune_clear()
    best, ms = F.fl_tune_assemble(m.h, s, ref.clone(), reps=3)
    assert best in (1, 2, 3, 4) and ms > 0
    assert F.fl_tune_lookup("far_tile_dw<7>", len(T), 1, 1) == (best, 0)
    m2 = F.Mesh(V, T)
    assert torch.equal(m2.assemble(s, "fp64"), ref)
    with pytest.raises(F.FlError) as e:
        F.fl_tune_assemble(m2.h, 0.6, ref.clone(), reps=1)  # generic s: no double-word kernel
    assert e.value.code == F.FL_ENOTIMPL
    m2.close()
    m.close()
    F.fl_tune_clear()
