"""GPU parity of the dense matvec, conversions and the solvers against plain
float64 references (the oracle's Cholesky solve and numpy products)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import OracleMesh, assemble_matrix, exact, load_vector, solve  # noqa: E402
from paper_1708_03912_gb300 import fraclap as F  # noqa: E402
from paper_1708_03912_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def test_matvec_dtypes():
    g = torch.Generator(device="cpu").manual_seed(5)
    for n in (1, 37, 256, 1000, 1031):
        A = torch.randn(n, n, generator=g, dtype=torch.float64).cuda()
        X = torch.randn(n, 3, generator=g, dtype=torch.float64).cuda()
        Y = torch.empty(n, 3, dtype=torch.float64, device="cuda")
        F.fl_matvec(F.FL_F64, A, X, Y)
        ref = (A.cpu() @ X.cpu()).numpy()
        assert np.allclose(Y.cpu().numpy(), ref, rtol=1e-13, atol=1e-12 * np.sqrt(n))
        for dt, tdt, tol in ((F.FL_F32, torch.float32, 1e-5), (F.FL_BF16, torch.bfloat16, 2e-2)):
            Al = torch.empty(n, n, dtype=tdt, device="cuda")
            F.fl_convert(A, dt, Al)
            # round to nearest: within half a unit in the last place of the target type
            ulp = 2.0 ** -23 if dt == F.FL_F32 else 2.0 ** -7
            rel = ((Al.double() - A).abs() / A.abs()).max().item()
            assert rel <= 0.5 * ulp * (1 + 1e-9)
            F.fl_matvec(dt, Al, X, Y)
            ref = (Al.double().cpu() @ X.float().double().cpu()).numpy()
            assert np.allclose(Y.cpu().numpy(), ref, rtol=tol, atol=tol * np.sqrt(n))


def test_matvec_padded_rows():
    # leading dimension larger than n: 16-byte aligned rows (lda % 4 == 0) and rows whose
    # starts drift across the 16-byte boundary (odd lda), every storage type
    g = torch.Generator(device="cpu").manual_seed(6)
    n = 777
    for lda in (780, 781):
        Af = torch.randn(n, lda, generator=g, dtype=torch.float64).cuda()
        A = Af[:, :n]
        X = torch.randn(n, 2, generator=g, dtype=torch.float64).cuda()
        Y = torch.empty(n, 2, dtype=torch.float64, device="cuda")
        F.fl_matvec(F.FL_F64, A, X, Y)
        ref = (A.cpu() @ X.cpu()).numpy()
        assert np.allclose(Y.cpu().numpy(), ref, rtol=1e-13, atol=1e-12 * np.sqrt(n))
        for dt, tdt, tol in ((F.FL_F32, torch.float32, 1e-5), (F.FL_BF16, torch.bfloat16, 2e-2)):
            Alf = torch.zeros(n, lda, dtype=tdt, device="cuda")
            Al = Alf[:, :n]
            F.fl_convert(A, dt, Al)
            F.fl_matvec(dt, Al, X, Y)
            ref = (Al.double().cpu() @ X.float().double().cpu()).numpy()
            assert np.allclose(Y.cpu().numpy(), ref, rtol=tol, atol=tol * np.sqrt(n))


def test_f32x2_storage_and_product():
    # hi + lo float32 storage: bit-exact against the oracle's split; the double-float product
    # within 2^-40 of sum_j |a_ij x_j| of the float64 product, for 16-byte aligned rows, rows
    # drifting across the boundary (odd leading dimension), and an x too long to stage
    from oracle.lowprec import f32x2_product, f32x2_split

    g = torch.Generator(device="cpu").manual_seed(12)
    for n, lda in ((1, 1), (1000, 1000), (777, 781)):
        Af = torch.randn(n, lda, generator=g, dtype=torch.float64)
        A = Af[:, :n]
        X = torch.randn(n, 2, generator=g, dtype=torch.float64)
        A2 = torch.zeros(n, 2 * lda, dtype=torch.float32, device="cuda")  # (hi, lo) pairs, ld = lda
        Ad = Af.cuda()[:, :n]
        F.fl_convert(Ad, F.FL_F32X2, A2[:, :2 * n])
        hi, lo = f32x2_split(A.numpy())
        got = A2[:, :2 * n].cpu().numpy().reshape(n, n, 2)
        assert np.array_equal(got[..., 0], hi) and np.array_equal(got[..., 1], lo)
        Y = torch.empty(n, 2, dtype=torch.float64, device="cuda")
        F.fl_matvec(F.FL_F32X2, A2[:, :2 * n], X.cuda(), Y)
        ref = f32x2_product(hi, lo, X.numpy())
        bound = 2.0 ** -40 * (np.abs(A.numpy()) @ np.abs(X.numpy()))
        assert np.all(np.abs(Y.cpu().numpy() - ref) <= bound)
    # x beyond the shared-memory staging (25593 entries): sampled rows
    n = 25600
    gc = torch.Generator(device="cuda").manual_seed(13)
    Ad = torch.randn(n, n, generator=gc, dtype=torch.float64, device="cuda")
    A2 = torch.empty(n, 2 * n, dtype=torch.float32, device="cuda")
    F.fl_convert(Ad, F.FL_F32X2, A2)
    x = torch.randn(n, 1, generator=gc, dtype=torch.float64, device="cuda")
    y = torch.empty(n, 1, dtype=torch.float64, device="cuda")
    F.fl_matvec(F.FL_F32X2, A2, x, y)
    rows = synth.random_rows(n, 16)
    Ar = Ad[rows].cpu().numpy()
    hi, lo = f32x2_split(Ar)
    ref = f32x2_product(hi, lo, x.cpu().numpy())
    bound = 2.0 ** -40 * (np.abs(Ar) @ np.abs(x.cpu().numpy()))
    assert np.all(np.abs(y.cpu().numpy()[rows] - ref) <= bound)
    del Ad, A2


def test_matvec_autotuner_records_and_is_used():
    # the tuner sweeps blocks per SM of the staged product (float32: the row-dot product),
    # records the fastest, and the product taken with the recorded shape is still the product
    g = torch.Generator(device="cpu").manual_seed(9)
    n = 3001
    A = torch.randn(n, n, generator=g, dtype=torch.float64).cuda()
    A32 = torch.empty(n, n, dtype=torch.float32, device="cuda")
    F.fl_convert(A, F.FL_F32, A32)
    x = torch.randn(n, 1, generator=g, dtype=torch.float64).cuda()
    x1 = x[:, 0].contiguous()
    y1 = torch.empty(n, dtype=torch.float64, device="cuda")
    Y = torch.empty(n, 1, dtype=torch.float64, device="cuda")
    F.fl_tune_clear()
    for dt, Ad, name, ref, tol in ((F.FL_F64, A, "gemv_smem_f64", A.cpu() @ x.cpu(), 1e-13),
                                   (F.FL_F32, A32, "gemv_rows_f32", A32.double().cpu() @ x.float().double().cpu(), 1e-5)):
        per_sm, ms = F.fl_tune_matvec(dt, Ad, x1, y1, reps=3)
        assert per_sm >= 1 and ms > 0
        assert F.fl_tune_lookup(name, n, 1, 1) == (per_sm, 0)
        F.fl_matvec(dt, Ad, x, Y)
        assert np.allclose(Y.cpu().numpy(), ref.numpy(), rtol=tol, atol=tol * np.sqrt(n))
    F.fl_tune_clear()


def test_pcg_matches_cholesky_1d_closed_form():
    s = 0.25
    V, T = synth.interval(128)
    om = OracleMesh(V, T)
    m = F.Mesh(V, T)
    A = m.assemble(s)
    b = m.load_vector(s)
    u, info = m.solve(A, b, tol=1e-12)
    assert info.status == F.FL_OK and info.rel_residual <= 1e-12
    Ao, vod = assemble_matrix(om, s)
    uo = solve.cholesky_solve(Ao, load_vector(om, s))
    ug = u.cpu().numpy()
    assert np.max(np.abs(ug - uo)) <= 1e-8 * np.max(np.abs(uo))
    # energy identity against the closed form (Section 7.1)
    gap = exact.energy_f1(1, s) - float(b.cpu().numpy() @ ug)
    assert 0 < gap < 0.01
    m.close()


def test_pcg_and_mixed_refinement_2d():
    s = 0.75
    V, T = synth.disc(12)
    om = OracleMesh(V, T)
    m = F.Mesh(V, T)
    A = m.assemble(s)
    b = m.load_vector(s)
    Ao, _ = assemble_matrix(om, s)
    uo = solve.cholesky_solve(Ao, load_vector(om, s))
    u, info = m.solve(A, b, tol=1e-12)
    assert info.status == F.FL_OK
    assert np.max(np.abs(u.cpu().numpy() - uo)) <= 1e-8 * np.max(np.abs(uo))
    A32 = torch.empty_like(A, dtype=torch.float32)
    F.fl_convert(A, F.FL_F32, A32)
    u2, info2 = m.solve(A, b, tol=1e-10, A_lo=A32, inner_tol=1e-3)
    assert info2.status == F.FL_OK and info2.rel_residual <= 1e-10 and info2.outer_iterations >= 2
    assert np.max(np.abs(u2.cpu().numpy() - uo)) <= 1e-7 * np.max(np.abs(uo))
    # an inner tolerance below float32 resolution: the float32 recurrences lose accuracy
    # before reaching it, the inner solve ends there and the refinement still converges
    u4, info4 = m.solve(A, b, tol=1e-11, A_lo=A32, inner_tol=1e-9, inner_maxit=500)
    assert info4.status == F.FL_OK and info4.rel_residual <= 1e-11
    assert np.max(np.abs(u4.cpu().numpy() - uo)) <= 1e-8 * np.max(np.abs(uo))
    # the refinement's step limit is reported, not raised
    u5, info5 = m.solve(A, b, tol=1e-14, maxit=1, A_lo=A32, inner_tol=1e-3)
    assert info5.status == F.FL_ENOTCONV and info5.outer_iterations == 1
    # iteration limit is reported, not raised
    u3, info3 = m.solve(A, b, tol=1e-14, maxit=3)
    assert info3.status == F.FL_ENOTCONV
    m.close()


def test_pcg_reports_breakdown_on_indefinite_matrix():
    # [[1,2],[2,1]] has eigenvalues 3 and -1; from b = e_0 the second step meets p^T A p < 0
    n = 64
    A = torch.eye(n, dtype=torch.float64, device="cuda")
    A[0, 1] = A[1, 0] = 2.0
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    b[0] = 1.0
    V, T = synth.interval(4)
    m = F.Mesh(V, T)
    u = torch.empty_like(b)
    info = F.fl_solve(m.h, A, b, u)
    assert info.status == F.FL_ENOTSPD
    # the same through the refinement with the float32 inner solve
    A32 = A.to(torch.float32)
    _, info2 = m.solve(A, b, tol=1e-10, A_lo=A32)
    assert info2.status == F.FL_ENOTSPD
    m.close()


def test_small_systems_solve():
    # n = 1 (two intervals) and n = 39 (4-ring disc): workspace layout at tiny sizes
    for (V, T), s in ((synth.interval(2), 0.3), (synth.disc(4), 0.75)):
        om = OracleMesh(V, T)
        m = F.Mesh(V, T)
        A = m.assemble(s)
        b = m.load_vector(s)
        u, info = m.solve(A, b, tol=1e-12)
        Ao, _ = assemble_matrix(om, s)
        uo = solve.cholesky_solve(Ao, load_vector(om, s))
        assert info.status == F.FL_OK
        assert np.max(np.abs(u.cpu().numpy() - uo)) <= 1e-8 * np.max(np.abs(uo))
        m.close()


@pytest.mark.parametrize("s", [0.25, 0.5, 0.75])
def test_full_size_graded_disc_refined_solve(s):
    # the graded disc (8195 DOFs): float64-refined float32 Jacobi-PCG to 1e-8; the residual
    # ||b - A u|| / ||b|| recomputed on the host in float64 meets the tolerance, and the
    # plain float64 solve agrees with the refined one to within what the two residuals allow
    V, T = synth.disc(30, 2.0)
    m = F.Mesh(V, T)
    A = m.assemble(s, "mixed")
    A32 = torch.empty_like(A, dtype=torch.float32)
    F.fl_convert(A, F.FL_F32, A32)
    b = m.load_vector(s)
    u, info = m.solve(A, b, tol=1e-8, A_lo=A32, inner_tol=1e-3)
    assert info.status == F.FL_OK
    Ah, bh, uh = A.cpu().numpy(), b.cpu().numpy(), u.cpu().numpy()
    rel = np.linalg.norm(bh - Ah @ uh) / np.linalg.norm(bh)
    assert rel <= 1.05e-8 and abs(rel - info.rel_residual) <= 1e-3 * rel + 1e-15
    u64, i64 = m.solve(A, b, tol=1e-8)
    assert i64.status == F.FL_OK
    d = u64.cpu().numpy() - uh
    # A d = r_refined - r_f64, so ||d||_A^2 <= (||r1|| + ||r2||) ||d||
    assert float(d @ (Ah @ d)) <= 2.1e-8 * np.linalg.norm(bh) * np.linalg.norm(d) + 1e-30
    m.close()


def test_barrier_timeout_is_reported_and_the_handle_stays_usable():
    # a grid-barrier bound of 1 us cannot be met by 152 blocks doing real work between
    # barriers: the cooperative solve gives up, reports FL_ETIMEOUT, and the next call on the
    # same handle (default bound) converges.  Every wait gives up and returns; nothing hangs.
    V, T = synth.disc(25)
    s = 0.75
    m = F.Mesh(V, T)
    A = m.assemble(s, "fp64")
    A32 = torch.empty(A.shape, dtype=torch.float32, device="cuda")
    F.fl_convert(A, F.FL_F32, A32)
    b = m.load_vector(s)
    u = torch.empty_like(b)
    for refined in (False, True):
        o = F.fl_default_solve_opts()
        assert o.barrier_timeout_us == 0
        o.tol = 1e-10
        if refined:
            o.inner_dtype = F.FL_F32
            o.A_lo_dev = A32.data_ptr()
            o.ld_lo = A32.stride(0)
        o.barrier_timeout_us = 1
        with pytest.raises(F.FlError) as e:
            F.fl_solve(m.h, A, b, u, o)
        assert e.value.code == F.FL_ETIMEOUT
        assert "grid barrier" in str(e.value)
        o.barrier_timeout_us = 0
        info = F.fl_solve(m.h, A, b, u, o)
        assert info.status == F.FL_OK and info.rel_residual <= 1e-10
    o = F.fl_default_solve_opts()
    o.barrier_timeout_us = -1
    with pytest.raises(F.FlError) as e:
        F.fl_solve(m.h, A, b, u, o)
    assert e.value.code == F.FL_EINVAL
    m.close()
