"""GPU parity of the batched path through the C ABI: the bfloat16 slices (bit for
bit), the tensor-core product (against the oracle's float64 evaluation of the same
split product, within the float32-accumulation bound) and the batched refined
solve (against Cholesky solves of the oracle matrix)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import OracleMesh, assemble_matrix, load_vector  # noqa: E402
from oracle.lowprec import abs_product, matmul_split, split_bf16  # noqa: E402
from oracle.solve import cholesky_solve  # noqa: E402
from paper_1708_03912_gb300 import fraclap as F  # noqa: E402
from paper_1708_03912_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def gpu_split(A, nslices):
    Ad = torch.tensor(A, device="cuda")
    S, d = F.split_bf16(Ad, nslices)
    torch.cuda.synchronize()
    return Ad, S, d


def untile(S, n, ns):
    """The slices as float64 arrays [ns, rows, cols] (padded to whole tiles), read from the
    tiled layout fraclap.h documents: 128 x 64 blocks, 128-byte swizzle inside a block."""
    mt, ch = -(-n // 128), -(-n // 64)
    raw = S.cpu().numpy().view(np.uint16).reshape(ns, mt, ch, 128, 64)
    r = np.arange(128)[:, None]
    q = np.arange(64)[None, :]
    pos = ((q // 8) ^ (r % 8)) * 8 + q % 8  # storage position of entry (r, q) in its row
    ent = np.take_along_axis(raw, np.broadcast_to(pos, raw.shape), axis=-1)
    full = ent.transpose(0, 1, 3, 2, 4).reshape(ns, mt * 128, ch * 64)
    return (full.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def sym_oracle(V, T, s):
    A, _ = assemble_matrix(OracleMesh(V, T), s)
    return 0.5 * (A + A.T)


@pytest.fixture(scope="module")
def disc10():
    V, T = synth.disc(10)
    return V, T, sym_oracle(V, T, 0.75)


def test_split_bit_exact(disc10):
    _, _, A = disc10
    n = A.shape[0]
    for ns in (1, 2):
        _, S, d = gpu_split(A, ns)
        assert S.numel() == F.fl_split_bf16_bytes(n, ns)
        dd, So = split_bf16(A, ns)
        assert np.array_equal(d.cpu().numpy(), dd)
        Sg = untile(S, n, ns)
        for k in range(ns):
            assert np.array_equal(Sg[k, :n, :n], So[k])
            assert not Sg[k, n:, :].any() and not Sg[k, :, n:].any()  # zero padding


@pytest.mark.parametrize("nrhs", [16, 64, 128])
@pytest.mark.parametrize("ns", [1, 2])
def test_tensor_core_product(disc10, nrhs, ns):
    _, _, A = disc10  # n = 284: 3 row tiles and 5 chunks, both ragged
    n = A.shape[0]
    _, S, _ = gpu_split(A, ns)
    rng = np.random.default_rng(nrhs + ns)
    X = rng.standard_normal((nrhs, n)).astype(np.float32)
    Y = torch.zeros((nrhs, n + 5), dtype=torch.float32, device="cuda")
    F.fl_matmul_bf16(S, n, ns, torch.tensor(X, device="cuda"), Y)
    torch.cuda.synchronize()
    Yg = Y[:, :n].cpu().numpy().astype(np.float64).T
    _, So = split_bf16(A, ns)
    Yo = matmul_split(So, X.T)
    scale = abs_product(So, X.T)
    err = np.max(np.abs(Yg - Yo) / scale)
    print(f"nrhs {nrhs} slices {ns}: max |Y - Y_oracle| / (|S||X|) = {err:.2e}")
    assert err < 2e-6  # float32 accumulation of a few hundred terms


def test_tensor_core_product_large():
    # several K ranges per CTA and several CTAs per tile: n = 5000 (40 row tiles, 79 chunks)
    rng = np.random.default_rng(1)
    n = 5000
    B = rng.standard_normal((n, n)) * 0.01
    A = B @ B.T / n + np.eye(n)
    A = 0.5 * (A + A.T)
    _, S, _ = gpu_split(A, 2)
    X = rng.standard_normal((64, n)).astype(np.float32)
    Y = torch.zeros((64, n), dtype=torch.float32, device="cuda")
    F.fl_matmul_bf16(S, n, 2, torch.tensor(X, device="cuda"), Y)
    torch.cuda.synchronize()
    Yg = Y.cpu().numpy().astype(np.float64).T
    _, So = split_bf16(A, 2)
    rows = synth.random_rows(n, 40)
    Yo = matmul_split([s[rows] for s in So], X.T)
    scale = abs_product([s[rows] for s in So], X.T)
    err = np.max(np.abs(Yg[rows] - Yo) / scale)
    print(f"n 5000: max |Y - Y_oracle| / (|S||X|) = {err:.2e}")
    assert err < 1e-5  # float32 accumulation of 5000 terms


def _problem(A, B, ns):
    Ad, S, d = gpu_split(A, ns)
    Bd = torch.tensor(B, device="cuda")
    U = torch.full_like(Bd, np.nan)
    return {"A": Ad, "S": S, "nslices": ns, "dscale": d, "B": Bd, "U": U}


def test_batched_solve_two_orders():
    V, T = synth.disc(10)
    om = OracleMesh(V, T)
    f = synth.gaussian_nodal(om.nv, 15)
    probs, ref = [], []
    for s in (0.25, 0.75):
        A = sym_oracle(V, T, s)
        B = np.concatenate([load_vector(om, s)[:, None], load_vector(om, s, f)], axis=1)
        probs.append(_problem(A, B, 2))
        ref.append(cholesky_solve(A, B))
    o = F.fl_default_batch_opts()
    o.tol = 1e-12
    # 1e-12 lies near the accuracy floor of the double-float residual for rough loads
    # (about 2^-46 || |A| |u| || / ||b||): judge this one with the float64 residual
    o.residual = F.FL_RESID_F64
    h = F.fl_create(V, T)
    r, info, rel, st = F.fl_batch_solve(h, probs, o)
    F.fl_destroy(h)
    assert r == F.FL_OK, (rel, st)
    assert np.all(st == F.FL_OK) and np.all(rel <= 1e-12)
    print(f"outer {info.outer_iterations} inner {info.inner_iterations} ctas {info.ctas} stages {info.stages}")
    for q, u in zip(probs, ref):
        Ug = q["U"].cpu().numpy()
        err = np.max(np.abs(Ug - u), axis=0) / np.max(np.abs(u), axis=0)
        assert np.all(err <= 1e-8), err


def test_batched_solve_uneven_meshes_and_edge_columns():
    h = F.fl_create(*synth.disc(4))
    problems = []
    refs = []
    for (V, T), s, nrhs, ns in (((synth.disc(8)), 0.5, 1, 2), (synth.square(7, 0.25), 0.9, 20, 2),
                                 (synth.lshape(0.25, 0), 0.3, 3, 1)):
        A = sym_oracle(V, T, s)
        n = A.shape[0]
        rng = np.random.default_rng(nrhs)
        B = rng.standard_normal((n, nrhs))
        if nrhs > 2:
            B[:, 1] = 0.0  # a zero right-hand side finishes at once with u = 0
        problems.append(_problem(A, B, ns))
        refs.append(cholesky_solve(A, B))
    o = F.fl_default_batch_opts()
    o.tol = 1e-10
    o.max_outer = 12
    r, info, rel, st = F.fl_batch_solve(h, problems, o)
    assert r == F.FL_OK, (rel, st)
    for q, u in zip(problems, refs):
        Ug = q["U"].cpu().numpy()
        scale = np.maximum(np.max(np.abs(u), axis=0), 1e-300)
        assert np.all(np.max(np.abs(Ug - u), axis=0) / scale <= 1e-7)
    assert np.all(problems[2]["U"][:, 1].cpu().numpy() == 0.0)
    F.fl_destroy(h)


def test_batched_solve_rejects_bad_input():
    h = F.fl_create(*synth.disc(4))
    A = sym_oracle(*synth.disc(4), 0.5)
    q = _problem(A, np.ones((A.shape[0], 1)), 2)
    with pytest.raises(F.FlError):
        F.fl_batch_solve(h, [], None)
    with pytest.raises(F.FlError):
        F.fl_batch_solve(h, [q] * 9, None)
    bad = dict(q)
    bad["nslices"] = 3
    with pytest.raises(F.FlError):
        F.fl_batch_solve(h, [bad], None)
    with pytest.raises(F.FlError):
        F.fl_matmul_bf16(q["S"], A.shape[0], 2, torch.zeros((20, A.shape[0]), device="cuda"),
                         torch.zeros((20, A.shape[0]), device="cuda"))
    F.fl_destroy(h)


@pytest.mark.parametrize("mode", ["df", "f64"])
def test_reported_residual_matches_float64(disc10, mode):
    # the residual that decides convergence (double-float or float64 FMA) agrees with a
    # float64 recomputation of B - A U on the host
    V, T, A = disc10
    rng = np.random.default_rng(2)
    B = rng.standard_normal((A.shape[0], 70))  # two column tiles of the residual
    q = _problem(A, B, 2)
    o = F.fl_default_batch_opts()
    o.tol = 1e-10
    o.residual = F.FL_RESID_DF if mode == "df" else F.FL_RESID_F64
    h = F.fl_create(V, T)
    r, info, rel, st = F.fl_batch_solve(h, [q], o)
    F.fl_destroy(h)
    assert r == F.FL_OK
    U = q["U"].cpu().numpy()
    nb = np.linalg.norm(B, axis=0)
    rel_host = np.linalg.norm(B - A @ U, axis=0) / nb
    assert np.all(rel <= 1e-10)
    # operands carried to 2^-48 (double-float) or 2^-53 (float64): the residual of column j
    # is exact to about 2^-46 || |A| |u_j| || (random right-hand sides make |A||u| >> |b|)
    floor = 2.0 ** -46 * np.linalg.norm(np.abs(A) @ np.abs(U), axis=0) / nb
    dev = np.abs(rel - rel_host)
    print(f"{mode}: max |rel - rel_host| = {dev.max():.2e}, max floor {floor.max():.2e}")
    assert np.all(dev <= 1e-3 * rel_host + floor)


def test_autotuner_feeds_the_solver(disc10):
    V, T, A = disc10
    rng = np.random.default_rng(4)
    q = _problem(A, rng.standard_normal((A.shape[0], 32)), 2)
    h = F.fl_create(V, T)
    F.fl_tune_clear()
    best, ms = F.fl_tune_batch(h, [q], reps=3)
    assert 2 <= best.stages <= 8 and 1 <= best.ctas and ms > 0
    assert F.fl_tune_lookup("batch_gemm", A.shape[0], 32, 2) == (best.stages, best.ctas)
    o = F.fl_default_batch_opts()
    o.tol = 1e-10
    r, info, rel, st = F.fl_batch_solve(h, [q], o)
    assert r == F.FL_OK and (info.stages, info.ctas) == (best.stages, best.ctas)
    F.fl_tune_clear()
    F.fl_destroy(h)


def test_batched_barrier_timeout_is_reported(disc10):
    # a 1 us grid-barrier bound in the persistent batched kernel: FL_ETIMEOUT, then the same
    # handle solves the same problem with the default bound
    V, T, A = disc10
    om = OracleMesh(V, T)
    B = np.concatenate([load_vector(om, 0.75)[:, None], load_vector(om, 0.75, synth.gaussian_nodal(om.nv, 15))], 1)
    q = _problem(A, B, 2)
    h = F.fl_create(V, T)
    o = F.fl_default_batch_opts()
    assert o.barrier_timeout_us == 0
    o.barrier_timeout_us = 1
    with pytest.raises(F.FlError) as e:
        F.fl_batch_solve(h, [q], o)
    assert e.value.code == F.FL_ETIMEOUT
    o.barrier_timeout_us = 0
    r, info, rel, st = F.fl_batch_solve(h, [q], o)
    F.fl_destroy(h)
    assert r == F.FL_OK and np.all(rel <= 1e-8)
