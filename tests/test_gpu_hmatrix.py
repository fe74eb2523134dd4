"""GPU parity of the cluster method (Section 6) through the C ABI: the H-matrix product
against the oracle's restatement (same tree, partition and Chebyshev data, near entries
from the float64 matrices), and against the dense product with an error that falls
geometrically with the Chebyshev order."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import OracleMesh, assemble_matrix  # noqa: E402
from oracle.cluster import hmatvec  # noqa: E402
from paper_1708_03912_gb300 import fraclap as F  # noqa: E402
from paper_1708_03912_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["disc", "interval"])
def test_hmatrix_product_matches_oracle(case):
    (V, T), s, leaf, m, eta = {"disc": (synth.disc(7, 2.0), 0.5, 4, 4, 1.0),
                               "interval": (synth.graded_interval(60, 2.0), 0.25, 2, 5, 1.0)}[case]
    om = OracleMesh(V, T)
    Ao, _ = assemble_matrix(om, s)
    x = np.sin(np.arange(Ao.shape[0]) * 0.37)
    yo = hmatvec(Ao, om, s, x, m=m, eta=eta, leaf=leaf)
    mesh = F.Mesh(V, T)
    A = mesh.assemble(s, "fp64")
    H = F.HMatrix(mesh.h, s, m=m, eta=eta, leaf=leaf)
    H.set_near(A)
    xd = torch.tensor(x, device="cuda")
    y = torch.full_like(xd, float("nan"))
    H.matvec(xd, y)
    y2 = torch.empty_like(y)
    H.matvec(xd, y2)
    torch.cuda.synchronize()
    assert torch.equal(y, y2)  # fixed summation order
    yg = y.cpu().numpy()
    err = np.linalg.norm(yg - yo) / np.linalg.norm(yo)
    print(f"{case}: GPU H-matrix product vs oracle: {err:.2e}; info {H.info()}")
    assert err < 1e-12
    H.close()
    mesh.close()


def test_hmatrix_converges_to_dense_product():
    V, T = synth.lshape(0.25, 3)  # 19188 triangles, n = 9083
    s = 0.5
    mesh = F.Mesh(V, T)
    A = mesh.assemble(s, "fp64")
    n = A.shape[0]
    g = torch.Generator().manual_seed(7)
    x = torch.randn(n, generator=g, dtype=torch.float64).cuda()
    ref = A @ x
    errs = []
    for m in (2, 3, 4, 5, 6):
        H = F.HMatrix(mesh.h, s, m=m, eta=1.0, leaf=32)
        H.set_near(A)
        y = torch.empty_like(x)
        H.matvec(x, y)
        errs.append(float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref)))
        info = H.info()
        H.close()
    print("H-matrix relative error by Chebyshev order 2..6:", errs, info)
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6
    assert info["near_entries"] < 0.25 * n * n  # the near field is a small part of the matrix
    mesh.close()


def test_hmatrix_errors():
    V, T = synth.disc(5)
    mesh = F.Mesh(V, T)
    H = F.HMatrix(mesh.h, 0.5, m=3, leaf=4)
    x = torch.ones(mesh.num_dofs(0.5), dtype=torch.float64, device="cuda")
    with pytest.raises(F.FlError):
        H.matvec(x, torch.empty_like(x))  # no near field yet
    H.set_near(mesh.assemble(0.5, "fp64"))
    with pytest.raises(F.FlError):
        H.matvec(x, x)
    with pytest.raises(F.FlError):
        F.HMatrix(mesh.h, 0.5, m=0)
    H.close()
    mesh.close()


def test_hmatrix_solve():
    # Jacobi-PCG with the H-matrix product (Section 5's solver, Section 6's operator): the
    # returned u satisfies the stated residual with the oracle's H-matrix product, and it is
    # the dense solution up to the far field's interpolation error
    from oracle import load_vector, solve

    V, T = synth.disc(7, 2.0)
    s, m, leaf = 0.5, 6, 4
    om = OracleMesh(V, T)
    Ao, _ = assemble_matrix(om, s)
    bo = load_vector(om, s)
    mesh = F.Mesh(V, T)
    A = mesh.assemble(s, "fp64")
    H = F.HMatrix(mesh.h, s, m=m, eta=1.0, leaf=leaf)
    H.set_near(A)
    b = torch.tensor(bo, device="cuda")
    u, info = H.solve(b, tol=1e-10)
    assert info.status == F.FL_OK and info.rel_residual <= 1e-10
    ug = u.cpu().numpy()
    res = np.linalg.norm(bo - hmatvec(Ao, om, s, ug, m=m, eta=1.0, leaf=leaf)) / np.linalg.norm(bo)
    assert res <= 2e-10, res
    uo = solve.cholesky_solve(Ao, bo)
    err = np.max(np.abs(ug - uo)) / np.max(np.abs(uo))
    _, idense = mesh.solve(A, b, tol=1e-10)
    print(f"H-matrix solve: {info.iterations} steps (dense {idense.iterations}), residual {res:.1e}, "
          f"error vs dense {err:.1e}")
    assert err < 1e-6
    assert abs(info.iterations - idense.iterations) <= 3
    # a limit of one step reports that it did not converge
    _, i1 = H.solve(b, tol=1e-12, maxit=1)
    assert i1.status == F.FL_ENOTCONV and i1.iterations == 1
    H.close()
    mesh.close()


def _share_cell(om, vod, rows, cols):
    """For entries (rows[z], cols[z]): whether the two DOFs lie in a common cell."""
    dov = -np.ones(om.nv, dtype=np.int64)
    dov[vod] = np.arange(len(vod))
    pairs = set()
    for cell in om.C:
        ds = [int(dov[v]) for v in cell if dov[v] >= 0]
        for i in ds:
            for j in ds:
                pairs.add((i, j))
    return np.array([(int(i), int(j)) in pairs for i, j in zip(rows, cols)], dtype=bool)


@pytest.mark.parametrize("case", ["disc", "interval"])
def test_near_field_assembled_matches_oracle(case):
    # Section 6's near field from local computations: the diagonal blocks take the integral over
    # the boundary of N(K) (oracle: assemble_matrix(self_term="near_region")); entries of DOFs
    # sharing no cell are the dense float64 matrix's, bit for bit
    (V, T), s, leaf = {"disc": (synth.disc(7, 2.0), 0.5, 8),
                       "interval": (synth.graded_interval(60, 2.0), 0.25, 4)}[case]
    om = OracleMesh(V, T)
    B, vod = assemble_matrix(om, s, self_term="near_region")
    mesh = F.Mesh(V, T)
    A = mesh.assemble(s, "fp64").cpu().numpy()
    H = F.HMatrix(mesh.h, s, m=4, eta=1.0, leaf=leaf)
    H.assemble_near()
    rowptr, col, val = H.get_near()
    H.assemble_near()  # recomputed in the same order
    _, _, val2 = H.get_near()
    assert torch.equal(val, val2)
    rp = rowptr.cpu().numpy()
    r = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    c = col.cpu().numpy()
    v = val.cpu().numpy()
    assert np.all(np.isfinite(v))
    share = _share_cell(om, vod, r, c)
    D = np.sqrt(np.abs(np.diag(B))[r] * np.abs(np.diag(B))[c])
    err_share = float(np.max(np.abs(v - B[r, c])[share] / D[share]))
    err_other = float(np.max(np.abs(v - B[r, c])[~share] / np.abs(B[r, c])[~share]))
    print(f"{case}: {len(v)} near entries, {int(share.sum())} sharing a cell: vs oracle {err_share:.2e} (scaled), "
          f"others {err_other:.2e} (relative); plan {H.near_info()}")
    assert err_share < 1e-12 and err_other < 1e-12
    assert np.array_equal(v[~share], A[r, c][~share])
    # the pattern is symmetric and so are the values, bit for bit
    key = dict(zip(zip(r.tolist(), c.tolist()), v.tolist()))
    assert all(key[(j, i)] == x for (i, j), x in key.items())
    # the product with this near field against the oracle's H-matrix product with B's entries
    x = np.cos(np.arange(len(vod)) * 0.41)
    yo = hmatvec(B, om, s, x, m=4, eta=1.0, leaf=leaf)
    y = torch.empty(len(vod), dtype=torch.float64, device="cuda")
    H.matvec(torch.tensor(x, device="cuda"), y)
    assert np.linalg.norm(y.cpu().numpy() - yo) / np.linalg.norm(yo) < 1e-12
    H.close()
    mesh.close()


def test_near_field_assembled_at_size_against_dense():
    # L-shape level 3 (n = 9083): the assembled near field against the one gathered from the dense
    # float64 matrix; the two solves agree to the quadrature error of the diagonal blocks' far part
    V, T = synth.lshape(0.25, 3)
    s = 0.5
    mesh = F.Mesh(V, T)
    A = mesh.assemble(s, "fp64")
    n = A.shape[0]
    Hd = F.HMatrix(mesh.h, s, m=5, eta=1.0, leaf=32)
    Hd.set_near(A)
    Ha = F.HMatrix(mesh.h, s, m=5, eta=1.0, leaf=32)
    Ha.assemble_near()
    rp, col, vd = Hd.get_near()
    _, _, va = Ha.get_near()
    r = torch.repeat_interleave(torch.arange(n, device="cuda"), (rp[1:] - rp[:-1]).long())
    c = col.long()
    dg = torch.diagonal(A)
    scale = torch.sqrt(dg[r] * dg[c])
    diff = (va - vd).abs()
    same = diff == 0
    rel = float((diff / scale).max())
    info = Ha.near_info()
    print(f"near entries {len(vd)}, bitwise equal {int(same.sum())}, max scaled difference {rel:.2e}; {info}")
    assert rel < 5e-6
    assert int(same.sum()) > 0.9 * len(vd)
    st = F.fl_get_stats(mesh.h, s)
    assert 0 < info["tiles"] < st["n_tiles"]
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    ud, idd = Hd.solve(b, tol=1e-10)
    ua, ia = Ha.solve(b, tol=1e-10)
    assert idd.status == F.FL_OK and ia.status == F.FL_OK
    assert float((ua - ud).abs().max() / ud.abs().max()) < 1e-5
    # the mixed mode (float32 tiles, near and touching pairs, identical pair): within the dense mixed
    # mode's bound of the float64 entries
    Hm = F.HMatrix(mesh.h, s, m=5, eta=1.0, leaf=32)
    Hm.assemble_near("mixed")
    _, _, vm = Hm.get_near()
    relm = float(((vm - va).abs() / scale).max())
    print(f"mixed near field vs float64: {relm:.2e} (scaled)")
    assert relm < 2e-5
    um, im = Hm.solve(b, tol=1e-10)
    assert im.status == F.FL_OK and float((um - ua).abs().max() / ua.abs().max()) < 1e-4
    Hm.close()
    # the dense assembly on the same handle is unchanged by it
    A2 = mesh.assemble(s, "fp64")
    assert torch.equal(A, A2)
    Hd.close()
    Ha.close()
    mesh.close()


def test_near_field_assembled_without_dense_tables():
    # the direct near field never allocates the dense assembly's O(n^2) tables: on a fresh handle
    # the workspace stays a small multiple of the near field's own size
    V, T = synth.lshape(0.25, 4)
    s = 0.5
    mesh = F.Mesh(V, T)
    H = F.HMatrix(mesh.h, s, m=4, eta=1.0, leaf=32)
    H.assemble_near()
    st = F.fl_get_stats(mesh.h, s)
    info, ninfo = H.info(), H.near_info()
    n = st["n_dofs"]
    print(f"n = {n}: handle workspace {st['workspace_bytes'] / 2**20:.0f} MiB, near field {info['near_entries']} "
          f"entries, near plan {ninfo}")
    # (the dense tables alone would take ~250 KB per DOF at this size: row sums nblk x cells x 16)
    assert st["workspace_bytes"] < 64 * 1024 * n
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    u, i = H.solve(b, tol=1e-8)
    assert i.status == F.FL_OK and torch.isfinite(u).all()
    H.close()
    mesh.close()


def test_heat_steps_with_the_hmatrix():
    # implicit Euler (M + dt A) u^{k+1} = M u^k + dt F with the cluster method (shifted H-matrix PCG,
    # near field by local computations) against the dense heat steps: within the far field's
    # interpolation error
    V, T = synth.disc(10, 2.0)
    s, dt, steps = 0.5, 1e-3, 5
    mesh = F.Mesh(V, T)
    A = mesh.assemble(s, "fp64")
    b = mesh.load_vector(s)
    u0 = torch.zeros_like(b)
    ud, _ = mesh.heat_steps(A, s, dt, u0, b, steps)
    H = F.HMatrix(mesh.h, s, m=6, eta=1.0, leaf=16)
    H.assemble_near()
    uh, infos = H.heat_steps(dt, u0, b, steps)
    err = float((uh - ud).abs().max() / ud.abs().max())
    print(f"heat steps, H-matrix vs dense: {err:.2e}; CG steps {[i.iterations for i in infos]}")
    assert err < 1e-5
    assert all(i.status == F.FL_OK for i in infos)
    # alpha = 0, beta = 1 is the plain solve
    u1, i1 = H.solve(b, tol=1e-10)
    u2, i2 = H.solve_shifted(b, 0.0, 1.0, tol=1e-10)
    assert torch.equal(u1, u2) and i1.iterations == i2.iterations
    with pytest.raises(F.FlError):
        H.solve_shifted(b, 1.0, 0.0)
    H.close()
    mesh.close()


def _near_rows_error(rows, rp, col, val, B, om, vod, diag):
    """Max errors of near-field rows against the oracle's rows B (one per sampled DOF): entries of DOFs
    sharing a cell scaled by sqrt(a_ii a_jj) (diag: the near field's own diagonal), the others relative
    to themselves."""
    dov = -np.ones(om.nv, dtype=np.int64)
    dov[vod] = np.arange(len(vod))
    e_share = e_other = 0.0
    for k, i in enumerate(rows):
        cols = col[rp[i]:rp[i + 1]]
        v = val[rp[i]:rp[i + 1]]
        share = set()
        for c in om.cells_of_vertex[vod[i]]:
            share.update(int(dov[w]) for w in om.C[c] if dov[w] >= 0)
        sh = np.isin(cols, sorted(share))
        ref = B[k, cols]
        if sh.any():
            e_share = max(e_share, float(np.max(np.abs(v[sh] - ref[sh]) / np.sqrt(diag[i] * diag[cols[sh]]))))
        if (~sh).any():
            e_other = max(e_other, float(np.max(np.abs(v[~sh] - ref[~sh]) / np.abs(ref[~sh]))))
    return e_share, e_other


def test_near_field_full_size_sampled_rows():
    # the headline mesh (L-shape level 5, n = 35,693; 47 M near-field entries), two seeded DOF rows of
    # the directly assembled near field against the oracle's near-region rows
    V, T = synth.lshape(0.25, 5)
    s = 0.5
    om = OracleMesh(V, T)
    vod, _ = om.dofs(s)
    rows = np.sort(np.random.default_rng(11).choice(len(vod), 2, replace=False))
    B, _ = assemble_matrix(om, s, rows=rows, self_term="near_region")
    mesh = F.Mesh(V, T)
    H = F.HMatrix(mesh.h, s, m=4, eta=1.0, leaf=32)
    H.assemble_near()
    rp, col, val = H.get_near()
    rp = rp.cpu().numpy().astype(np.int64)
    col = col.cpu().numpy()
    val = val.cpu().numpy()
    n = len(vod)
    diag = np.empty(n)
    for i in range(n):
        c = col[rp[i]:rp[i + 1]]
        diag[i] = val[rp[i] + int(np.searchsorted(c, i))]
    e_share, e_other = _near_rows_error(rows, rp, col, val, B, om, vod, diag)
    print(f"full-size near-field rows {rows.tolist()}: {e_share:.2e} (sharing a cell, scaled), {e_other:.2e} (others)")
    assert e_share < 1e-12 and e_other < 1e-12
    H.close()
    mesh.close()
