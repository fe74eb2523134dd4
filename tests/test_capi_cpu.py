"""CPU-side checks of the C ABI: the library loads, exports every entry point the
header declares, and its host planner (no GPU involved) agrees with the oracle's
degree-of-freedom sets and rejects invalid meshes."""
import os
import re

import numpy as np
import pytest

from oracle import OracleMesh
from paper_1708_03912_gb300 import fraclap as F
from paper_1708_03912_gb300 import synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "fraclap.h")


def _lib_or_skip():
    if not os.path.exists(F.LIB_PATH):
        pytest.skip("libfraclap.so not built (run __graft_entry__.build())")
    return F.lib()


def test_header_declarations_are_exported():
    L = _lib_or_skip()
    text = open(HEADER).read()
    declared = set(re.findall(r"\b(fl_[a-z0-9_]+)\s*\(", text))
    declared = {d for d in declared if not d.endswith("_t")}
    assert declared, "no declarations parsed"
    for name in sorted(declared):
        assert hasattr(L, name), f"{name} declared in fraclap.h but not exported"
    assert set(F.EXPORTS) <= declared


@pytest.mark.parametrize("mesh", ["interval", "disc", "square", "lshape"])
def test_planner_dofs_match_oracle(mesh):
    _lib_or_skip()
    V, T = {"interval": synth.interval(20), "disc": synth.disc(6), "square": synth.square(5, 0.2),
            "lshape": synth.lshape(0.25, 0)}[mesh]
    for mode in ("interior", "paper"):
        h = F.fl_create(V, T, F.FL_DOF_PAPER if mode == "paper" else F.FL_DOF_INTERIOR)
        om = OracleMesh(V, T)
        for s in (0.3, 0.7):
            vod = F.fl_dof_vertices(h, s)
            ov, _ = om.dofs(s, mode)
            assert np.array_equal(vod, ov)
        F.fl_destroy(h)


def test_create_rejects_bad_input():
    _lib_or_skip()
    V, T = synth.square(2)
    with pytest.raises(F.FlError) as e:
        F.fl_create(V, np.array([[0, 1, 99]]))
    assert e.value.code == F.FL_EINVAL
    Vd = V.copy()
    with pytest.raises(F.FlError):
        F.fl_create(np.zeros((3, 2)), np.array([[0, 1, 2]]))  # degenerate
    # an edge shared by three triangles
    V3 = np.array([[0, 0], [1, 0], [0.5, 1], [0.5, -1], [0.5, 2.0]], dtype=float)
    with pytest.raises(F.FlError):
        F.fl_create(V3, np.array([[0, 1, 2], [0, 1, 3], [0, 4, 1]]))
    o = F.fl_default_options()
    o.k_far = 0
    with pytest.raises(F.FlError):
        F.fl_create(Vd, T, F.FL_DOF_INTERIOR, o)
    h = F.fl_create(V, T)
    with pytest.raises(F.FlError):
        F.fl_num_dofs(h, 1.0)
    F.fl_destroy(h)


def test_default_options():
    _lib_or_skip()
    o = F.fl_default_options()
    assert (o.k_far, o.k_near, o.k_touch, o.k_bnd, o.regional, o.k_vertex) == (4, 6, 8, 8, 0, 6)
    so = F.fl_default_solve_opts()
    assert so.tol == 1e-8 and so.inner_dtype == F.FL_F64


def test_prolongation_matches_oracle():
    _lib_or_skip()
    from oracle.multigrid import prolongation

    Vc, Tc = synth.square(3, 0.15)
    Vf, Tf = synth.bisect_all(Vc, Tc, 2)
    hc, hf = F.fl_create(Vc, Tc), F.fl_create(Vf, Tf)
    for s in (0.3, 0.8):
        ptr, col, val = F.fl_prolongation(hf, hc, s)
        n, nc = F.fl_num_dofs(hf, s), F.fl_num_dofs(hc, s)
        P = np.zeros((n, nc))
        for i in range(n):
            P[i, col[ptr[i]:ptr[i + 1]]] = val[ptr[i]:ptr[i + 1]]
        Po = prolongation(Vf, OracleMesh(Vf, Tf).dofs(s)[0], Vc, Tc, OracleMesh(Vc, Tc).dofs(s)[0])
        assert np.allclose(P, Po, rtol=0, atol=1e-14)
    # a point outside the coarse mesh is an error, not a silent zero row
    Vo, To = synth.square(2, 0.0, lo=0.0, hi=3.0)
    ho = F.fl_create(Vo, To)
    with pytest.raises(F.FlError):
        F.fl_prolongation(ho, hc, 0.5)
    for h in (hc, hf, ho):
        F.fl_destroy(h)


def test_patch_table_matches_oracle():
    _lib_or_skip()
    from oracle.mlp import patches

    for V, T in (synth.square(6, 0.2), synth.lshape(0.25, 0)):
        h = F.fl_create(V, T)
        for s in (0.4, 0.7):
            nbr, hl, hop = F.fl_patches(h, s, 12)
            on, oh, ohop = patches(OracleMesh(V, T), s, 12)
            assert np.array_equal(nbr, on)
            assert np.allclose(hl, oh, rtol=1e-13, atol=0)
            assert np.array_equal(hop, ohop)
        F.fl_destroy(h)


def test_pool_stats_without_device_work():
    # nothing has been allocated in a process without a GPU: the cache is empty
    st = F.fl_pool_stats()
    assert st["cached_device_bytes"] == 0 and st["cached_host_bytes"] == 0
    assert F.fl_pool_trim() == 0


def test_nearfield_csr_size_query_matches_oracle_pattern():
    # the size query of fl_assemble_nearfield_csr is host work only (planner); its nonzero
    # count equals the oracle's combinatorial near-field pattern
    _lib_or_skip()
    import ctypes

    from oracle.assemble import nearfield_pattern

    for (V, T), s in ((synth.disc(4), 0.6), (synth.interval(20), 0.3), (synth.lshape(0.25, 0), 0.5)):
        h = F.fl_create(V, T)
        nnz = ctypes.c_int64(-1)
        assert F.lib().fl_assemble_nearfield_csr(h, s, F.FL_FP64, ctypes.byref(nnz), None, None, None, None) == F.FL_OK
        assert nnz.value == int(nearfield_pattern(OracleMesh(V, T), s).sum())
        assert nnz.value == F.fl_get_stats(h, s)["nnz_nearfield"]
        assert F.lib().fl_assemble_nearfield_csr(h, s, F.FL_FP64, None, None, None, None, None) == F.FL_EINVAL
        F.fl_destroy(h)


def test_header_constants_match_binding():
    # every #define of include/fraclap.h that the binding mirrors has the same value there
    text = open(HEADER).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define (FL_[A-Z0-9_]+)\s+(-?\d+)", text, re.M)}
    mirrored = [k for k in defs if hasattr(F, k)]
    assert len(mirrored) >= 20
    for k in mirrored:
        assert getattr(F, k) == defs[k], k
    assert F.STAGES == ["prep", "far", "near", "touch", "bnd", "element", "compose"]
    assert len(F.STAGES) == defs["FL_NSTAGES"]


@pytest.mark.parametrize("mesh", ["interval", "disc", "square", "lshape"])
def test_planner_pair_classes_match_oracle(mesh):
    # the host planner's counts of unordered element pairs with a DOF on either side, by class
    # (touching, separated at vertex-graph distance 1, farther), equal the oracle's
    _lib_or_skip()
    V, T = {"interval": synth.interval(20), "disc": synth.disc(6), "square": synth.square(5, 0.2),
            "lshape": synth.lshape(0.25, 0)}[mesh]
    om = OracleMesh(V, T)
    for s in (0.3, 0.6):
        _, dov = om.dofs(s)
        has = (dov[om.C] >= 0).any(axis=1)
        counts = np.zeros(3, dtype=np.int64)
        for k in range(om.nc):
            shared, near = om.classify_cells(k)
            m = np.arange(k + 1, om.nc)
            m = m[has[k] | has[m]]
            counts += [(shared[m] > 0).sum(), ((shared[m] == 0) & near[m]).sum(), ((shared[m] == 0) & ~near[m]).sum()]
        h = F.fl_create(V, T)
        st = F.fl_get_stats(h, s)
        F.fl_destroy(h)
        assert (st["n_touch_pairs"], st["n_near_pairs"], st["n_far_pairs"]) == tuple(counts)
