"""Host refinement of the adaptive loop (fl_refine, newest-vertex bisection with closure,
Section 7) against the oracle's refinement: the same vertices, cells and numbering."""
import numpy as np
import pytest

from oracle.adaptive import refine
from paper_1708_03912_gb300 import fraclap as fl
from paper_1708_03912_gb300 import synth


def _lib_or_skip():
    try:
        fl.lib()
    except OSError as e:  # the library is built by __graft_entry__.build()
        pytest.skip(f"library not built: {e}")


@pytest.mark.parametrize("case", ["lshape", "disc", "square", "all", "none"])
def test_refine_matches_oracle(case):
    _lib_or_skip()
    rng = np.random.default_rng(11)
    if case == "lshape":
        V, T = synth.lshape(levels=2)
    elif case == "disc":
        V, T = synth.disc(6, 2.0)
    else:
        V, T = synth.square(6, jitter=0.1)
    marks = {"all": np.ones(len(T), bool), "none": np.zeros(len(T), bool)}.get(case, rng.random(len(T)) < 0.15)
    V1, T1 = fl.fl_refine(V, T, marks.astype(np.uint8))
    V2, T2 = refine(V, T, marks)
    assert np.array_equal(T1, T2.astype(np.int32))
    assert np.array_equal(V1, V2)
    # several rounds in a row stay equal (the children's refinement edges are the new ones)
    for _ in range(3):
        marks = rng.random(len(T1)) < 0.2
        V1, T1 = fl.fl_refine(V1, T1, marks.astype(np.uint8))
        V2, T2 = refine(V2, T2, marks)
        assert np.array_equal(T1, T2.astype(np.int32)) and np.array_equal(V1, V2)


def test_refine_1d_and_errors():
    _lib_or_skip()
    V, T = synth.graded_interval(10, 2.0)
    marks = np.zeros(len(T), np.uint8)
    marks[[0, 3, 9]] = 1
    V1, T1 = fl.fl_refine(V, T, marks)
    V2, T2 = refine(V, T, marks.astype(bool))
    assert np.array_equal(T1, T2.astype(np.int32)) and np.array_equal(V1, V2)
    # dim 3 and NULL arrays are rejected
    assert fl.lib().fl_refine(3, 4, None, 1, None, None, 0, 0, None, None, None, None) == fl.FL_EINVAL
    # out-of-range vertex index
    bad = np.array(T, dtype=np.int32).copy()
    bad[0, 0] = len(V) + 5
    with pytest.raises(fl.FlError):
        fl.fl_refine(V, bad, marks)


def test_refine_capacity_reports_sizes():
    _lib_or_skip()
    import ctypes

    V, T = synth.disc(3)
    V = np.ascontiguousarray(V)
    C = np.ascontiguousarray(T, dtype=np.int32)
    M = np.ones(len(C), np.uint8)
    nv, nc = ctypes.c_int64(), ctypes.c_int64()
    Vo = np.empty((len(V), 2))
    Co = np.empty((len(C), 3), np.int32)
    r = fl.lib().fl_refine(2, len(V), V.ctypes.data, len(C), C.ctypes.data, M.ctypes.data, len(V), len(C),
                           Vo.ctypes.data, Co.ctypes.data, ctypes.byref(nv), ctypes.byref(nc))
    assert r == fl.FL_EINVAL
    V2, T2 = refine(V, T, M.astype(bool))
    assert (nv.value, nc.value) == (len(V2), len(T2))
    assert b"capacity" in fl.lib().fl_last_error(None)
