"""Pins of the low-precision oracle (oracle/lowprec.py): bfloat16 rounding,
Jacobi scaling, the two-slice split and the product the batched solver forms.
No GPU."""
import numpy as np
import pytest

from oracle import OracleMesh, assemble_matrix
from oracle.lowprec import abs_product, bf16_round, jacobi_scale, matmul_split, split_bf16, split_vec
from paper_1708_03912_gb300 import synth


def test_bf16_matches_library_conversion_from_float32():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    x = (rng.standard_normal(200000) * np.exp(rng.uniform(-40, 40, 200000))).astype(np.float32)
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(bf16_round(x.astype(np.float64)), ref)


def test_bf16_ties_and_single_rounding():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties go to the even significand (1)
    assert bf16_round(np.array([1 + 2.0 ** -8]))[0] == 1.0
    # 1 + 3 2^-8 lies halfway between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert bf16_round(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6
    # just above a tie rounds up; rounding through float32 first would give 1
    assert bf16_round(np.array([1 + 2.0 ** -8 + 2.0 ** -30]))[0] == 1 + 2.0 ** -7
    assert bf16_round(np.array([-(1 + 2.0 ** -8 + 2.0 ** -30)]))[0] == -(1 + 2.0 ** -7)
    with pytest.raises(ValueError):
        bf16_round(np.array([1e-40]))


def test_bf16_is_nearest_on_the_grid():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(5000) * 10.0 ** rng.uniform(-8, 8, 5000)
    r = bf16_round(x)
    m, e = np.frexp(x)
    ulp = np.ldexp(1.0, e - 8)  # spacing of bf16 values in the binade of x
    # r on the grid, within half a spacing, and no grid neighbour strictly closer
    assert np.all(np.abs(x - r) <= 0.5 * ulp)
    assert np.all(np.abs(r / ulp - np.rint(r / ulp)) == 0)
    assert np.all(np.abs(x - r) <= 2.0 ** -8 * np.abs(x))  # unit roundoff of 8 significant bits


def test_jacobi_scaling_and_split():
    V, T = synth.disc(5)
    A, _ = assemble_matrix(OracleMesh(V, T), 0.6)
    A = 0.5 * (A + A.T)  # the oracle's sums differ by rounding between a_ij and a_ji
    d, At = jacobi_scale(A)
    assert np.allclose(np.diag(At), 1.0, rtol=4e-16, atol=0)
    assert np.array_equal(At, At.T)
    assert np.all(np.linalg.eigvalsh(At) > 0)
    d2, S = split_bf16(A, 2)
    assert np.array_equal(d, d2)
    # the first difference is exact, the second slice rounds it
    assert np.array_equal(S[0] + (At - S[0]), At)
    assert np.all(np.abs(At - S[0]) <= 2.0 ** -8 * np.abs(At))
    assert np.all(np.abs(At - S[0] - S[1]) <= 2.0 ** -16 * np.abs(At))
    _, S1 = split_bf16(A, 1)
    assert len(S1) == 1 and np.array_equal(S1[0], S[0])


def test_vector_split():
    rng = np.random.default_rng(11)
    x = rng.standard_normal(1000).astype(np.float32)
    hi, lo = split_vec(x)
    # x - x_hi is exact in float32
    assert np.array_equal((hi.astype(np.float32) + (x - hi.astype(np.float32))), x)
    assert np.all(np.abs(x - hi - lo) <= 2.0 ** -16 * np.abs(x))


def test_product_bound_against_float64():
    V, T = synth.disc(5)
    A, _ = assemble_matrix(OracleMesh(V, T), 0.75)
    _, At = jacobi_scale(A)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((A.shape[0], 16)).astype(np.float32)
    for ns, bound in ((2, 4 * 2.0 ** -16), (1, 2.0 ** -8 + 2.0 ** -15)):
        _, S = split_bf16(A, ns)
        Y = matmul_split(S, X)
        E = At @ X.astype(np.float64)
        scale = abs_product([np.abs(At)], X)
        assert np.all(np.abs(Y - E) <= bound * scale)
    # with one slice the error is of order 2^-9 (not smaller): the split matters
    _, S = split_bf16(A, 1)
    assert np.max(np.abs(matmul_split(S, X) - At @ X.astype(np.float64)) / scale) > 2.0 ** -14


def test_f32x2_split_pins():
    # hi is the library's float32 rounding, hi + lo reproduces a to 2^-48 |a| (half an ulp of
    # the float32 remainder), values exact in float32 have lo = 0, signs and scales carry over
    from oracle.lowprec import f32x2_split, f32x2_product

    rng = np.random.default_rng(20170813)
    A = rng.standard_normal((40, 40)) * np.exp(rng.uniform(-20, 20, (40, 40)))
    hi, lo = f32x2_split(A)
    assert np.array_equal(hi, A.astype(np.float32))
    err = np.abs(A - (hi.astype(np.float64) + lo.astype(np.float64)))
    assert np.all(err <= 2.0 ** -48 * np.abs(A))
    assert np.all(np.abs(lo.astype(np.float64)) <= 2.0 ** -24 * np.abs(A))
    E = A.astype(np.float32).astype(np.float64)
    h2, l2 = f32x2_split(E)
    assert np.array_equal(h2.astype(np.float64), E) and not l2.any()
    x = rng.standard_normal(40)
    y = f32x2_product(hi, lo, x)
    assert np.all(np.abs(y - A @ x) <= 2.0 ** -46 * (np.abs(A) @ np.abs(x)))
