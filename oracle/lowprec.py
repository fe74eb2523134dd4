"""Low-precision copies of the stiffness matrix and the products formed with them
(oracle; test infrastructure only).

The batched solver keeps the float64 matrix A as the reference for the residual and
iterates on a Jacobi-scaled copy in bfloat16.  What that copy and its product
are, written out from their definitions:

* bfloat16 is the IEEE-style format with 8 exponent bits and 8 significant bits
  (7 stored); rounding is to nearest, ties to the even significand.
* Jacobi scaling: D = diag(A)^{-1/2}, Ã = D A D (unit diagonal), formed entry by
  entry as (d_i d_j) a_ij in float64, which keeps Ã exactly symmetric.
* Slices: S_0 = bf16(Ã) and, with two slices, S_1 = bf16(Ã - S_0); the
  difference Ã - S_0 is exact in float64.
* A float32 vector x is carried as x_hi = bf16(x), x_lo = bf16(x - x_hi)
  (x - x_hi exact in float32).
* The product the tensor cores form is S_0 (x_hi + x_lo) + S_1 x_hi: every
  slice/vector pair except the smallest, S_1 x_lo.

* Hi + lo float32 storage (the 8-byte matrix the float32 pipe multiplies):
  hi = fl32(a), lo = fl32(a - hi).

Parity status: pinned in ``tests/test_oracle_lowprec.py`` against the
float32 -> bfloat16 conversion of PyTorch (a library routine), against tie
cases constructed from the definition, and against the float64 product within
the stated bound.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x):
    """Round float64 (or float32) values to the nearest bfloat16, ties to even,
    directly from the given precision (a single rounding).  Returned as float64.
    Values must be zero or of magnitude in [2^-126, 2^128) (normal float32 range)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)            # x = m 2^e, 0.5 <= |m| < 1
    nz = x != 0
    ax = np.abs(x[nz])
    if ax.size and (ax.min() < 2.0 ** -126 or ax.max() >= 2.0 ** 128):
        raise ValueError("bf16_round: value outside the normal range")
    # 8 significant bits: |m| 2^8 in [128, 256); round half to even
    r = np.rint(np.ldexp(m, 8))
    return np.ldexp(r, e - 8)


def jacobi_scale(A):
    """d = diag(A)^{-1/2} and Ã_ij = (d_i d_j) a_ij."""
    A = np.asarray(A, dtype=np.float64)
    d = 1.0 / np.sqrt(np.diag(A))
    At = np.outer(d, d) * A
    return d, At


def split_bf16(A, nslices=2):
    """(d, [S_0, S_1][:nslices]) for the Jacobi-scaled matrix, slices as float64."""
    d, At = jacobi_scale(A)
    S0 = bf16_round(At)
    S = [S0]
    if nslices == 2:
        S.append(bf16_round(At - S0))
    return d, S


def split_vec(x):
    """(x_hi, x_lo) of a float32 array, returned as float64."""
    x = np.asarray(x, dtype=np.float32)
    hi = bf16_round(x.astype(np.float64))
    lo = bf16_round((x - hi.astype(np.float32)).astype(np.float64))
    return hi, lo


def matmul_split(S, X):
    """Y = S_0 (X_hi + X_lo) + S_1 X_hi for float32 X of shape (n, nrhs), in float64."""
    hi, lo = split_vec(X)
    Y = S[0] @ (hi + lo)
    if len(S) > 1:
        Y = Y + S[1] @ hi
    return Y


def abs_product(S, X):
    """|S_0| |X| + |S_1| |X|: the scale of the rounding error of matmul_split."""
    Xa = np.abs(np.asarray(X, dtype=np.float64))
    Y = np.abs(S[0]) @ Xa
    if len(S) > 1:
        Y = Y + np.abs(S[1]) @ Xa
    return Y


def f32x2_split(A):
    """Hi + lo float32 storage of a float64 matrix: hi = fl32(a) (round to nearest even),
    lo = fl32(a - hi) (a - hi is exact in float64).  Returns (hi, lo) as float32 arrays;
    hi + lo equals a to within 2^-48 |a| (for a in the normal float32 range)."""
    A = np.asarray(A, dtype=np.float64)
    hi = A.astype(np.float32)
    lo = (A - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def f32x2_product(hi, lo, x):
    """The product the hi + lo storage represents, (hi + lo) x, in float64."""
    return (hi.astype(np.float64) + lo.astype(np.float64)) @ np.asarray(x, dtype=np.float64)
