"""The exact slice-product scheme of the fit's Gram matrix (Eq. 63a normal
equations), checked in exact rational arithmetic on the CPU: the column slicing
the tensor-core kernels use (eight 8-bit slices on a grid set by the column's
largest magnitude, slice pairs with s + t < 8) reproduces A^T A to within
R 2^(e_m + e_n - 59), and every 256-row partial sum of a slice product is an
integer below 2^24 (so an FP32 accumulator holds it exactly).  This pins the
argument the kernels rely on; the kernels themselves are compared with the FP64
SYRK on the GPU."""
import math
from fractions import Fraction

import numpy as np


def _exponent(col):
    """Smallest integer e with max |a| < 2^e (0 for an all-zero column)."""
    mx = max(abs(float(a)) for a in col)
    if mx == 0.0:
        return 0
    m, e = math.frexp(mx)  # mx = m 2^e, m in [0.5, 1)
    return e


def _slices(a, e):
    """Signed 8-bit slices v_0..v_7 of a on the grid 2^(e - 64): X = floor(|a| 2^(64 - e))."""
    X = math.floor(abs(Fraction(float(a))) * Fraction(2) ** (64 - e))
    assert 0 <= X < 2 ** 64
    sign = -1 if a < 0 else 1
    return [sign * ((X >> (56 - 8 * s)) & 0xFF) for s in range(8)]


def test_slice_products_reproduce_gram():
    g = np.random.default_rng(20221229)
    R, M = 48, 6
    scales = 10.0 ** g.uniform(-6, 4, size=M)
    A = g.normal(size=(R, M)) * scales
    A[3, 2] = 0.0
    A[:, 5] = 0.0  # an all-zero column
    A[7, 1] = -A[7, 1]
    ex = [_exponent(A[:, m]) for m in range(M)]
    V = [[_slices(A[r, m], ex[m]) for m in range(M)] for r in range(R)]  # V[r][m][s]
    pairs = [(s, t) for s in range(8) for t in range(8) if s + t < 8]
    for m in range(M):
        for n in range(M):
            est = Fraction(0)
            for s, t in pairs:
                P = sum(V[r][m][s] * V[r][n][t] for r in range(R))
                est += Fraction(P) * Fraction(2) ** (ex[m] + ex[n] - 8 * (s + t + 2))
            exact = sum(Fraction(float(A[r, m])) * Fraction(float(A[r, n])) for r in range(R))
            assert abs(est - exact) <= R * Fraction(2) ** (ex[m] + ex[n] - 59)
            if m == 5 or n == 5:
                assert est == 0


def test_chunk_sums_fit_fp32_exactly():
    # |v_s| <= 255, so a 256-row sum of slice products stays below 2^24
    assert 256 * 255 * 255 < 2 ** 24
    # a block's int32 sums (at most 32,768 rows) stay below 2^31
    assert 32768 * 255 * 255 < 2 ** 31
