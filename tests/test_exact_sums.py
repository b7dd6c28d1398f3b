"""The exactness test behind the IVF list means (Sec. 2.2 centroid update), checked on the CPU
with exact rational arithmetic: when every element of a float32 column is a multiple of
2^(e - 150) (e the smallest biased exponent among its nonzero elements, subnormals counted as 1)
and the column's sum of magnitudes is below 2^(e - 97), every partial sum of the row-order FP64
accumulation is exact, so that accumulation equals the exact sum.  The kernels use this to
replace the FP64 chain by an exact integer sum; the test plants columns on both sides of the
bound."""
from fractions import Fraction

import numpy as np
import pytest


def min_exponent(col):
    b = col.view(np.uint32)
    nz = (b & 0x7FFFFFFF) != 0
    if not nz.any():
        return None
    return int(np.maximum((b[nz] >> 23) & 0xFF, 1).min())


def bound_holds(col):
    e = min_exponent(col)
    if e is None:
        return True
    sabs = float(np.sum(np.abs(col.astype(np.float64))))
    return sabs * (1.0 + 1.2e-7 * len(col)) < 2.0 ** (e - 97)


def row_order_fp64(col):
    s = 0.0
    for v in col.astype(np.float64):
        s = s + v
    return s


@pytest.mark.parametrize("seed", range(6))
def test_row_order_sum_is_exact_under_the_bound(seed):
    rng = np.random.default_rng(900 + seed)
    hits = 0
    for trial in range(60):
        n = int(rng.integers(1, 3000))
        scale = float(rng.choice([1e-3, 1.0, 40.0, 255.0]))
        col = (rng.standard_normal(n) * scale).astype(np.float32)
        if trial % 3 == 1:
            col = np.rint(col).astype(np.float32)  # integer-valued, like the 0..255 data
        if trial % 3 == 2:
            col[rng.random(n) < 0.01] *= np.float32(1e-9)  # a few values far below the others' ulp
        if not bound_holds(col):
            continue
        hits += 1
        exact = sum((Fraction(float(v)) for v in col), Fraction(0))
        assert Fraction(row_order_fp64(col)) == exact
    assert hits > 10


def test_bound_rejects_columns_whose_fp64_chain_rounds():
    # 2^30 ones after one 2^-24: the bound fails, and indeed the chain loses the small term
    col = np.array([2.0 ** -24] + [2.0 ** 30] * 4, dtype=np.float32)
    assert not bound_holds(col)
    exact = sum((Fraction(float(v)) for v in col), Fraction(0))
    assert Fraction(row_order_fp64(col)) != exact
