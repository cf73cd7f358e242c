"""Pins of the oracle's dot products and SpMV against exact rational arithmetic.

The exact dot must equal RN(sum a_i b_i), the correctly rounded real sum
(Section 2: the ExBLAS long accumulator delivers correctly rounded results).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from tests import dotcases
from tests.fracref import exact_dot, fma_dot, fma_spmv, fr, rn

CASES = dotcases.cases(0)


@pytest.mark.parametrize("name,a,b", CASES, ids=[c[0] for c in CASES])
def test_exact_dot_matches_fraction(orc, name, a, b):
    got = orc.dot_exact(a, b)
    want = rn(exact_dot(a, b))
    if math.isinf(want):
        assert got == want
    else:
        assert got == want, (name, got, want)
        if want == 0.0:
            # exact zero is +0; a nonzero tiny sum keeps its sign
            assert math.copysign(1.0, got) == math.copysign(1.0, want) or exact_dot(a, b) == 0


@pytest.mark.parametrize("name,a,b", CASES, ids=[c[0] for c in CASES])
def test_exact_fixed_integer(orc, name, a, b):
    """The big integer the oracle accumulates is the exact sum times 2^2148."""
    N = orc.dot_exact_fixed(a, b)
    assert Fraction(N, 2 ** orc.SCALE) == exact_dot(a, b)
    # the oracle's rounding routine agrees with correctly rounded division
    want = rn(Fraction(N, 2 ** orc.SCALE))
    assert orc.round_fixed(N) == want


def test_exact_zero_is_positive(orc):
    got = orc.dot_exact([1.5, -1.5], [1.0, 1.0])
    assert got == 0.0 and math.copysign(1.0, got) == 1.0
    got = orc.dot_exact([-0.0], [1.0])
    assert math.copysign(1.0, got) == 1.0


def test_negative_tiny_rounds_to_negative_zero(orc):
    got = orc.dot_exact([-(2.0 ** -1074)], [0.25])
    assert got == 0.0 and math.copysign(1.0, got) == -1.0


def test_fsum_of_twoprod(orc):
    """Normal-range products: the exact dot equals math.fsum (Shewchuk, correctly
    rounded) of the TwoProd pairs (p, e) with p + e = a*b exactly."""
    rng = np.random.default_rng(1)
    for trial in range(20):
        n = int(rng.integers(1, 300))
        a = rng.standard_normal(n) * np.ldexp(1.0, rng.integers(-60, 60, n))
        b = rng.standard_normal(n) * np.ldexp(1.0, rng.integers(-60, 60, n))
        terms = []
        for x, y in zip(a, b):
            p = float(x) * float(y)
            e = float(fr(x) * fr(y) - fr(p))   # exact: representable in normal range
            assert fr(p) + fr(e) == fr(x) * fr(y)
            terms += [p, e]
        assert orc.dot_exact(a, b) == math.fsum(terms)


def test_closed_forms(orc):
    # sum of distinct powers of two over a wide range is exact when it fits 53 bits
    k = np.arange(0, 53)
    a = np.ldexp(1.0, k - 30)
    assert orc.dot_exact(a, np.ones_like(a)) == float(sum(Fraction(2) ** int(e) for e in (k - 30)))
    # x . (+1,-1,+1,...) telescopes for x = (c, c, c, ...)
    c = np.full(1001, 0.1)
    sgn = np.where(np.arange(1001) % 2 == 0, 1.0, -1.0)
    assert orc.dot_exact(c, sgn) == 0.1
    # 2^k * 2^-k = 1 summed n times
    e = np.arange(-500, 500)
    assert orc.dot_exact(np.ldexp(1.0, e), np.ldexp(1.0, -e)) == float(e.size)
    # 1e300 - 1e300 + 1
    assert orc.dot_exact([1e300, -1e300, 1.0], [1.0, 1.0, 1.0]) == 1.0


def test_nonfinite_and_overflow(orc):
    assert math.isnan(orc.dot_exact([1.0, np.nan], [1.0, 1.0]))
    assert math.isnan(orc.dot_exact([1.0, np.inf], [1.0, 0.0]))
    assert orc.dot_exact([1e300, 1e300], [1e10, 1e10]) == math.inf
    assert orc.dot_exact([-1e300, -1e300], [1e10, 1e10]) == -math.inf
    assert orc.dot_exact_fixed([np.nan], [1.0]) is None


def test_permutation_and_split_invariance(orc):
    """Exact dots do not depend on order or partitioning (Section 2, Tables 2-3):
    P-way partial integers summed and rounded once give the same double."""
    for name, a, b in CASES:
        if a.size < 2:
            continue
        rng = np.random.default_rng(7)
        want = orc.dot_exact(a, b)
        perm = rng.permutation(a.size)
        got = orc.dot_exact(a[perm], b[perm])
        assert got == want or (math.isnan(got) and math.isnan(want))
        if orc.dot_exact_fixed(a, b) is None:
            continue
        for P in (2, 3, 7):
            cuts = np.linspace(0, a.size, P + 1).astype(int)
            N = sum(orc.dot_exact_fixed(a[cuts[i]:cuts[i + 1]], b[cuts[i]:cuts[i + 1]]) for i in range(P))
            assert orc.round_fixed(N) == want


def test_threaded_exact_equals_sequential(orc):
    rng = np.random.default_rng(3)
    a = rng.standard_normal(300_000) * np.ldexp(1.0, rng.integers(-200, 200, 300_000))
    b = rng.standard_normal(300_000)
    s1 = orc.dot_exact(a, b, nthreads=1)
    for t in (2, 5, 8):
        assert orc.dot_exact(a, b, nthreads=t) == s1


def test_plain_dot_is_sequential_fma(orc):
    rng = np.random.default_rng(4)
    for n in (0, 1, 2, 17, 100):
        a = rng.standard_normal(n)
        b = rng.standard_normal(n) * 1e3
        assert orc.dot_plain(a, b) == fma_dot(a, b)


def test_plain_dot_differs_from_naive_when_it_should(orc):
    # fma keeps the product exact before the add: (1+2^-30)^2 - (1+2^-29)
    a = np.array([1.0 + 2.0 ** -30, 1.0])
    b = np.array([1.0 + 2.0 ** -30, -(1.0 + 2.0 ** -29)])
    # sequential: s = fma(a0,b0,0) = RN((1+2^-30)^2); s = fma(1, -(1+2^-29), s)
    assert orc.dot_plain(a, b) == fma_dot(a, b)
    assert orc.dot_exact(a, b) == 2.0 ** -60


def test_spmv_fixed_fma_order(orc):
    rng = np.random.default_rng(5)
    n = 40
    rows = []
    for i in range(n):
        k = int(rng.integers(0, 9))
        cols = np.sort(rng.choice(n, size=k, replace=False))
        rows.append(cols)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    col_idx = np.concatenate(rows).astype(np.int32) if row_ptr[-1] else np.zeros(0, np.int32)
    vals = rng.standard_normal(row_ptr[-1]) * np.ldexp(1.0, rng.integers(-20, 20, row_ptr[-1]))
    x = rng.standard_normal(n)
    got = orc.spmv(row_ptr, col_idx, vals, x)
    want = fma_spmv(row_ptr, col_idx, vals, x)
    assert np.array_equal(got, np.array(want))
    # integer data: every fma is exact, so y equals the integer product
    vi = rng.integers(-5, 6, row_ptr[-1]).astype(np.float64)
    xi = rng.integers(-5, 6, n).astype(np.float64)
    yi = orc.spmv(row_ptr, col_idx, vi, xi)
    dense = np.zeros((n, n))
    for i in range(n):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            dense[i, col_idx[k]] += vi[k]
    assert np.array_equal(yi, dense @ xi)
