"""Property-based pins of the oracle (CPU; Hypothesis draws the inputs).

Every drawn case is checked against plain rational arithmetic:
- the exact dot is RN(sum a_i b_i), the correctly rounded real sum, for any
  finite doubles (subnormals, signed zeros, cancellation, overflow to inf);
- the plain dot is the sequential fma chain s = fma(a_i, b_i, s);
- the SpMV of a random CSR matrix is each row's fma chain in stored order.
Rationals carry no sign of zero, so a zero result is compared by value (an
IEEE fma that rounds a tiny negative sum to zero gives -0.0 where the
rational reference gives +0.0); every nonzero result is compared bit for bit.
"""
import math

import numpy as np
import pytest

from tests.fracref import exact_dot, fma_dot, fma_spmv, rn

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

finite = st.floats(allow_nan=False, allow_infinity=False, width=64)
# doubles whose products stay inside the double range, with wide exponents
scaled = st.builds(lambda m, e: math.ldexp(m, e), st.floats(-1.0, 1.0, allow_nan=False), st.integers(-1100, 500))

pairs = st.integers(0, 24).flatmap(lambda n: st.tuples(st.lists(finite, min_size=n, max_size=n),
                                                          st.lists(finite, min_size=n, max_size=n)))
scaled_pairs = st.integers(1, 40).flatmap(lambda n: st.tuples(st.lists(scaled, min_size=n, max_size=n),
                                                                 st.lists(scaled, min_size=n, max_size=n)))


def same(x, y):
    if x == 0.0 and y == 0.0:
        return True
    return np.array([x]).view(np.int64)[0] == np.array([y]).view(np.int64)[0]


@settings(max_examples=300, deadline=None, derandomize=True)
@given(pairs)
def test_fuzz_exact_dot_any_finite(orc, ab):
    a, b = (np.array(v, dtype=np.float64) for v in ab)
    want = rn(exact_dot(a, b))
    got = orc.dot_exact(a, b)
    if math.isinf(want):
        assert got == want
    elif want == 0.0:
        assert got == 0.0
    else:
        assert same(got, want), (got, want)


@settings(max_examples=300, deadline=None, derandomize=True)
@given(scaled_pairs)
def test_fuzz_exact_dot_wide_range(orc, ab):
    a, b = (np.array(v, dtype=np.float64) for v in ab)
    a = np.concatenate([a, -a[::2]])            # forced cancellation
    b = np.concatenate([b, b[::2]])
    want = rn(exact_dot(a, b))
    got = orc.dot_exact(a, b)
    assert got == want or (want == 0.0 and got == 0.0), (got, want)


@settings(max_examples=200, deadline=None, derandomize=True)
@given(scaled_pairs)
def test_fuzz_plain_dot_is_fma_chain(orc, ab):
    a, b = (np.array(v, dtype=np.float64) for v in ab)
    assert same(orc.dot_plain(a, b), fma_dot(a, b))


@st.composite
def small_csr(draw):
    n = draw(st.integers(1, 12))
    rows, cols, vals = [0], [], []
    for _ in range(n):
        k = draw(st.integers(0, n))
        cs = sorted(draw(st.lists(st.integers(0, n - 1), min_size=k, max_size=k, unique=True)))
        cols += cs
        vals += [draw(scaled) for _ in cs]
        rows.append(len(cols))
    x = [draw(scaled) for _ in range(n)]
    return (np.array(rows, np.int32), np.array(cols, np.int32), np.array(vals, np.float64),
            np.array(x, np.float64))


@settings(max_examples=200, deadline=None, derandomize=True)
@given(small_csr())
def test_fuzz_spmv_is_row_fma_chain(orc, m):
    rp, ci, va, x = m
    got = orc.spmv(rp, ci, va, x)
    want = fma_spmv(rp, ci, va, x)
    assert all(same(g, w) for g, w in zip(got, want))


@st.composite
def tiny_dominant_system(draw):
    n = draw(st.integers(2, 5))
    A = np.array([[draw(st.integers(-4, 4)) for _ in range(n)] for _ in range(n)], dtype=np.int64)
    A += np.diag(np.abs(A).sum(axis=1) + draw(st.integers(1, 5)))
    b = np.array([draw(st.integers(-6, 6)) for _ in range(n)], dtype=np.int64)
    b[draw(st.integers(0, n - 1))] = draw(st.integers(1, 9))      # b != 0
    return A, b


@settings(max_examples=40, deadline=None, derandomize=True)
@given(tiny_dominant_system())
def test_fuzz_oracle_follows_rational_algorithms(orc, sysb):
    """Drawn diagonally dominant integer systems: in rational arithmetic
    Algorithms 1 and 2 give identical iterates and Algorithm 2's invariants
    hold; the FP64 oracle (both algorithms, exact dots) follows the rational
    residual norms and alpha, omega over the first two iterations (omega
    only while the rational q is nonzero: where the exact run reaches the
    solution, FP64 keeps a rounding-level residual and its own omega)."""
    from fractions import Fraction
    from tests import ratref
    A, b = sysb
    n = A.shape[0]
    Af = [[Fraction(int(a)) for a in row] for row in A]
    bf = [Fraction(int(v)) for v in b]
    bad = []
    p = ratref.pbicgstab(Af, bf, [Fraction(0)] * n, 2, check=lambda name, l, r: bad.append(name) if l != r else None)
    c = ratref.bicgstab(Af, bf, [Fraction(0)] * n, 2)
    assert not bad, set(bad)
    assert len(p) == len(c)
    for rp_, rc_ in zip(p, c):
        for key in ("x", "r", "alpha", "omega", "beta"):
            assert rp_[key] == rc_[key], key
    rp, ci, v = [0], [], []
    for i in range(n):
        for j in range(n):
            if A[i, j] != 0:
                ci.append(j)
                v.append(float(A[i, j]))
        rp.append(len(ci))
    rp, ci, v = np.array(rp, np.int32), np.array(ci, np.int32), np.array(v)
    normb = math.sqrt(float(ratref.dot(bf, bf)))
    for alg in (0, 1):
        res = orc.solve(rp, ci, v, b.astype(float), tol=1e-300, maxit=2, alg=alg, mode=orc.EXACT, trace=True)
        for i in range(min(len(c), res.iters)):
            r = c[i]["r"]
            want = math.sqrt(float(ratref.dot(r, r))) / normb
            got = res.history[i + 1]
            assert abs(got - want) <= 1e-9 * want + 1e-13, (alg, i, got, want)
            for col, key in ((0, "alpha"), (1, "omega")):
                if key == "omega" and c[i][key] == 0:
                    continue     # q = 0: the rational run ends here; FP64 keeps a rounding-level q
                w = float(c[i][key])
                assert abs(res.trace[i, col] - w) <= 1e-9 * abs(w) + 1e-300, (alg, i, key)


@st.composite
def small_csr_repeats(draw):
    """Rows whose columns repeat and come in any order: the stored order is the order of the fma chain."""
    n = draw(st.integers(1, 10))
    rows, cols, vals = [0], [], []
    for _ in range(n):
        k = draw(st.integers(0, 2 * n))
        cs = draw(st.lists(st.integers(0, n - 1), min_size=k, max_size=k))      # with repeats, unsorted
        cols += cs
        vals += [draw(scaled) for _ in cs]
        rows.append(len(cols))
    x = [draw(scaled) for _ in range(n)]
    return (np.array(rows, np.int32), np.array(cols, np.int32), np.array(vals, np.float64),
            np.array(x, np.float64))


@settings(max_examples=200, deadline=None, derandomize=True)
@given(small_csr_repeats())
def test_fuzz_spmv_repeated_unsorted_columns(orc, m):
    rp, ci, va, x = m
    got = orc.spmv(rp, ci, va, x)
    want = fma_spmv(rp, ci, va, x)
    assert all(same(g, w) for g, w in zip(got, want))


@st.composite
def split_diagonal_system(draw):
    """A dominant integer system whose diagonal entries are +-2^k, each stored
    as two parts at two places in its row: 5/8 of it first and 3/8 last.  The
    parts sum to d exactly, and neither alone is a power of two, so a
    diagonal taken from one entry cannot hide behind the exact power-of-two
    scaling invariance of the iteration.  With b and x0."""
    n = draw(st.integers(2, 6))
    off = np.array([[draw(st.integers(-3, 3)) if i != j else 0 for j in range(n)] for i in range(n)])
    k = [draw(st.integers(5, 8)) for _ in range(n)]
    sgn = [draw(st.sampled_from([-1, 1])) for _ in range(n)]
    d = np.array([s * 2.0 ** e for s, e in zip(sgn, k)])
    rp, ci, va = [0], [], []
    for i in range(n):
        ci.append(i)
        va.append(d[i] * 0.625)
        for j in range(n):
            if off[i, j] != 0:
                ci.append(j)
                va.append(float(off[i, j]))
        ci.append(i)
        va.append(d[i] * 0.375)
        rp.append(len(ci))
    b = np.array([float(draw(st.integers(-6, 6))) for _ in range(n)])
    b[0] = 5.0
    x0 = np.array([float(draw(st.integers(-2, 2))) for _ in range(n)])
    return np.array(rp, np.int32), np.array(ci, np.int32), np.array(va), d, b, x0


@settings(max_examples=30, deadline=None, derandomize=True)
@given(split_diagonal_system(), st.sampled_from([0, 1]))
def test_fuzz_jacobi_sums_a_split_diagonal(orc, sysd, alg):
    """Right Jacobi takes d_i as the sum of row i's stored diagonal entries.
    With d_i = +-2^k stored as two parts, every scaled entry v / d_col is
    exact, so the preconditioned solve must equal, bit for bit, the plain
    solve of the column-scaled matrix (each stored entry scaled on its own)
    from y0 = d x0, followed by x = y / d."""
    rp, ci, va, d, b, x0 = sysd
    vs = np.array([math.ldexp(abs(v), -int(math.log2(abs(d[c])))) * math.copysign(1.0, v) * math.copysign(1.0, d[c])
                   for v, c in zip(va, ci)])
    got = orc.solve(rp, ci, va, b, x0=x0, tol=1e-12, maxit=12, alg=alg, mode=orc.EXACT, jacobi=True)
    ref = orc.solve(rp, ci, vs, b, x0=x0 * d, tol=1e-12, maxit=12, alg=alg, mode=orc.EXACT)
    assert got.status == ref.status and got.iters == ref.iters
    assert np.array_equal(got.history.view(np.int64), ref.history.view(np.int64))
    assert np.array_equal(got.x.view(np.int64), (ref.x / d).view(np.int64))
