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
