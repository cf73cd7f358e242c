"""Exact rational references used to pin the oracle (tests only).

Everything here is plain Python ``fractions.Fraction`` arithmetic; a double is
converted exactly with ``Fraction(float)`` and a rational is rounded to the
nearest double (ties to even) by ``float(Fraction)``, which Python computes by
correctly rounded integer division.
"""
from fractions import Fraction
import math


def fr(x) -> Fraction:
    return Fraction(float(x))


def rn(q: Fraction) -> float:
    """Round a rational to the nearest double, ties to even (overflow -> inf)."""
    try:
        return float(q)
    except OverflowError:
        return math.inf if q > 0 else -math.inf


def exact_dot(a, b) -> Fraction:
    s = Fraction(0)
    for x, y in zip(a, b):
        s += fr(x) * fr(y)
    return s


def fma(a, b, c) -> float:
    """Single-rounding fused multiply-add from its definition."""
    return rn(fr(a) * fr(b) + fr(c))


def fma_dot(a, b) -> float:
    s = 0.0
    for x, y in zip(a, b):
        s = fma(x, y, s)
    return s


def fma_spmv(row_ptr, col_idx, vals, x):
    n = len(row_ptr) - 1
    y = []
    for i in range(n):
        acc = 0.0
        for k in range(row_ptr[i], row_ptr[i + 1]):
            acc = fma(vals[k], x[col_idx[k]], acc)
        y.append(acc)
    return y
