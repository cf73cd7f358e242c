"""Algorithms 1 and 2 of arXiv 2404.13216 in exact rational arithmetic (tests only).

Used on tiny systems to pin the FP64 oracle: in exact arithmetic the two
algorithms produce identical iterates (Section 2 calls them mathematically
equivalent), Algorithm 2's auxiliary vectors satisfy w = A r, s = A p, z = A s,
t = A w, v = A z, y = A q, and both terminate with r = 0 in at most n steps.
The tests check these facts on the rational runs, then compare the FP64
oracle with them.
"""
from fractions import Fraction


def matvec(A, x):
    return [sum((A[i][j] * x[j] for j in range(len(x))), Fraction(0)) for i in range(len(A))]


def dot(a, b):
    return sum((x * y for x, y in zip(a, b)), Fraction(0))


def axpy(alpha, x, y):
    return [alpha * a + b for a, b in zip(x, y)]


def sub(x, y):
    return [a - b for a, b in zip(x, y)]


def bicgstab(A, b, x0, maxit):
    """Algorithm 1.  Returns per-iteration records (x_{i+1}, r_{i+1}, alpha_i, omega_i, beta_i)."""
    x = list(x0)
    r0 = sub(b, matvec(A, x))
    r = list(r0)
    p = list(r0)
    out = []
    for i in range(maxit):
        s = matvec(A, p)
        alpha = dot(r0, r) / dot(r0, s)
        q = axpy(-alpha, s, r)
        y = matvec(A, q)
        yy = dot(y, y)
        omega = dot(q, y) / yy if yy != 0 else Fraction(0)
        x = [xi + alpha * pi + omega * qi for xi, pi, qi in zip(x, p, q)]
        r_new = axpy(-omega, y, q)
        rec = {"x": x, "r": r_new, "alpha": alpha, "omega": omega, "beta": None}
        out.append(rec)
        if all(v == 0 for v in r_new) or omega == 0:
            break
        beta = (alpha / omega) * (dot(r0, r_new) / dot(r0, r))
        rec["beta"] = beta
        p = [rn + beta * (pi - omega * si) for rn, pi, si in zip(r_new, p, s)]
        r = r_new
    return out


def pbicgstab(A, b, x0, maxit, check=None):
    """Algorithm 2.  Same records as bicgstab(); ``check(name, lhs, rhs)`` is
    called for every auxiliary-vector invariant at every iteration."""
    x = list(x0)
    r0 = sub(b, matvec(A, x))
    r = list(r0)
    w = matvec(A, r0)
    t = matvec(A, w)
    alpha = dot(r0, r0) / dot(r0, w)
    beta = Fraction(0)
    omega = Fraction(0)
    p = s = z = v = None
    out = []
    for i in range(maxit):
        if i == 0:
            p, s, z = list(r), list(w), list(t)
        else:
            p = [ri + beta * (pi - omega * si) for ri, pi, si in zip(r, p, s)]
            s = [wi + beta * (si - omega * zi) for wi, si, zi in zip(w, s, z)]
            z = [ti + beta * (zi - omega * vi) for ti, zi, vi in zip(t, z, v)]
        q = axpy(-alpha, s, r)
        y = axpy(-alpha, z, w)
        v = matvec(A, z)
        if check:
            check("w=Ar", w, matvec(A, r))
            check("s=Ap", s, matvec(A, p))
            check("z=As", z, matvec(A, s))
            check("t=Aw", t, matvec(A, w))
            check("v=Az", v, matvec(A, z))
            check("y=Aq", y, matvec(A, q))
        yy = dot(y, y)
        omega = dot(q, y) / yy if yy != 0 else Fraction(0)
        x = [xi + alpha * pi + omega * qi for xi, pi, qi in zip(x, p, q)]
        r_new = axpy(-omega, y, q)
        w = [yi - omega * (ti - alpha * vi) for yi, ti, vi in zip(y, t, v)]
        t = matvec(A, w)
        rec = {"x": x, "r": r_new, "alpha": alpha, "omega": omega, "beta": None}
        out.append(rec)
        if all(val == 0 for val in r_new) or omega == 0:
            break
        beta = (alpha / omega) * (dot(r0, r_new) / dot(r0, r))
        rec["beta"] = beta
        alpha = dot(r0, r_new) / (dot(r0, w) + beta * dot(r0, s) - beta * omega * dot(r0, z))
        r = r_new
    return out
