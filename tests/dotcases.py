"""Seeded adversarial vector pairs for exact-dot tests (inputs only, no dot arithmetic)."""
import numpy as np


def _rand_wide(rng, n, emin, emax):
    m = rng.uniform(0.5, 1.0, n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    return np.ldexp(m, rng.integers(emin, emax + 1, n))


def cases(seed: int = 0):
    """List of (name, a, b) float64 vector pairs."""
    rng = np.random.default_rng(seed)
    out = []
    out.append(("empty", np.zeros(0), np.zeros(0)))
    out.append(("single", np.array([3.0]), np.array([-0.5])))
    out.append(("cancel_1e300", np.array([1e300, -1e300, 1.0]), np.array([1.0, 1.0, 1.0])))
    out.append(("cancel_huge_tiny", np.array([1e300, 1e-300, -1e300]), np.array([1e7, 1e-7, 1e7])))
    # 1 + 2^-53 is a tie between 1 and 1+2^-52: rounds to even (1.0)
    out.append(("tie_even_down", np.array([1.0, 2.0 ** -53]), np.array([1.0, 1.0])))
    # 1 + 3*2^-53 ties between 1+2^-52 and 1+2^-51: rounds to even (1+2^-51)
    out.append(("tie_even_up", np.array([1.0, 3 * 2.0 ** -53]), np.array([1.0, 1.0])))
    # just above the tie: rounds up
    out.append(("above_tie", np.array([1.0, 2.0 ** -53, 2.0 ** -200]), np.array([1.0, 1.0, 1.0])))
    out.append(("subnormal_products", np.array([2.0 ** -540, 3 * 2.0 ** -541, -2.0 ** -537]),
                np.array([2.0 ** -540 * 1.25, 2.0 ** -539, 2.0 ** -545])))
    out.append(("subnormal_operands", np.array([5e-324, 1e-310, -2.5e-320]), np.array([1.0, 3.0, 7.0])))
    out.append(("below_min_subnormal", np.array([2.0 ** -1074]), np.array([0.25])))
    out.append(("tie_at_min_subnormal", np.array([2.0 ** -1074]), np.array([0.5])))
    out.append(("neg_tiny_to_zero", np.array([-(2.0 ** -1074)]), np.array([0.25])))
    out.append(("overflow", np.array([1e300, 1e300]), np.array([1e10, 1e10])))
    out.append(("near_max", np.array([1.7976931348623157e308, -1.7976931348623157e308, 1.0]),
                np.array([1.0, 1.0, 1.0])))
    out.append(("zero_sum", np.array([1.5, -1.5, 2.0 ** -1074, -(2.0 ** -1074)]), np.ones(4)))
    out.append(("signed_zeros", np.array([-0.0, 0.0, -0.0]), np.array([1.0, -1.0, -2.0])))
    # TwoProd error term underflows: products near 2^-1000 with full mantissas
    a = _rand_wide(rng, 64, -520, -490)
    b = _rand_wide(rng, 64, -520, -490)
    out.append(("twoprod_underflow", a, b))
    # wide dynamic range with heavy cancellation
    a = _rand_wide(rng, 257, -300, 300)
    b = _rand_wide(rng, 257, -300, 300)
    a = np.concatenate([a, -a, rng.standard_normal(31)])
    b = np.concatenate([b, b, rng.standard_normal(31)])
    out.append(("wide_cancel", a, b))
    # everything range
    a = _rand_wide(rng, 500, -1074 + 60, 1000)
    b = _rand_wide(rng, 500, -1000, 15)
    out.append(("full_range", a, b))
    # ill-conditioned: sum of large alternating terms with a small remainder
    big = rng.standard_normal(200) * 1e20
    a = np.concatenate([big, -big[::-1], [1e-5, 3.0]])
    b = np.concatenate([np.ones(200), np.ones(200), [1.0, 1.0]])
    perm = rng.permutation(a.size)
    out.append(("ill_conditioned", a[perm], b[perm]))
    # ordinary Krylov-like vectors
    out.append(("gaussian_1000", rng.standard_normal(1000), rng.standard_normal(1000)))
    return out
