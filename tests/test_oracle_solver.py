"""Pins of the FP64 oracle's BiCGStab (Algorithm 1) and p-BiCGStab (Algorithm 2).

Chain of evidence: the rational transcriptions in ``ratref`` are checked
against facts exact arithmetic fixes (Algorithm 2's invariants, equality of the
two algorithms' iterates, finite termination); the FP64 oracle is then checked
against them, and against closed-form and invariance properties.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2404_13216_gb300 import inputs
from tests import ratref


def tiny_system(seed, n):
    """Integer, diagonally dominant, unsymmetric: well-conditioned and breakdown-free."""
    rng = np.random.default_rng(seed)
    A = rng.integers(-3, 4, (n, n)).astype(np.int64)
    A += np.diag(np.abs(A).sum(axis=1) + rng.integers(1, 4, n))
    b = rng.integers(-5, 6, n)
    b[0] = 7
    return A, b


def dense_to_csr(A):
    n = A.shape[0]
    rp, ci, v = [0], [], []
    for i in range(n):
        for j in range(n):
            if A[i, j] != 0:
                ci.append(j)
                v.append(float(A[i, j]))
        rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32), np.array(v)


def frac_mat(A):
    return [[Fraction(int(a)) for a in row] for row in A]


@pytest.mark.parametrize("seed", range(6))
def test_rational_invariants_equivalence_termination(seed):
    n = 3 + seed % 4
    A, b = tiny_system(seed, n)
    Af, bf = frac_mat(A), [Fraction(int(v)) for v in b]
    x0 = [Fraction(0)] * n
    bad = []

    def check(name, lhs, rhs):
        if lhs != rhs:
            bad.append(name)

    p = ratref.pbicgstab(Af, bf, x0, n + 2, check=check)
    c = ratref.bicgstab(Af, bf, x0, n + 2)
    assert not bad, f"Algorithm 2 invariant broken: {set(bad)}"
    # identical iterates in exact arithmetic
    assert len(p) == len(c)
    for rp_, rc_ in zip(p, c):
        for key in ("x", "r", "alpha", "omega", "beta"):
            assert rp_[key] == rc_[key], key
        # r_{i+1} = b - A x_{i+1}
        assert rp_["r"] == ratref.sub(bf, ratref.matvec(Af, rp_["x"]))
    # terminates with the exact solution within n steps
    assert len(p) <= n
    assert all(v == 0 for v in p[-1]["r"])


@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_fp64_oracle_follows_rational(orc, alg, seed):
    n = 6
    A, b = tiny_system(100 + seed, n)
    Af, bf = frac_mat(A), [Fraction(int(v)) for v in b]
    runs = ratref.bicgstab(Af, bf, [Fraction(0)] * n, 4)
    rp, ci, v = dense_to_csr(A)
    res = orc.solve(rp, ci, v, b.astype(float), tol=1e-300, maxit=3, alg=alg, mode=orc.EXACT, trace=True)
    normb = math.sqrt(float(ratref.dot(bf, bf)))
    k = min(3, len(runs))
    for i in range(k):
        r = runs[i]["r"]
        want = math.sqrt(float(ratref.dot(r, r))) / normb
        got = res.history[i + 1]
        if want == 0:
            assert got < 1e-12
        else:
            assert abs(got - want) <= 1e-9 * want + 1e-15, (i, got, want)
        assert abs(res.trace[i, 0] - float(runs[i]["alpha"])) <= 1e-9 * abs(float(runs[i]["alpha"]))
        assert abs(res.trace[i, 1] - float(runs[i]["omega"])) <= 1e-9 * abs(float(runs[i]["omega"]))


@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_scaled_identity_lucky_breakdown(orc, alg, mode):
    """A = 4 I: one iteration gives x = b/4 exactly (q = 0, y = 0, omega = 0)."""
    n = 50
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    v = np.full(n, 4.0)
    b = np.random.default_rng(0).standard_normal(n)
    res = orc.solve(rp, ci, v, b, tol=1e-14, maxit=10, alg=alg, mode=mode)
    assert res.status == orc.CONVERGED and res.iters == 1
    assert np.array_equal(res.x, b / 4.0)
    assert res.history[1] == 0.0 and res.relres_true == 0.0


@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_power_of_two_scaling_is_exact(orc, alg, mode):
    A = inputs.convdiff2d(16, 5.0)
    b = inputs.rhs_ones(A)
    r1 = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-10, maxit=200, alg=alg, mode=mode)
    r2 = orc.solve(A.row_ptr, A.col_idx, A.vals * 2.0 ** 40, b * 2.0 ** 40, tol=1e-10, maxit=200,
                   alg=alg, mode=mode)
    r3 = orc.solve(A.row_ptr, A.col_idx, A.vals, b * 2.0 ** -30, tol=1e-10, maxit=200, alg=alg, mode=mode)
    assert r1.iters == r2.iters == r3.iters
    assert np.array_equal(r1.history, r2.history) and np.array_equal(r1.history, r3.history)
    assert np.array_equal(r1.x, r2.x)
    assert np.array_equal(r1.x * 2.0 ** -30, r3.x)


@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("N,Pe,tol", [(32, 10.0, 1e-8), (24, 60.0, 1e-10)])
def test_true_residual_reaches_tol(orc, alg, mode, N, Pe, tol):
    A = inputs.convdiff2d(N, Pe)
    b = inputs.rhs_ones(A)
    res = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=tol, maxit=3000, alg=alg, mode=mode)
    assert res.status == orc.CONVERGED
    assert res.relres_true <= tol
    assert res.history.size == res.iters + 1
    assert res.history[-1] <= tol
    assert np.max(np.abs(res.x - 1.0)) < 1e3 * tol * N * N


def test_bicgstab_and_pipelined_agree_early(orc):
    """Equivalent in exact arithmetic: FP64 histories agree closely at first."""
    A = inputs.convdiff2d(16, 1.0)
    b = inputs.rhs_ones(A)
    for mode in (0, 1):
        h1 = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-300, maxit=5, alg=0, mode=mode).history
        h2 = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-300, maxit=5, alg=1, mode=mode).history
        assert h1.size == h2.size == 6
        assert np.all(np.abs(h1 - h2) <= 1e-6 * np.abs(h1))


def test_exact_start_converges_at_zero(orc):
    A = inputs.convdiff2d(8, 3.0)
    b = inputs.rhs_ones(A)
    for alg in (0, 1):
        res = orc.solve(A.row_ptr, A.col_idx, A.vals, b, x0=np.ones(A.n), tol=1e-12, maxit=10, alg=alg)
        assert res.status == orc.CONVERGED and res.iters == 0 and res.history.tolist() == [0.0]


def test_maxit_zero_and_nonfinite(orc):
    A = inputs.convdiff2d(8, 3.0)
    b = inputs.rhs_ones(A)
    for alg in (0, 1):
        res = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-12, maxit=0, alg=alg)
        assert res.status == orc.MAXIT and res.iters == 0 and res.history.size == 1
        bn = b.copy()
        bn[3] = np.nan
        res = orc.solve(A.row_ptr, A.col_idx, A.vals, bn, tol=1e-12, maxit=10, alg=alg)
        assert res.status == orc.NONFINITE and res.iters == 0
        vn = A.vals.copy()
        vn[5] = np.inf
        res = orc.solve(A.row_ptr, A.col_idx, vn, b, tol=1e-12, maxit=10, alg=alg)
        assert res.status == orc.NONFINITE


def test_breakdown_skew(orc):
    """(r0, A r0) = 0 for skew-symmetric A: alpha_0 is infinite -> BREAKDOWN."""
    rp = np.array([0, 1, 2], np.int32)
    ci = np.array([1, 0], np.int32)
    v = np.array([1.0, -1.0])
    b = np.array([1.0, 0.0])
    for alg in (0, 1):
        for mode in (0, 1):
            res = orc.solve(rp, ci, v, b, tol=1e-10, maxit=10, alg=alg, mode=mode)
            assert res.status == orc.BREAKDOWN and res.iters == 0
            assert np.array_equal(res.x, [0.0, 0.0])


def test_invalid_inputs(orc):
    rp = np.array([0, 1, 2], np.int32)
    ci = np.array([1, 0], np.int32)
    v = np.array([1.0, 1.0])
    b = np.ones(2)
    with pytest.raises(ValueError):
        orc.solve(rp, ci, v, b, tol=0.0)
    with pytest.raises(ValueError):
        orc.solve(rp, np.array([1, 2], np.int32), v, b)
    with pytest.raises(ValueError):
        orc.solve(np.array([0, 2, 1], np.int32), ci, v, b)
    with pytest.raises(ValueError):
        orc.solve(rp, ci, v, b, maxit=-1)


def test_exact_mode_history_is_partition_free(orc):
    """Exact dots make the whole run independent of how dots are split across
    threads (the single-node analogue of the process-count invariance of Tables 2-3)."""
    A = inputs.convdiff3d(42, 50.0)
    b = inputs.rhs_ones(A)
    ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-10, maxit=40, alg=1, mode=1, nthreads=1)
    for t in (3, 8):
        res = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-10, maxit=40, alg=1, mode=1, nthreads=t)
        assert np.array_equal(res.history, ref.history) and np.array_equal(res.x, ref.x)


@pytest.mark.parametrize("seed", range(3))
def test_rr_iterates_follow_rational(orc, seed):
    """Residual replacement swaps recurrence vectors for their true values,
    which are equal in exact arithmetic: the FP64 oracle with replacement every
    2 iterations still follows the rational Algorithm 2."""
    n = 6
    A, b = tiny_system(200 + seed, n)
    Af, bf = frac_mat(A), [Fraction(int(v)) for v in b]
    runs = ratref.pbicgstab(Af, bf, [Fraction(0)] * n, 5)
    rp, ci, v = dense_to_csr(A)
    res = orc.solve(rp, ci, v, b.astype(float), tol=1e-300, maxit=4, alg=1, mode=orc.EXACT, rr_period=2)
    normb = math.sqrt(float(ratref.dot(bf, bf)))
    for i in range(min(4, len(runs))):
        r = runs[i]["r"]
        want = math.sqrt(float(ratref.dot(r, r))) / normb
        if want == 0:
            assert res.history[i + 1] < 1e-12
        else:
            assert abs(res.history[i + 1] - want) <= 1e-9 * want + 1e-15


def test_rr_keeps_true_residual_on_track(orc):
    """48^3 convection-diffusion to 1e-12: plain p-BiCGStab loses its true
    residual; with replacement every 25 iterations it converges."""
    A = inputs.convdiff3d(32, 50.0)
    b = inputs.rhs_ones(A)
    rr = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-12, maxit=1500, alg=1, mode=1, rr_period=25, nthreads=8)
    assert rr.status == orc.CONVERGED and rr.relres_true <= 1e-12
    with pytest.raises(ValueError):
        orc.solve(A.row_ptr, A.col_idx, A.vals, b, alg=0, rr_period=5)


def test_rr_period_zero_is_algorithm_2(orc):
    A = inputs.convdiff2d(16, 5.0)
    b = inputs.rhs_ones(A)
    r0 = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-10, maxit=300, alg=1, mode=1)
    r1 = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-10, maxit=300, alg=1, mode=1, rr_period=0)
    assert np.array_equal(r0.history, r1.history) and np.array_equal(r0.x, r1.x)


# ---------------------------------------------------------------------------
# right Jacobi preconditioning (orc_solve_jacobi)
# ---------------------------------------------------------------------------
def _scaled_columns(A, d):
    """A with column j multiplied by 1/d_j, computed exactly for powers of two."""
    v = A.vals.astype(np.float64).copy()
    for i in range(A.n):
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            v[k] = math.ldexp(v[k], -int(math.log2(abs(d[A.col_idx[k]]))))
            if d[A.col_idx[k]] < 0:
                v[k] = -v[k]
    return v


@pytest.mark.parametrize("alg", [0, 1])
def test_jacobi_with_unit_diagonal_is_the_plain_solve(orc, alg):
    A = inputs.convdiff2d(10, 20.0)
    diag = np.zeros(A.n)
    for i in range(A.n):
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            if A.col_idx[k] == i:
                diag[i] = A.vals[k]
    # divide every row by its diagonal entry (exact for this test's purpose: a new matrix with unit diagonal)
    v = A.vals / np.repeat(diag, np.diff(A.row_ptr))
    U = inputs.CSR(A.n, A.row_ptr, A.col_idx, v)
    b = inputs.rhs_ones(U)
    x0 = np.linspace(-1.0, 1.0, A.n)
    ref = orc.solve(U.row_ptr, U.col_idx, U.vals, b, x0=x0, tol=1e-10, maxit=300, alg=alg, mode=1)
    got = orc.solve(U.row_ptr, U.col_idx, U.vals, b, x0=x0, tol=1e-10, maxit=300, alg=alg, mode=1, jacobi=True)
    assert got.status == ref.status and got.iters == ref.iters
    assert np.array_equal(got.x.view(np.int64), ref.x.view(np.int64))
    assert np.array_equal(got.history.view(np.int64), ref.history.view(np.int64))


@pytest.mark.parametrize("alg", [0, 1])
def test_jacobi_is_the_solve_of_the_column_scaled_system(orc, alg):
    """Diagonal entries +-2^k: A M^-1 and the unscaling are exact, so the
    preconditioned solve must equal, bit for bit, the plain solve of the
    column-scaled matrix from y0 = d x0, followed by x = y / d."""
    rng = np.random.default_rng(4)
    A = inputs.convdiff2d(9, 15.0)
    n = A.n
    d = np.ldexp(1.0, rng.integers(-6, 7, n)) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    v = A.vals.copy()
    for i in range(n):                       # put d on the diagonal, keep the off-diagonals
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            if A.col_idx[k] == i:
                v[k] = d[i]
    B = inputs.CSR(n, A.row_ptr, A.col_idx, v)
    b = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    got = orc.solve(B.row_ptr, B.col_idx, B.vals, b, x0=x0, tol=1e-9, maxit=400, alg=alg, mode=1, jacobi=True)
    vs = _scaled_columns(B, d)
    ref = orc.solve(B.row_ptr, B.col_idx, vs, b, x0=x0 * d, tol=1e-9, maxit=400, alg=alg, mode=1)
    assert got.status == ref.status and got.iters == ref.iters
    assert np.array_equal(got.history.view(np.int64), ref.history.view(np.int64))
    assert np.array_equal(got.x.view(np.int64), (ref.x / d).view(np.int64))


def test_jacobi_helps_a_badly_scaled_matrix(orc):
    A = inputs.powerlaw(n=600, mean_len=8.0, max_len=60, seed=9)
    b = inputs.rhs_ones(A)
    plain = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-10, maxit=600, alg=1, mode=1)
    jac = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-10, maxit=600, alg=1, mode=1, jacobi=True)
    assert jac.status == 0 and jac.iters < plain.iters
    r = b - orc.spmv(A.row_ptr, A.col_idx, A.vals, jac.x)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-8


def test_jacobi_rejects_a_missing_or_zero_diagonal(orc):
    A = inputs.convdiff2d(5, 1.0)
    v = A.vals.copy()
    v[A.row_ptr[3]:A.row_ptr[4]][A.col_idx[A.row_ptr[3]:A.row_ptr[4]] == 3] = 0.0
    with pytest.raises(ValueError):
        orc.solve(A.row_ptr, A.col_idx, v, inputs.rhs_ones(A), tol=1e-8, maxit=10, jacobi=True)


def _true_relres(A, b, x):
    """||b - A x|| / ||b|| as the stopping rule defines it: the SpMV row as its
    fma chain, r_i = b_i - (A x)_i in FP64, both dots correctly rounded, then
    sqrt((r,r)) / sqrt((b,b)) -- computed here with rationals, not the oracle."""
    from tests.fracref import exact_dot, fma_spmv, rn
    r = np.asarray(b) - np.array(fma_spmv(A.row_ptr, A.col_idx, A.vals, x))
    sb = math.sqrt(rn(exact_dot(b, b)))
    return math.sqrt(rn(exact_dot(r, r))) / (sb if sb != 0.0 else 1.0)


# (side, Peclet, tol, alg, mode, the oracle's status): tolerances at the level
# of attainable accuracy, where the recursive residual passes the target
# before the true residual does
STOP_CASES = [
    (6, 3.0, 1.35e-15, 0, 0, 0),      # one failed check, then a stop
    (8, 10.0, 4e-15, 0, 1, 0),
    (12, 5.0, 4e-15, 0, 1, 0),        # two failed checks
    (10, 30.0, 3.6e-15, 0, 0, 0),     # three
    (6, 3.0, 1e-15, 0, 1, 2),         # every check fails until a breakdown
    (8, 10.0, 3e-15, 1, 1, 1),        # p-BiCGStab: checks fail, the iterate drifts, maxit
]


@pytest.mark.parametrize("case", STOP_CASES, ids=[f"{c[0]}x{c[0]}-tol{c[2]:g}-alg{c[3]}-mode{c[4]}" for c in STOP_CASES])
def test_stop_rule_true_residual_decides(orc, case):
    """Reading 6 simulated outside the oracle: from the oracle's residual
    history and its iterates x_k (a rerun with maxit = k), a check happens at
    the first k whose recursive residual is <= the target; the true residual
    (computed above with rationals) ends the solve if it is <= tol, else the
    target becomes tol*(tol/true) and the loop goes on.  The predicted stop
    must be the oracle's, and where no check passes the oracle must not
    report convergence.  (On these systems a target left at tol predicts the
    same stops: the skipped iterations have true residuals above tol.)"""
    N, Pe, tol, alg, mode, status = case
    A = inputs.convdiff2d(N, Pe)
    b = inputs.rhs_ones(A)
    maxit = 300
    full = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=tol, maxit=maxit, alg=alg, mode=mode)
    assert full.status == status
    h = full.history
    target, failed, stop = tol, 0, None
    for k in range(len(h)):
        if not h[k] <= target:
            continue
        xk = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=tol, maxit=k, alg=alg, mode=mode).x
        true = _true_relres(A, b, xk)
        if true <= tol:
            stop = k
            break
        failed += 1
        target = tol * (tol / true)
    assert failed >= 1                       # the recursive residual alone would have stopped earlier
    if status == orc.CONVERGED:
        assert stop == full.iters
        assert full.relres_true == _true_relres(A, b, full.x) <= tol
    else:
        assert stop is None and full.relres_true > tol


# (name, system, tolerance): tolerances at which plain p-BiCGStab stalls on these systems
TIGHT = [
    ("2D 96^2, Pe 60", lambda: inputs.convdiff2d(96, 60.0), 1e-10),
    ("3D 32^3, Pe 50", lambda: inputs.convdiff3d(32, 50.0), 1e-12),
]


@pytest.mark.parametrize("name,make,tol", TIGHT, ids=["2d96", "3d32"])
def test_exact_dots_let_pipelined_reach_a_tight_tolerance(orc, name, make, tol):
    """Section 3's observation, on synthetic systems: at a tight tolerance
    p-BiCGStab with plain FP64 dots loses its true residual (the recursive
    one falls below tol, the iterate drifts away) while the same iteration
    with exactly rounded dots converges, and classical BiCGStab converges
    with either.  A measured, deterministic fact of the oracle; exact mode is
    bit-identical on the GPU, plain mode here is the sequential dot order."""
    A = make()
    b = inputs.rhs_ones(A)
    kw = dict(tol=tol, maxit=1000, nthreads=4)
    plain = orc.solve(A.row_ptr, A.col_idx, A.vals, b, alg=1, mode=orc.PLAIN, **kw)
    exact = orc.solve(A.row_ptr, A.col_idx, A.vals, b, alg=1, mode=orc.EXACT, **kw)
    assert plain.status == orc.MAXIT and plain.relres_recursive <= tol and plain.relres_true > 1e3 * tol
    assert exact.status == orc.CONVERGED and exact.relres_true <= tol and exact.iters < 300
    for mode in (orc.PLAIN, orc.EXACT):
        classical = orc.solve(A.row_ptr, A.col_idx, A.vals, b, alg=0, mode=mode, **kw)
        assert classical.status == orc.CONVERGED and classical.relres_true <= tol


@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_zero_rhs_uses_the_absolute_residual(orc, alg, mode):
    """b = 0: sqrt((b,b)) is replaced by 1, so the residual is absolute.
    x0 = 0 stops at k = 0 with res_0 = 0.  With A = 4I (n = 100) and x0 = 1,
    r0 = -4 * 1 and res_0 = sqrt(1600) = 40 exactly; then alpha = 1/4, q = 0,
    omega = 0 (lucky breakdown) and x = 1 + (1/4)(-4) = 0 exactly in one
    step, with res_1 = 0."""
    n = 100
    A = inputs.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.full(n, 4.0))
    b = np.zeros(n)
    r = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-12, maxit=10, alg=alg, mode=mode)
    assert r.status == orc.CONVERGED and r.iters == 0 and list(r.history) == [0.0]
    assert np.all(r.x == 0.0) and r.relres_true == 0.0
    r = orc.solve(A.row_ptr, A.col_idx, A.vals, b, x0=np.ones(n), tol=1e-12, maxit=10, alg=alg, mode=mode)
    assert r.status == orc.CONVERGED and r.iters == 1
    assert list(r.history) == [40.0, 0.0]
    assert np.all(r.x == 0.0) and r.relres_true == 0.0


def _with_empty_row(A, p):
    """A with an empty row (and a column nothing references) inserted at index p."""
    rp, ci, v = [0], [], []
    for i in range(A.n + 1):
        if i == p:
            rp.append(len(ci))
        if i < A.n:
            for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
                c = int(A.col_idx[k])
                ci.append(c + 1 if c >= p else c)
                v.append(float(A.vals[k]))
            rp.append(len(ci))
    return inputs.CSR(A.n + 1, np.array(rp, np.int32), np.array(ci, np.int32), np.array(v))


@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_empty_row_with_zero_rhs_changes_nothing(orc, alg, mode):
    """An empty row i (SpMV gives +0 there) with b_i = 0 and x0_i = 0 keeps
    r_i = 0, so every dot gains only exact zero terms: the residual history is
    the reduced system's bit for bit, x_i stays 0 and the other entries of x
    are the reduced solution's, wherever the row is inserted."""
    A = inputs.convdiff2d(9, 12.0)
    b = inputs.rhs_ones(A)
    ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-11, maxit=200, alg=alg, mode=mode)
    for p in (0, A.n // 2, A.n):
        B = _with_empty_row(A, p)
        bb = np.insert(b, p, 0.0)
        got = orc.solve(B.row_ptr, B.col_idx, B.vals, bb, tol=1e-11, maxit=200, alg=alg, mode=mode)
        assert got.status == ref.status and got.iters == ref.iters, p
        assert np.array_equal(got.history.view(np.int64), ref.history.view(np.int64)), p
        assert got.x[p] == 0.0 and np.array_equal(np.delete(got.x, p).view(np.int64), ref.x.view(np.int64)), p


@pytest.mark.parametrize("mode", [0, 1])
def test_first_iteration_copies_keep_the_sign_of_zero(orc, mode):
    """Reading 4: Algorithm 2 starts from p0 = r0, s0 = w0, z0 = t0 as bit
    copies.  On an unknown that nothing couples (an empty row and column)
    with b_p = -0 and x0_p = -0, the IEEE sign rules fix every value by hand:
    (A v)_p = +0 for any v, so s, z, w, t, v and y stay +0 there, and with
    alpha, omega > 0 (and beta > 0 wherever the p it forms reaches an x
    update) the forms q = fma(-a, s, r), r = fma(-w, y, q),
    p = fma(b, fma(-w, s, p), r) and x = fma(w, q, fma(a, p, x)) keep
    r_p = q_p = p_p = x_p = -0 after every iteration.  Had p0 been formed as
    fma(0, ., r0), p0_p would be +0 and x_p would turn +0 at once."""
    A = inputs.convdiff2d(9, 12.0)
    b = inputs.rhs_ones(A)
    p = 5
    B = _with_empty_row(A, p)
    bb = np.insert(b, p, -0.0)
    x0 = np.zeros(B.n)
    x0[p] = -0.0
    for its in (1, 2, 6):
        r = orc.solve(B.row_ptr, B.col_idx, B.vals, bb, x0=x0, tol=1e-300, maxit=its, alg=1, mode=mode, trace=True)
        # alpha, omega > 0 in every iteration run; beta > 0 where it forms a p that an x update uses
        assert r.iters == its and np.all(r.trace[:, :2] > 0) and np.all(r.trace[:-1, 2] > 0)
        assert r.x[p] == 0.0 and math.copysign(1.0, r.x[p]) == -1.0, its
