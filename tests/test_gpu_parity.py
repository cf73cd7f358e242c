"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Exact mode: residual history, iteration count, status and x bit-identical.
Plain mode: history within a relative 1e-8 over the first 20 iterations and
the true relative residual <= tol.  Dots and SpMV are checked on their own too.
"""
import math

import numpy as np
import pytest

from paper_2404_13216_gb300 import inputs
from tests import dotcases

pytestmark = pytest.mark.gpu

PLAIN_HIST_RTOL = 1e-8      # relative, first 20 iterations (plain-mode dot order differs)


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2404_13216_gb300 import build
    build.build_library()
    from paper_2404_13216_gb300 import pbcg
    c = pbcg.Context(0)
    yield c
    c.close()


def same(a, b):
    return np.array_equal(np.asarray(a).view(np.int64), np.asarray(b).view(np.int64))


# --------------------------------------------------------------------------- dots
CASES = dotcases.cases(0)


@pytest.mark.parametrize("name,a,b", CASES, ids=[c[0] for c in CASES])
def test_exact_dot_bitwise(ctx, orc, name, a, b):
    got = ctx.dot(a, b, mode=1)
    want = orc.dot_exact(a, b)
    if math.isnan(want):
        assert math.isnan(got)
    else:
        assert same([got], [want]), (name, got, want)


def test_exact_dot_large_random(ctx, orc):
    rng = np.random.default_rng(11)
    for n in (1, 31, 32, 33, 1000, 65537, 1_000_003):
        a = rng.standard_normal(n) * np.ldexp(1.0, rng.integers(-40, 40, n))
        b = rng.standard_normal(n) * np.ldexp(1.0, rng.integers(-300, 300, n))
        assert same([ctx.dot(a, b, 1)], [orc.dot_exact(a, b, nthreads=8)]), n


def test_exact_dot_random_sweep(ctx, orc):
    """120 seeded cases: random lengths (ragged against warps and tiles), exponent
    spans from narrow to the whole double range (subnormals included), signs,
    exact zeros, and planted cancellation; every result bit-identical."""
    rng = np.random.default_rng(2024)
    for case in range(120):
        n = int(rng.integers(1, 5000))
        lo = int(rng.integers(-1074, 900))
        hi = int(min(1000, lo + rng.integers(0, 2000)))
        ea = rng.integers(lo, hi + 1, n) // 2
        eb = rng.integers(lo, hi + 1, n) - ea
        a = np.ldexp(rng.uniform(0.5, 1.0, n), ea) * rng.choice([-1.0, 1.0], n)
        b = np.ldexp(rng.uniform(0.5, 1.0, n), np.clip(eb, -1074, 1000)) * rng.choice([-1.0, 1.0], n)
        a[rng.random(n) < 0.05] = 0.0
        if case % 3 == 0 and n > 1:                  # cancel half of the terms exactly
            h = n // 2
            a[h:2 * h] = -a[:h]
            b[h:2 * h] = b[:h]
        want = orc.dot_exact(a, b, nthreads=4)
        got = ctx.dot(a, b, 1)
        if math.isnan(want):
            assert math.isnan(got), case
        else:
            assert same([got], [want]) or (got == 0.0 and want == 0.0), (case, n, lo, hi, got, want)


def test_exact_dot_empty_and_nonfinite(ctx):
    assert ctx.dot(np.zeros(0), np.zeros(0), 1) == 0.0
    a = np.ones(100)
    a[57] = np.inf
    assert math.isnan(ctx.dot(a, np.ones(100), 1))
    # the accumulator is clean afterwards: the next dot sees none of the finite terms above
    assert ctx.dot(np.ones(10), np.ones(10), 1) == 10.0


def test_plain_dot_close(ctx, orc):
    rng = np.random.default_rng(12)
    a, b = rng.standard_normal(100_000), rng.standard_normal(100_000)
    want = orc.dot_exact(a, b)
    assert abs(ctx.dot(a, b, 0) - want) <= 1e-12 * np.abs(a * b).sum()


# --------------------------------------------------------------------------- SpMV
@pytest.mark.parametrize("gen", ["2d64", "3d20", "powerlaw"])
def test_spmv_bitwise(ctx, orc, gen):
    if gen == "2d64":
        A = inputs.convdiff2d(64, 10.0)
    elif gen == "3d20":
        A = inputs.convdiff3d(20, 50.0)
    else:
        A = inputs.powerlaw(n=5000, mean_len=30, max_len=400, seed=2)
    M = ctx.upload_csr(A)
    x = np.random.default_rng(1).standard_normal(A.n)
    assert same(ctx.spmv(M, x), orc.spmv(A.row_ptr, A.col_idx, A.vals, x))
    M.free()


# --------------------------------------------------------------------------- solves
def run_both(ctx, orc, A, b, tol, maxit, alg, mode, x0=None):
    ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, x0=x0, tol=tol, maxit=maxit, alg=alg, mode=mode, nthreads=8)
    M = ctx.upload_csr(A)
    x = np.zeros(A.n) if x0 is None else np.array(x0, dtype=np.float64)
    res = ctx.solve(M, b, x, tol, maxit, alg, mode)
    hist = ctx.history()
    M.free()
    return ref, res, x, hist


SYSTEMS = {
    "2d64_pe10": lambda: inputs.convdiff2d(64, 10.0),
    "2d37_pe40": lambda: inputs.convdiff2d(37, 40.0),          # ragged: n = 1369
    "3d24_pe50": lambda: inputs.convdiff3d(24, 50.0),
    "2d5_pe3": lambda: inputs.convdiff2d(5, 3.0),               # n = 25 < one tile
}


@pytest.mark.parametrize("alg", [0, 1], ids=["bicgstab", "pbicgstab"])
@pytest.mark.parametrize("sysname", list(SYSTEMS))
def test_exact_solve_bitwise(ctx, orc, sysname, alg):
    A = SYSTEMS[sysname]()
    b = inputs.rhs_ones(A)
    ref, res, x, hist = run_both(ctx, orc, A, b, 1e-8, 2000, alg, 1)
    assert res.status == ref.status and res.iters == ref.iters, (res, ref.status, ref.iters)
    assert same(hist, ref.history)
    assert same(x, ref.x)
    assert same([res.relres_true], [ref.relres_true])


@pytest.mark.parametrize("alg", [0, 1], ids=["bicgstab", "pbicgstab"])
def test_plain_solve_tolerance_2d64(ctx, orc, alg):
    """The 64x64 configuration: plain-mode history within 1e-8 (relative) of the
    oracle's over the first 20 iterations, true relative residual <= tol."""
    A = SYSTEMS["2d64_pe10"]()
    b = inputs.rhs_ones(A)
    tol = 1e-8
    ref, res, x, hist = run_both(ctx, orc, A, b, tol, 2000, alg, 0)
    assert res.status == 0 and res.relres_true <= tol
    k = min(21, hist.size, ref.history.size)
    rel = np.abs(hist[:k] - ref.history[:k]) / np.abs(ref.history[:k])
    assert np.all(rel <= PLAIN_HIST_RTOL), rel.max()


def sensitivity_bar(orc, A, b, alg, k):
    """Per-iteration spread between two valid FP64 dot orders on the CPU (the
    oracle's sequential fma dot and its correctly rounded dot)."""
    hp = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-300, maxit=k, alg=alg, mode=0).history
    he = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-300, maxit=k, alg=alg, mode=1, nthreads=8).history
    return hp, np.abs(hp - he) / np.abs(he)


@pytest.mark.parametrize("alg", [0, 1], ids=["bicgstab", "pbicgstab"])
def test_plain_solve_3d_sensitivity_relative(ctx, orc, alg):
    """3D systems separate faster than 1e-8 under any change of dot order (the
    CPU's own two orders differ by ~3e-8 within 20 iterations), so the plain-mode
    history is held to 4x that spread plus 1e-13, and the solve must converge."""
    A = SYSTEMS["3d24_pe50"]()
    b = inputs.rhs_ones(A)
    k = 20
    hp, spread = sensitivity_bar(orc, A, b, alg, k)
    M = ctx.upload_csr(A)
    x = np.zeros(A.n)
    ctx.solve(M, b, x, 1e-300, k, alg, 0)
    hist = ctx.history()
    rel = np.abs(hist - hp) / np.abs(hp)
    assert np.all(rel <= 4 * spread + 1e-13), (rel.max(), spread.max())
    x = np.zeros(A.n)
    res = ctx.solve(M, b, x, 1e-8, 2000, alg, 0)
    assert res.status == 0 and res.relres_true <= 1e-8
    M.free()


def test_golden_fixture_exact(ctx):
    """The committed oracle fixture for the 64x64 system (tests/golden)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "convdiff64.json")))
    A = inputs.convdiff2d(64, 10.0, (1.0, 0.5))
    b = inputs.rhs_ones(A)
    M = ctx.upload_csr(A)
    for alg, an in ((0, "bicgstab"), (1, "pbicgstab")):
        want = g["runs"][f"{an}_exact"]
        x = np.zeros(A.n)
        r = ctx.solve(M, b, x, 1e-8, 2000, alg, 1)
        assert r.status == want["status"] and r.iters == want["iters"]
        assert same(ctx.history(), np.array([float.fromhex(h) for h in want["history"]]))
    M.free()


# --------------------------------------------------------------------------- edge cases
@pytest.fixture(params=[1, 0], ids=["cluster", "passes"])
def small_path(ctx, request):
    """Small systems run as one cluster launch by default; 0 keeps the passes."""
    from paper_2404_13216_gb300 import pbcg
    ctx.set_option(pbcg.OPT_SMALL_CLUSTER, request.param)
    yield request.param
    ctx.set_option(pbcg.OPT_SMALL_CLUSTER, 1)


@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_edge_cases(ctx, orc, alg, mode, small_path):
    # one unknown
    A = inputs.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0]))
    ref, res, x, hist = run_both(ctx, orc, A, np.array([6.0]), 1e-12, 10, alg, mode)
    assert res.status == ref.status == 0 and res.iters == ref.iters and same(x, ref.x)
    # exact start
    A = inputs.convdiff2d(8, 3.0)
    b = inputs.rhs_ones(A)
    ref, res, x, hist = run_both(ctx, orc, A, b, 1e-12, 10, alg, mode, x0=np.ones(A.n))
    assert res.status == 0 and res.iters == 0 and same(hist, ref.history)
    # maxit = 0
    ref, res, x, hist = run_both(ctx, orc, A, b, 1e-12, 0, alg, mode)
    assert res.status == ref.status == 1 and res.iters == 0
    # NaN in b
    bn = b.copy()
    bn[3] = np.nan
    ref, res, x, hist = run_both(ctx, orc, A, bn, 1e-12, 10, alg, mode)
    assert res.status == ref.status == 3 and res.iters == 0
    # skew breakdown
    A = inputs.CSR(2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.array([1.0, -1.0]))
    ref, res, x, hist = run_both(ctx, orc, A, np.array([1.0, 0.0]), 1e-10, 10, alg, mode)
    assert res.status == ref.status == 2 and res.iters == 0
    # A = 4 I: lucky breakdown, exact in one step
    n = 100
    A = inputs.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.full(n, 4.0))
    bb = np.random.default_rng(0).standard_normal(n)
    ref, res, x, hist = run_both(ctx, orc, A, bb, 1e-14, 10, alg, mode)
    assert res.status == 0 and res.iters == 1 and same(x, bb / 4.0)


def test_invalid_inputs(ctx):
    from paper_2404_13216_gb300 import pbcg
    with pytest.raises(pbcg.PbcgError):
        ctx.upload(np.array([0, 1, 2], np.int32), np.array([1, 5], np.int32), np.ones(2))
    with pytest.raises(pbcg.PbcgError):
        ctx.upload(np.array([0, 2, 1], np.int32), np.array([1, 0], np.int32), np.ones(2))
    A = inputs.convdiff2d(4, 1.0)
    M = ctx.upload_csr(A)
    with pytest.raises(pbcg.PbcgError):
        ctx.solve(M, np.ones(A.n), np.zeros(A.n), 0.0, 10)
    with pytest.raises(pbcg.PbcgError):
        ctx.solve(M, np.ones(A.n), np.zeros(A.n), 1e-8, -1)
    with pytest.raises(pbcg.PbcgError):
        ctx.solve(M, np.ones(A.n), np.zeros(A.n), 1e-8, 10, alg=7)
    with pytest.raises(pbcg.PbcgError) as e:                     # maxit + 1 history entries must fit int32
        ctx.solve(M, np.ones(A.n), np.zeros(A.n), 1e-8, 2 ** 31 - 1)
    assert e.value.code == pbcg.ERR_INVALID
    M.free()


def test_device_pointers(ctx, orc):
    import torch
    A = inputs.convdiff2d(40, 20.0)
    b = inputs.rhs_ones(A)
    ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-9, maxit=1000, alg=1, mode=1)
    M = ctx.upload(torch.from_numpy(A.row_ptr).cuda(), torch.from_numpy(A.col_idx).cuda(),
                   torch.from_numpy(A.vals).cuda())
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    res = ctx.solve(M, bd, xd, 1e-9, 1000, 1, 1)
    assert res.iters == ref.iters and same(xd.cpu().numpy(), ref.x)
    M.free()


# --------------------------------------------------------------------------- full size
def test_full_size_128cubed_first_iterations(ctx, orc):
    """3D 128^3 (n = 2,097,152) in the launch shape the benchmark uses: exact mode
    bit-identical to the oracle over the first iterations; plain mode within
    4x the CPU's own two-order spread over 20 iterations."""
    A = inputs.convdiff3d(128, 50.0)
    b = inputs.rhs_ones(A)
    ref, res, x, hist = run_both(ctx, orc, A, b, 1e-10, 4, 1, 1)
    assert res.iters == ref.iters == 4
    assert same(hist, ref.history) and same(x, ref.x)
    k = 20
    hp, spread = sensitivity_bar(orc, A, b, 1, k)
    M = ctx.upload_csr(A)
    x = np.zeros(A.n)
    ctx.solve(M, b, x, 1e-300, k, 1, 0)
    hist = ctx.history()
    M.free()
    rel = np.abs(hist - hp) / np.abs(hp)
    assert np.all(rel <= 4 * spread + 1e-13), (rel.max(), spread.max())


def test_full_size_128cubed_benchmark_solve(ctx, orc):
    """The benchmark's whole solve: 128^3, exact p-BiCGStab, tol 1e-10, maxit
    1000, in the launch graph the benchmark times.  All 1001 residual-history
    entries, the iteration count, the status, the true residual and x
    bit-identical to the oracle (about a minute of oracle time on 16 cores)."""
    import os
    A = inputs.convdiff3d(128, 50.0)
    b = inputs.rhs_ones(A)
    ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-10, maxit=1000, alg=1, mode=1,
                    nthreads=max(1, min(16, os.cpu_count() or 1)))
    M = ctx.upload_csr(A)
    x = np.zeros(A.n)
    res = ctx.solve(M, b, x, 1e-10, 1000, 1, 1)
    hist = ctx.history()
    M.free()
    assert res.status == ref.status and res.iters == ref.iters, (res, ref.status, ref.iters)
    assert hist.size == ref.history.size and same(hist, ref.history)
    assert same(x, ref.x)
    assert same([res.relres_true], [ref.relres_true])


def test_full_size_powerlaw_first_iterations(ctx, orc):
    """The power-law configuration at full size (n = 2^22, about 126 M stored
    entries, rows sorted by length, tiles claimed dynamically), in the
    launches the benchmark times (pbcg_solve, tol 1e-300): exact p-BiCGStab
    over 3 iterations and right-Jacobi exact p-BiCGStab over 2, the residual
    histories and all 4,194,304 entries of x bit-identical to the oracle."""
    import os
    from paper_2404_13216_gb300 import pbcg
    A = inputs.powerlaw()
    b = inputs.rhs_ones(A)
    nt = max(1, min(16, os.cpu_count() or 1))
    M = ctx.upload_csr(A)
    try:
        for jac, its in ((False, 3), (True, 2)):
            ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-300, maxit=its, alg=1, mode=1, nthreads=nt,
                            jacobi=jac)
            ctx.set_option(pbcg.OPT_PRECOND, pbcg.PRECOND_JACOBI if jac else pbcg.PRECOND_NONE)
            x = np.zeros(A.n)
            res = ctx.solve(M, b, x, 1e-300, its, pbcg.PIPELINED, pbcg.EXACT)
            hist = ctx.history()
            assert res.status == ref.status and res.iters == ref.iters == its, (jac, res)
            assert same(hist, ref.history), jac
            assert same(x, ref.x), jac
    finally:
        ctx.set_option(pbcg.OPT_PRECOND, pbcg.PRECOND_NONE)
        M.free()


@pytest.mark.parametrize("alg", [0, 1], ids=["bicgstab", "pbicgstab"])
def test_powerlaw_exact_bitwise(ctx, orc, alg):
    """Random power-law rows (the rows are sorted by length inside the library
    and most tiles gather from global memory): exact solve bit-identical."""
    A = inputs.powerlaw(n=30000, mean_len=30, max_len=600, seed=5)
    b = inputs.rhs_ones(A)
    ref, res, x, hist = run_both(ctx, orc, A, b, 1e-10, 500, alg, 1)
    assert res.status == ref.status and res.iters == ref.iters
    assert same(hist, ref.history) and same(x, ref.x)


def test_mixed_window_tiles_exact_bitwise(ctx, orc):
    """A stencil matrix with a few long random rows: some tiles gather from
    staged blocks, others from global memory, in the same pass (the passes are
    forced: 8000 rows would otherwise run as one cluster launch)."""
    from paper_2404_13216_gb300 import pbcg
    A = inputs.convdiff3d(20, 30.0)
    rng = np.random.default_rng(9)
    rows = []
    for i in range(A.n):
        c = list(A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]])
        v = list(A.vals[A.row_ptr[i]:A.row_ptr[i + 1]])
        if i % 997 == 0:
            extra = rng.choice(A.n, size=12, replace=False)
            for j in extra:
                if j not in c:
                    c.append(int(j))
                    v.append(float(rng.uniform(-1e-3, 1e-3)))
            order = np.argsort(c)
            c = [c[k] for k in order]
            v = [v[k] for k in order]
        rows.append((c, v))
    rp = np.zeros(A.n + 1, np.int32)
    rp[1:] = np.cumsum([len(c) for c, _ in rows])
    B = inputs.CSR(A.n, rp, np.concatenate([c for c, _ in rows]).astype(np.int32),
                   np.concatenate([v for _, v in rows]))
    b = inputs.rhs_ones(B)
    ctx.set_option(pbcg.OPT_SMALL_CLUSTER, 0)
    try:
        ref, res, x, hist = run_both(ctx, orc, B, b, 1e-10, 600, 1, 1)
    finally:
        ctx.set_option(pbcg.OPT_SMALL_CLUSTER, 1)
    assert res.status == ref.status and res.iters == ref.iters
    assert same(hist, ref.history) and same(x, ref.x)


@pytest.mark.parametrize("mode", [1, 0], ids=["exact", "plain"])
@pytest.mark.parametrize("k", [7, 25])
def test_residual_replacement_vs_oracle(ctx, orc, mode, k):
    """p-BiCGStabRR (residual replacement every k iterations)."""
    from paper_2404_13216_gb300 import pbcg
    A = inputs.convdiff3d(24, 50.0)
    b = inputs.rhs_ones(A)
    tol = 1e-12
    ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=tol, maxit=1000, alg=1, mode=mode, rr_period=k, nthreads=8)
    ctx.set_option(pbcg.OPT_RR_PERIOD, k)
    M = ctx.upload_csr(A)
    x = np.zeros(A.n)
    res = ctx.solve(M, b, x, tol, 1000, pbcg.PIPELINED_RR, mode)
    hist = ctx.history()
    M.free()
    ctx.set_option(pbcg.OPT_RR_PERIOD, 50)
    if mode == 1:
        assert res.status == ref.status and res.iters == ref.iters
        assert same(hist, ref.history) and same(x, ref.x)
    else:
        assert res.status == 0 and res.relres_true <= tol


@pytest.mark.parametrize("alg", [0, 1, 2], ids=["bicgstab", "pbicgstab", "pbicgstab_rr"])
@pytest.mark.parametrize("sysname", ["2d_scaled", "powerlaw"])
def test_jacobi_exact_bitwise(ctx, orc, sysname, alg):
    """Right Jacobi preconditioning: the exact solve equals the oracle's bit for
    bit (a convection-diffusion matrix with a varied diagonal, and power-law
    rows, which the library reorders by length)."""
    from paper_2404_13216_gb300 import pbcg
    if sysname == "2d_scaled":
        A = inputs.convdiff2d(30, 25.0)
        rng = np.random.default_rng(3)
        v = A.vals.copy()
        for i in range(A.n):
            for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
                if A.col_idx[k] == i:
                    v[k] *= 10.0 ** rng.uniform(-2, 2)
        A = inputs.CSR(A.n, A.row_ptr, A.col_idx, v)
    else:
        A = inputs.powerlaw(n=20000, mean_len=20, max_len=400, seed=8)
    b = inputs.rhs_ones(A)
    x0 = np.full(A.n, 0.25)
    rr = 9 if alg == 2 else 0
    ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, x0=x0, tol=1e-10, maxit=600, alg=min(alg, 1), mode=1,
                    nthreads=8, rr_period=rr, jacobi=True)
    ctx.set_option(pbcg.OPT_PRECOND, pbcg.PRECOND_JACOBI)
    if alg == 2:
        ctx.set_option(pbcg.OPT_RR_PERIOD, rr)
    try:
        M = ctx.upload_csr(A)
        x = x0.copy()
        res = ctx.solve(M, b, x, 1e-10, 600, alg, 1)
        hist = ctx.history()
        M.free()
    finally:
        ctx.set_option(pbcg.OPT_PRECOND, pbcg.PRECOND_NONE)
        ctx.set_option(pbcg.OPT_RR_PERIOD, 50)
    assert res.status == ref.status and res.iters == ref.iters, (res, ref.status, ref.iters)
    assert same(hist, ref.history) and same(x, ref.x)
    assert same([res.relres_true], [ref.relres_true])


def test_jacobi_rejections(ctx):
    from paper_2404_13216_gb300 import pbcg
    A = inputs.convdiff2d(6, 2.0)
    v = A.vals.copy()
    v[A.row_ptr[4]:A.row_ptr[5]][A.col_idx[A.row_ptr[4]:A.row_ptr[5]] == 4] = 0.0
    Z = inputs.CSR(A.n, A.row_ptr, A.col_idx, v)
    ctx.set_option(pbcg.OPT_PRECOND, pbcg.PRECOND_JACOBI)
    try:
        M = ctx.upload_csr(Z)
        with pytest.raises(pbcg.PbcgError):
            ctx.solve(M, inputs.rhs_ones(A), np.zeros(A.n), 1e-8, 10, 1, 1)     # zero diagonal
        M.free()
    finally:
        ctx.set_option(pbcg.OPT_PRECOND, pbcg.PRECOND_NONE)
    with pytest.raises(pbcg.PbcgError):
        ctx.set_option(pbcg.OPT_PRECOND, 7)


def test_jacobi_batched_bitwise(ctx, orc):
    """Jacobi in a batched solve is Jacobi on every block: each system equals
    the oracle's preconditioned solve bit for bit; switching it off again gives
    the unpreconditioned results (the cached layout is rebuilt)."""
    from paper_2404_13216_gb300 import pbcg
    rng = np.random.default_rng(12)
    systems = []
    for side in (14, 21, 9):
        A = inputs.convdiff2d(side, float(rng.uniform(5, 60)))
        v = A.vals.copy()
        for i in range(A.n):
            for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
                if A.col_idx[k] == i:
                    v[k] *= 10.0 ** rng.uniform(-1.5, 1.5)
        systems.append(inputs.CSR(A.n, A.row_ptr, A.col_idx, v))
    systems.append(inputs.powerlaw(n=900, mean_len=10, max_len=120, seed=4))
    Bm, srp = inputs.block_diag(systems)
    b = inputs.rhs_ones(Bm)
    M = ctx.upload_csr(Bm)
    for jac in (True, False, True):
        ctx.set_option(pbcg.OPT_PRECOND, pbcg.PRECOND_JACOBI if jac else pbcg.PRECOND_NONE)
        try:
            x = np.full(Bm.n, 0.5)
            res = ctx.solve_batched(M, srp, b, x, np.full(len(systems), 1e-10), 800, 1, 1)
        finally:
            ctx.set_option(pbcg.OPT_PRECOND, pbcg.PRECOND_NONE)
        for k, S in enumerate(systems):
            r0, r1 = srp[k], srp[k + 1]
            ref = orc.solve(S.row_ptr, S.col_idx, S.vals, b[r0:r1], x0=np.full(S.n, 0.5), tol=1e-10, maxit=800,
                            alg=1, mode=1, jacobi=jac)
            assert res[k].status == ref.status and res[k].iters == ref.iters, (jac, k)
            assert same(x[r0:r1], ref.x), (jac, k)
    M.free()


# --------------------------------------------------------------------------- degenerate inputs
# Written against the oracle pins of the same cases.


def _duplicated(A, rng):
    """A with about half its rows holding one entry as two stored copies,
    0.625 v at the row's start and 0.375 v at its end (both exact), so the
    row's fma chain and a Jacobi diagonal meet the same column twice."""
    rp, ci, va = [0], [], []
    for i in range(A.n):
        cols = list(A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]])
        vals = list(A.vals[A.row_ptr[i]:A.row_ptr[i + 1]])
        if rng.random() < 0.5 and cols:
            k = int(rng.integers(len(cols)))
            c, v = cols.pop(k), vals.pop(k)
            cols = [c] + cols + [c]
            vals = [v * 0.625] + vals + [v * 0.375]
        ci += [int(c) for c in cols]
        va += [float(v) for v in vals]
        rp.append(len(ci))
    return inputs.CSR(A.n, np.array(rp, np.int32), np.array(ci, np.int32), np.array(va))


@pytest.mark.parametrize("alg", [0, 1])
def test_duplicate_columns_exact_bitwise(ctx, orc, alg, small_path):
    from paper_2404_13216_gb300 import pbcg
    A = _duplicated(inputs.convdiff2d(30, 25.0), np.random.default_rng(3))
    b = inputs.rhs_ones(A)
    ref, res, x, hist = run_both(ctx, orc, A, b, 1e-10, 600, alg, 1)
    assert res.status == ref.status and res.iters == ref.iters
    assert same(hist, ref.history) and same(x, ref.x)
    ctx.set_option(pbcg.OPT_PRECOND, pbcg.PRECOND_JACOBI)         # the diagonal sums its copies
    try:
        refj = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-10, maxit=600, alg=alg, mode=1, nthreads=8,
                         jacobi=True)
        M = ctx.upload_csr(A)
        xj = np.zeros(A.n)
        rj = ctx.solve(M, b, xj, 1e-10, 600, alg, 1)
        hj = ctx.history()
        M.free()
    finally:
        ctx.set_option(pbcg.OPT_PRECOND, pbcg.PRECOND_NONE)
    assert rj.iters == refj.iters and same(hj, refj.history) and same(xj, refj.x)


@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_zero_rhs_and_empty_row(ctx, orc, alg, mode, small_path):
    n = 100
    A = inputs.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.full(n, 4.0))
    ref, res, x, hist = run_both(ctx, orc, A, np.zeros(n), 1e-12, 10, alg, mode)
    assert res.status == 0 and res.iters == 0 and list(hist) == [0.0] and np.all(x == 0.0)
    ref, res, x, hist = run_both(ctx, orc, A, np.zeros(n), 1e-12, 10, alg, mode, x0=np.ones(n))
    assert res.status == 0 and res.iters == 1 and list(hist) == [40.0, 0.0] and np.all(x == 0.0)
    B = inputs.convdiff2d(9, 12.0)
    b = inputs.rhs_ones(B)
    rp, ci, va = [0], [], []
    p = B.n // 2
    for i in range(B.n + 1):                # an empty row and an unreferenced column at index p
        if i == p:
            rp.append(len(ci))
        if i < B.n:
            for k in range(B.row_ptr[i], B.row_ptr[i + 1]):
                c = int(B.col_idx[k])
                ci.append(c + 1 if c >= p else c)
                va.append(float(B.vals[k]))
            rp.append(len(ci))
    E = inputs.CSR(B.n + 1, np.array(rp, np.int32), np.array(ci, np.int32), np.array(va))
    ref, res, x, hist = run_both(ctx, orc, E, np.insert(b, p, 0.0), 1e-11, 200, alg, mode)
    assert res.status == ref.status and res.iters == ref.iters
    if mode == 1:
        assert same(hist, ref.history) and same(x, ref.x)
    else:
        assert res.status == 0 and res.relres_true <= 1e-11
