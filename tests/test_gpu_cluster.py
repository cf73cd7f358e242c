"""Small systems through the one-launch cluster loops of Algorithms 1 and 2.

pbcg_solve runs BiCGStab and p-BiCGStab on a system of at most 16384 rows as
one launch over a thread-block cluster (PBCG_OPT_SMALL_CLUSTER, on by
default).  Exact mode must be bit-identical to the oracle and to the launch
graph of passes (the option off); plain mode must meet the same tolerance
bars as the passes.
"""
import numpy as np
import pytest

from paper_2404_13216_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def solve(ctx, A, b, tol, maxit, mode, cluster, x0=None, alg=1):
    from paper_2404_13216_gb300 import pbcg
    ctx.set_option(pbcg.OPT_SMALL_CLUSTER, 1 if cluster else 0)
    try:
        M = ctx.upload_csr(A)
        x = np.zeros(A.n) if x0 is None else np.array(x0, dtype=np.float64)
        r = ctx.solve(M, b, x, tol, maxit, alg, mode)
        h = ctx.history()
        M.free()
    finally:
        ctx.set_option(pbcg.OPT_SMALL_CLUSTER, 1)
    return r, x, h


# sizes: one CTA, a ragged few, 16 CTAs x 1 row per thread, 14 x 4 (ragged),
# 16 x 4 (the largest), and one row past it (two-pass graph)
SYSTEMS = {
    "2d5": lambda: inputs.convdiff2d(5, 3.0),            # n = 25
    "2d37": lambda: inputs.convdiff2d(37, 40.0),         # n = 1369
    "2d64": lambda: inputs.convdiff2d(64, 10.0),         # n = 4096
    "3d24": lambda: inputs.convdiff3d(24, 50.0),         # n = 13824
    "2d128": lambda: inputs.convdiff2d(128, 20.0),       # n = 16384
}


@pytest.mark.parametrize("alg", [0, 1], ids=["bicgstab", "pbicgstab"])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_cluster_exact_bitwise_vs_oracle_and_passes(ctx, orc, name, alg):
    A = SYSTEMS[name]()
    b = inputs.rhs_ones(A)
    ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-10, maxit=600, alg=alg, mode=1, nthreads=8)
    rc, xc, hc = solve(ctx, A, b, 1e-10, 600, 1, True, alg=alg)
    rp, xp, hp = solve(ctx, A, b, 1e-10, 600, 1, False, alg=alg)
    assert rc.status == ref.status and rc.iters == ref.iters, (rc, ref.status, ref.iters)
    assert same(hc, ref.history) and same(xc, ref.x)
    assert same([rc.relres_true], [ref.relres_true])
    assert rp.iters == rc.iters and same(hp, hc) and same(xp, xc)
    # the cluster loop is one launch per stop test; the graph counts every pass
    assert rc.launches < rp.launches


def test_cluster_limit_and_past_it(ctx, orc):
    """16384 rows take the cluster loop, 16385 rows the pass graph; both exact."""
    for n_extra, expect_cluster in ((0, True), (1, False)):
        A0 = inputs.convdiff2d(128, 20.0)
        n = A0.n + n_extra
        if n_extra:
            # append one decoupled unknown 2 x = 2
            rp = np.concatenate([A0.row_ptr, [A0.row_ptr[-1] + 1]]).astype(np.int32)
            ci = np.concatenate([A0.col_idx, [n - 1]]).astype(np.int32)
            va = np.concatenate([A0.vals, [2.0]])
            A = inputs.CSR(n, rp, ci, va)
        else:
            A = A0
        b = inputs.rhs_ones(A)
        ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-9, maxit=60, alg=1, mode=1, nthreads=8)
        r, x, h = solve(ctx, A, b, 1e-9, 60, 1, True)
        assert r.iters == ref.iters and same(h, ref.history) and same(x, ref.x)
        # a cluster solve is setup (3 launches), the loop (1 per stop test) and the true residual
        assert (r.launches <= 8) == expect_cluster, r.launches


@pytest.mark.parametrize("alg", [0, 1], ids=["bicgstab", "pbicgstab"])
def test_cluster_plain(ctx, orc, alg):
    A = SYSTEMS["2d64"]()
    b = inputs.rhs_ones(A)
    tol = 1e-8
    ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=tol, maxit=2000, alg=alg, mode=0, nthreads=1)
    r, x, h = solve(ctx, A, b, tol, 2000, 0, True, alg=alg)
    assert r.status == 0 and r.relres_true <= tol
    k = min(21, h.size, ref.history.size)
    rel = np.abs(h[:k] - ref.history[:k]) / np.abs(ref.history[:k])
    assert np.all(rel <= 1e-8), rel.max()


def test_cluster_jacobi_and_stops(ctx, orc):
    from paper_2404_13216_gb300 import pbcg
    A = inputs.convdiff2d(40, 30.0)
    b = inputs.rhs_ones(A)
    # right Jacobi through the cluster loop equals the oracle's
    ctx.set_option(pbcg.OPT_PRECOND, pbcg.PRECOND_JACOBI)
    try:
        ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-10, maxit=500, alg=1, mode=1, nthreads=8,
                        jacobi=True)
        r, x, h = solve(ctx, A, b, 1e-10, 500, 1, True)
    finally:
        ctx.set_option(pbcg.OPT_PRECOND, pbcg.PRECOND_NONE)
    assert r.iters == ref.iters and same(h, ref.history) and same(x, ref.x)
    # maxit stop inside the loop, and a NaN that stops it at once
    ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-14, maxit=7, alg=1, mode=1, nthreads=8)
    r, x, h = solve(ctx, A, b, 1e-14, 7, 1, True)
    assert r.status == ref.status == 1 and r.iters == 7 and same(x, ref.x)
    bn = b.copy()
    bn[11] = np.inf
    ref = orc.solve(A.row_ptr, A.col_idx, A.vals, bn, tol=1e-10, maxit=20, alg=1, mode=1, nthreads=8)
    r, x, h = solve(ctx, A, bn, 1e-10, 20, 1, True)
    assert r.status == ref.status and r.iters == ref.iters


def test_cluster_option_validation(ctx):
    from paper_2404_13216_gb300 import pbcg
    with pytest.raises(Exception):
        ctx.set_option(pbcg.OPT_SMALL_CLUSTER, 2)
    ctx.set_option(pbcg.OPT_SMALL_CLUSTER, 0)
    ctx.set_option(pbcg.OPT_SMALL_CLUSTER, 1)


@pytest.mark.parametrize("alg", [0, 1], ids=["bicgstab", "pbicgstab"])
def test_cluster_nonzero_x0_and_ragged_sizes(ctx, orc, alg):
    """A nonzero initial guess, and sizes one row past a CTA's share (4097 rows:
    2 rows per thread over 9 CTAs) and a prime (3001 rows)."""
    for n_target, seed in ((4097, 1), (3001, 2)):
        base = inputs.convdiff2d(int(np.ceil(np.sqrt(n_target))), 25.0)
        # keep the leading n_target rows and columns (a principal block stays nonsingular: diagonally dominant)
        m = n_target
        rp, ci, va = [0], [], []
        for i in range(m):
            for k in range(base.row_ptr[i], base.row_ptr[i + 1]):
                if base.col_idx[k] < m:
                    ci.append(int(base.col_idx[k]))
                    va.append(float(base.vals[k]))
            rp.append(len(ci))
        A = inputs.CSR(m, np.array(rp, np.int32), np.array(ci, np.int32), np.array(va))
        b = inputs.rhs_ones(A)
        x0 = np.random.default_rng(seed).standard_normal(m)
        ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, x0=x0, tol=1e-10, maxit=800, alg=alg, mode=1, nthreads=8)
        r, x, h = solve(ctx, A, b, 1e-10, 800, 1, True, x0=x0, alg=alg)
        assert r.status == ref.status and r.iters == ref.iters, (n_target, r, ref.status, ref.iters)
        assert same(h, ref.history) and same(x, ref.x), n_target
