"""Batched solves (many independent systems in one block-diagonal matrix):
every system must behave exactly as a solve of its own block -- bit for bit
against the CPU oracle in exact mode -- and stop on its own."""
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


def small_batch(seed=7, nsys=9):
    rng = np.random.default_rng(seed)
    systems = []
    for k in range(nsys):
        side = int(rng.integers(5, 40))
        pe = float(rng.uniform(1, 80))
        A = inputs.convdiff2d(side, pe) if k % 3 else inputs.convdiff3d(max(3, side // 4), pe)
        systems.append(A)
    A, srp = inputs.block_diag(systems)
    b = inputs.rhs_ones(A)
    return systems, A, srp, b


@pytest.mark.parametrize("alg", [0, 1], ids=["bicgstab", "pbicgstab"])
def test_batched_exact_matches_oracle_per_system(ctx, orc, alg):
    systems, A, srp, b = small_batch()
    tol = np.array([1e-8 if k % 2 else 1e-10 for k in range(len(systems))])
    M = ctx.upload_csr(A)
    x = np.zeros(A.n)
    res = ctx.solve_batched(M, srp, b, x, tol, 3000, alg, 1)
    for k, S in enumerate(systems):
        r0, r1 = srp[k], srp[k + 1]
        ref = orc.solve(S.row_ptr, S.col_idx, S.vals, b[r0:r1], tol=tol[k], maxit=3000, alg=alg, mode=1)
        assert res[k].status == ref.status and res[k].iters == ref.iters, (k, res[k], ref.status, ref.iters)
        assert same(ctx.history(k), ref.history), k
        assert same(x[r0:r1], ref.x), k
        assert same([res[k].relres_true], [ref.relres_true]), k
    M.free()


@pytest.mark.parametrize("alg", [0, 1], ids=["bicgstab", "pbicgstab"])
def test_batched_plain_converges(ctx, alg):
    systems, A, srp, b = small_batch(seed=3, nsys=6)
    tol = np.full(len(systems), 1e-8)
    M = ctx.upload_csr(A)
    x = np.zeros(A.n)
    res = ctx.solve_batched(M, srp, b, x, tol, 3000, alg, 0)
    for k in range(len(systems)):
        assert res[k].status == 0 and res[k].relres_true <= 1e-8, (k, res[k])
        assert np.max(np.abs(x[srp[k]:srp[k + 1]] - 1.0)) < 1e-3
    M.free()


def test_batched_isolation_and_edge_systems(ctx, orc):
    """A NaN in one system, a system solved at x0, a one-row system and a
    maxit-limited system do not disturb the others."""
    systems = [inputs.convdiff2d(12, 5.0), inputs.convdiff2d(9, 30.0),
               inputs.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.0])),
               inputs.convdiff2d(20, 60.0)]
    A, srp = inputs.block_diag(systems)
    b = inputs.rhs_ones(A)
    b[srp[1] + 3] = np.nan
    x0 = np.zeros(A.n)
    x0[srp[3]:srp[4]] = 0.5
    tol = np.array([1e-10, 1e-10, 1e-12, 1e-10])
    M = ctx.upload_csr(A)
    x = x0.copy()
    res = ctx.solve_batched(M, srp, b, x, tol, 25, 1, 1)
    assert res[1].status == 3
    for k in (0, 2, 3):
        r0, r1 = srp[k], srp[k + 1]
        S = systems[k]
        ref = orc.solve(S.row_ptr, S.col_idx, S.vals, b[r0:r1], x0=x0[r0:r1], tol=tol[k], maxit=25, alg=1, mode=1)
        assert res[k].status == ref.status and res[k].iters == ref.iters, (k, res[k], ref.status)
        assert same(x[r0:r1], ref.x)
    M.free()


def test_batched_invalid(ctx):
    from paper_2404_13216_gb300 import pbcg
    systems = [inputs.convdiff2d(6, 5.0), inputs.convdiff2d(5, 5.0)]
    A, srp = inputs.block_diag(systems)
    b = inputs.rhs_ones(A)
    M = ctx.upload_csr(A)
    with pytest.raises(pbcg.PbcgError):
        ctx.solve_batched(M, np.array([0, 10, A.n - 1], np.int32), b, np.zeros(A.n), np.full(2, 1e-8), 10)
    with pytest.raises(pbcg.PbcgError):          # boundary cuts through a block: off-block entries
        ctx.solve_batched(M, np.array([0, 30, A.n], np.int32), b, np.zeros(A.n), np.full(2, 1e-8), 10)
    with pytest.raises(pbcg.PbcgError):
        ctx.solve_batched(M, srp, b, np.zeros(A.n), np.array([1e-8, 0.0]), 10)
    with pytest.raises(pbcg.PbcgError) as e:
        ctx.solve_batched(M, srp, b, np.zeros(A.n), np.full(2, 1e-8), 2 ** 31 - 1)
    assert e.value.code == pbcg.ERR_INVALID
    M.free()


def test_batched_config_sample_bitwise_vs_single(ctx):
    """A 24-system sample of the 512-system configuration: the batched solve
    equals single solves of each block on the GPU, bit for bit (exact)."""
    B = inputs.batched_convdiff(nsys=24, side_lo=32, side_hi=96, seed=11)
    b = inputs.rhs_ones(B.A)
    tol = np.full(B.nsys, 1e-10)
    M = ctx.upload_csr(B.A)
    x = np.zeros(B.A.n)
    res = ctx.solve_batched(M, B.sys_row_ptr, b, x, tol, 20000, 1, 1)
    hb = [ctx.history(k) for k in range(B.nsys)]
    M.free()
    for k in range(B.nsys):
        r0, r1 = B.sys_row_ptr[k], B.sys_row_ptr[k + 1]
        S = inputs.convdiff2d(int(B.sides[k]), float(B.peclet[k]))
        Ms = ctx.upload_csr(S)
        xs = np.zeros(S.n)
        rs = ctx.solve(Ms, b[r0:r1], xs, 1e-10, 20000, 1, 1)
        assert rs.iters == res[k].iters and rs.status == res[k].status
        assert same(ctx.history(), hb[k]) and same(xs, x[r0:r1])
        Ms.free()


def test_batched_residual_replacement_bitwise(ctx, orc):
    from paper_2404_13216_gb300 import pbcg
    systems, A, srp, b = small_batch(seed=21, nsys=5)
    tol = np.full(len(systems), 1e-12)
    ctx.set_option(pbcg.OPT_RR_PERIOD, 10)
    M = ctx.upload_csr(A)
    x = np.zeros(A.n)
    res = ctx.solve_batched(M, srp, b, x, tol, 2000, pbcg.PIPELINED_RR, 1)
    for k, S in enumerate(systems):
        r0, r1 = srp[k], srp[k + 1]
        ref = orc.solve(S.row_ptr, S.col_idx, S.vals, b[r0:r1], tol=1e-12, maxit=2000, alg=1, mode=1, rr_period=10)
        assert res[k].status == ref.status and res[k].iters == ref.iters, k
        assert same(ctx.history(k), ref.history) and same(x[r0:r1], ref.x), k
    M.free()
    ctx.set_option(pbcg.OPT_RR_PERIOD, 50)


@pytest.mark.parametrize("alg", [0, 1, 2], ids=["bicgstab", "pbicgstab", "pbicgstab_rr"])
def test_batched_host_loop_equals_graph(ctx, alg):
    """PBCG_OPT_BATCH_GRAPH = 0 (host-driven launches, for profilers) gives the
    graph loop's results bit for bit, statuses and iteration counts included."""
    from paper_2404_13216_gb300 import pbcg
    systems, A, srp, b = small_batch(seed=11, nsys=7)
    tol = np.full(len(systems), 1e-10)
    M = ctx.upload_csr(A)
    out = []
    for graph in (1, 0):
        ctx.set_option(pbcg.OPT_BATCH_GRAPH, graph)
        try:
            x = np.zeros(A.n)
            res = ctx.solve_batched(M, srp, b, x, tol, 400, alg, 1)
            hist = [ctx.history(k) for k in range(len(systems))]
        finally:
            ctx.set_option(pbcg.OPT_BATCH_GRAPH, 1)
        out.append((res, x, hist))
    (rg, xg, hg), (rh, xh, hh) = out
    assert [(r.status, r.iters) for r in rg] == [(r.status, r.iters) for r in rh]
    assert same(xg, xh)
    assert all(same(a, b_) for a, b_ in zip(hg, hh))
    M.free()
