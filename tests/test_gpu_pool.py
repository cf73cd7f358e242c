"""Pools (continuous batching): systems admitted while others run, each one
retired on its own.  Every system must behave exactly as a solve of its own
-- bit for bit against the CPU oracle in exact mode -- whatever else shares
the launches, and a failing request must not disturb the others."""
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


def systems(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        if k % 3 == 2:
            A = inputs.convdiff3d(int(rng.integers(4, 12)), float(rng.uniform(1, 80)))
        else:
            A = inputs.convdiff2d(int(rng.integers(6, 48)), float(rng.uniform(1, 80)))
        out.append(A)
    return out


def drain(pool, live, got, K, history=False):
    """Step until every slot in `live` has finished; fill got[key] = (x, res, hist)."""
    for _ in range(100000):
        if not live:
            return
        pool.step(K)
        done, _ = pool.poll(wait=True)
        for s in done:
            key = live.pop(s)
            h = pool.history(s) if history else None
            x, r = pool.result(s)
            got[key] = (x, r, h)
    raise AssertionError("pool did not finish")


@pytest.mark.parametrize("alg", [0, 1, 2], ids=["bicgstab", "pbicgstab", "pbicgstab_rr"])
def test_pool_exact_staggered_matches_oracle(ctx, orc, alg):
    """Requests arrive between steps of uneven length; each result equals the oracle's bit for bit."""
    from paper_2404_13216_gb300 import pbcg
    syst = systems(11 + alg, 10)
    tols = [1e-10 if k % 2 else 1e-8 for k in range(len(syst))]
    if alg == 2:
        ctx.set_option(pbcg.OPT_RR_PERIOD, 7)
    pool = pbcg.Pool(ctx, max_rows=6 * 2048, max_entries=6 * 2048 * 16, max_slots=5, maxit=3000, alg=alg,
                     mode=pbcg.EXACT)
    live, got, queue = {}, {}, list(range(len(syst)))
    steps = [1, 3, 2, 5, 1, 4]
    it = 0
    while queue or live:
        while queue:
            A = syst[queue[0]]
            s = pool.admit(A, inputs.rhs_ones(A), tol=tols[queue[0]], maxit=3000)
            if s is None:
                break
            live[s] = queue.pop(0)
        pool.step(steps[it % len(steps)])
        it += 1
        done, _ = pool.poll(wait=(it % 2 == 0))
        for s in done:
            key = live.pop(s)
            h = pool.history(s)
            x, r = pool.result(s)
            got[key] = (x, r, h)
        assert it < 20000
    pool.close()
    if alg == 2:
        ctx.set_option(pbcg.OPT_RR_PERIOD, 50)
    for k, A in enumerate(syst):
        ref = orc.solve(A.row_ptr, A.col_idx, A.vals, inputs.rhs_ones(A), tol=tols[k], maxit=3000,
                        alg=min(alg, 1), mode=1, rr_period=7 if alg == 2 else 0)
        x, r, h = got[k]
        assert r.status == ref.status and r.iters == ref.iters, (k, r, ref.status, ref.iters)
        assert same(h, ref.history), k
        assert same(x, ref.x), k
        assert same([r.relres_true], [ref.relres_true]), k


def test_pool_alone_equals_in_mix(ctx):
    """One request solved alone in a pool and amid others: identical bits (exact)."""
    from paper_2404_13216_gb300 import pbcg
    syst = systems(5, 7)
    target = inputs.convdiff2d(40, 33.0)
    b = inputs.rhs_ones(target)

    def run(with_others):
        pool = pbcg.Pool(ctx, max_rows=10 * 2048, max_entries=10 * 2048 * 16, max_slots=8, maxit=2000)
        live, got = {}, {}
        if with_others:
            for k, A in enumerate(syst[:3]):
                live[pool.admit(A, inputs.rhs_ones(A), tol=1e-10, maxit=2000)] = k
            pool.step(3)
        live[pool.admit(target, b, tol=1e-10, maxit=2000)] = "t"
        if with_others:
            for k, A in enumerate(syst[3:], start=3):
                live[pool.admit(A, inputs.rhs_ones(A), tol=1e-10, maxit=2000)] = k
        drain(pool, live, got, 4, history=True)
        pool.close()
        return got["t"]

    xa, ra, ha = run(False)
    xb, rb, hb = run(True)
    assert ra.status == rb.status == 0 and ra.iters == rb.iters
    assert same(xa, xb) and same(ha, hb)
    # and equal to a single solve on the same context
    M = ctx.upload_csr(target)
    xs = np.zeros(target.n)
    rs = ctx.solve(M, b, xs, 1e-10, 2000, 1, 1)
    M.free()
    assert rs.iters == ra.iters and same(xs, xa) and same(ctx.history(), ha)


def test_pool_plain_converges(ctx):
    from paper_2404_13216_gb300 import pbcg
    syst = systems(9, 6)
    pool = pbcg.Pool(ctx, max_rows=8 * 2048, max_entries=8 * 2048 * 16, max_slots=6, maxit=3000, mode=pbcg.PLAIN)
    live, got = {}, {}
    for k, A in enumerate(syst):
        live[pool.admit(A, inputs.rhs_ones(A), tol=1e-8, maxit=3000)] = k
    drain(pool, live, got, 6)
    pool.close()
    for k in range(len(syst)):
        x, r, _ = got[k]
        assert r.status == 0 and r.relres_true <= 1e-8, (k, r)
        assert np.max(np.abs(x - 1.0)) < 1e-3


def test_pool_failures_stay_isolated(ctx, orc):
    """A NaN right-hand side, a column index out of range, a one-row system and
    a maxit-limited system finish on their own; the others match the oracle."""
    from paper_2404_13216_gb300 import pbcg
    good = [inputs.convdiff2d(12, 5.0), inputs.convdiff2d(20, 60.0)]
    nan_A = inputs.convdiff2d(9, 30.0)
    b_nan = inputs.rhs_ones(nan_A)
    b_nan[3] = np.nan
    bad_A = inputs.convdiff2d(8, 3.0)
    bad_ci = bad_A.col_idx.copy()
    bad_ci[5] = bad_A.n + 7
    bad = inputs.CSR(bad_A.n, bad_A.row_ptr, bad_ci, bad_A.vals)
    one = inputs.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.0]))
    pool = pbcg.Pool(ctx, max_rows=8 * 256, max_entries=8 * 256 * 16, max_slots=6, maxit=40)
    live, got = {}, {}
    live[pool.admit(good[0], inputs.rhs_ones(good[0]), tol=1e-10, maxit=40)] = "g0"
    live[pool.admit(nan_A, b_nan, tol=1e-10, maxit=40)] = "nan"
    live[pool.admit(bad, inputs.rhs_ones(bad_A), tol=1e-10, maxit=40)] = "bad"
    live[pool.admit(one, np.array([3.0]), tol=1e-12, maxit=40)] = "one"
    live[pool.admit(good[1], inputs.rhs_ones(good[1]), tol=1e-10, maxit=25)] = "g1"
    drain(pool, live, got, 5)
    pool.close()
    assert got["nan"][1].status == pbcg.NONFINITE
    assert got["bad"][1].status == pbcg.ERR_INVALID
    assert got["one"][1].status == 0 and got["one"][0][0] == 1.5
    for key, A, mx in (("g0", good[0], 40), ("g1", good[1], 25)):
        ref = orc.solve(A.row_ptr, A.col_idx, A.vals, inputs.rhs_ones(A), tol=1e-10, maxit=mx, alg=1, mode=1)
        x, r, _ = got[key]
        assert r.status == ref.status and r.iters == ref.iters and same(x, ref.x), key


def test_pool_room_and_reuse(ctx, orc):
    """No room -> None; retiring frees the room; a slot reused by a new request
    is never reported with its previous occupant's state."""
    from paper_2404_13216_gb300 import pbcg
    A = inputs.convdiff2d(30, 10.0)       # 900 rows -> 4 tiles
    b = inputs.rhs_ones(A)
    pool = pbcg.Pool(ctx, max_rows=4 * 256, max_entries=4 * 256 * 8, max_slots=2, maxit=500)
    s0 = pool.admit(A, b, tol=1e-10, maxit=500)
    assert s0 is not None
    assert pool.admit(A, b, tol=1e-10, maxit=500) is None        # tiles exhausted
    assert pool.room()[1] == 0
    with pytest.raises(pbcg.PbcgError):
        pool.result(s0)                                            # not finished
    got = {}
    drain(pool, {s0: 0}, got, 50)
    fs, fr, fe = pool.room()
    assert fs == 2 and fr == 4 * 256 and fe == 4 * 256 * 8
    ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-10, maxit=500, alg=1, mode=1)
    B = inputs.convdiff2d(25, 70.0)
    bb = inputs.rhs_ones(B)
    s1 = pool.admit(B, bb, tol=1e-10, maxit=500)
    assert s1 == s0
    done, _ = pool.poll(wait=True)            # snapshots from before the admission are stale for this slot
    assert done == []
    drain(pool, {s1: 1}, got, 7)
    pool.close()
    refB = orc.solve(B.row_ptr, B.col_idx, B.vals, bb, tol=1e-10, maxit=500, alg=1, mode=1)
    assert got[0][1].iters == ref.iters and same(got[0][0], ref.x)
    assert got[1][1].iters == refB.iters and same(got[1][0], refB.x)


def test_pool_invalid_arguments(ctx):
    from paper_2404_13216_gb300 import pbcg
    with pytest.raises(pbcg.PbcgError):
        pbcg.Pool(ctx, max_rows=0, max_entries=10, max_slots=1, maxit=10)
    with pytest.raises(pbcg.PbcgError):
        pbcg.Pool(ctx, max_rows=256, max_entries=10, max_slots=1, maxit=10, alg=7)
    with pytest.raises(pbcg.PbcgError) as e:
        pbcg.Pool(ctx, max_rows=256, max_entries=10, max_slots=1, maxit=2 ** 31 - 1)
    assert e.value.code == pbcg.ERR_INVALID
    pool = pbcg.Pool(ctx, max_rows=512, max_entries=4096, max_slots=2, maxit=10, max_request_rows=300,
                     max_request_nnz=2000)
    A = inputs.convdiff2d(18, 5.0)       # 324 rows: beyond max_request_rows
    with pytest.raises(pbcg.PbcgError):
        pool.admit(A, inputs.rhs_ones(A), tol=1e-8, maxit=10)
    A = inputs.convdiff2d(10, 5.0)
    with pytest.raises(pbcg.PbcgError):
        pool.admit(A, inputs.rhs_ones(A), tol=1e-8, maxit=11)      # maxit above the pool's
    with pytest.raises(pbcg.PbcgError):
        pool.admit(A, inputs.rhs_ones(A), tol=0.0, maxit=10)
    rp = A.row_ptr.copy()
    rp[3], rp[4] = rp[4], rp[3]
    with pytest.raises(pbcg.PbcgError):
        pool.admit(inputs.CSR(A.n, rp, A.col_idx, A.vals), inputs.rhs_ones(A), tol=1e-8, maxit=10)
    with pytest.raises(pbcg.PbcgError):
        pool.step(0)
    pool.close()


def test_pool_out_of_memory_leaves_context_usable(ctx, orc):
    """A pool whose residual histories cannot be allocated (2^20 slots x
    (2^30 + 1) iterations, about 9 PB) is refused with OOM; what it had taken
    is released, and the context still solves exactly, alone and in a pool."""
    from paper_2404_13216_gb300 import pbcg
    with pytest.raises(pbcg.PbcgError) as e:
        pbcg.Pool(ctx, max_rows=256, max_entries=2048, max_slots=1 << 20, maxit=1 << 30)
    assert e.value.code == pbcg.ERR_OOM
    A = inputs.convdiff2d(12, 20.0)
    b = inputs.rhs_ones(A)
    ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-10, maxit=300, alg=1, mode=1)
    M = ctx.upload_csr(A)
    x = np.zeros(A.n)
    r = ctx.solve(M, b, x, 1e-10, 300, pbcg.PIPELINED, pbcg.EXACT)
    M.free()
    assert r.iters == ref.iters and same(x, ref.x)
    with pbcg.Pool(ctx, max_rows=1024, max_entries=8192, max_slots=2, maxit=300) as pool:
        s = pool.admit(A, b, tol=1e-10, maxit=300)
        got = {}
        drain(pool, {s: 0}, got, 16)
    assert got[0][1].iters == ref.iters and same(got[0][0], ref.x)


def test_pool_and_batch_irregular_rows(ctx, orc):
    """Random power-law rows (some wider than a tile can stage) in a pool and in
    a batched solve: each system equals the oracle bit for bit (exact)."""
    from paper_2404_13216_gb300 import pbcg
    syst = [inputs.powerlaw(n=n, mean_len=12.0, max_len=300, seed=s) for n, s in ((700, 1), (1500, 2), (300, 3))]
    syst.append(inputs.convdiff3d(9, 40.0))
    refs = [orc.solve(A.row_ptr, A.col_idx, A.vals, inputs.rhs_ones(A), tol=1e-10, maxit=400, alg=1, mode=1)
            for A in syst]
    pool = pbcg.Pool(ctx, max_rows=16 * 256, max_entries=1 << 20, max_slots=4, maxit=400)
    live, got = {}, {}
    for k, A in enumerate(syst):
        live[pool.admit(A, inputs.rhs_ones(A), tol=1e-10, maxit=400)] = k
    drain(pool, live, got, 5)
    pool.close()
    for k, ref in enumerate(refs):
        x, r, _ = got[k]
        assert r.status == ref.status and r.iters == ref.iters and same(x, ref.x), k
    A, srp = inputs.block_diag(syst)
    b = inputs.rhs_ones(A)
    M = ctx.upload_csr(A)
    x = np.zeros(A.n)
    res = ctx.solve_batched(M, srp, b, x, np.full(len(syst), 1e-10), 400, 1, 1)
    M.free()
    for k, ref in enumerate(refs):
        assert res[k].status == ref.status and res[k].iters == ref.iters, k
        assert same(x[srp[k]:srp[k + 1]], ref.x), k


@pytest.mark.parametrize("alg", [0, 1, 2], ids=["bicgstab", "pbicgstab", "pbicgstab_rr"])
def test_pool_jacobi_matches_oracle(ctx, orc, alg):
    """A pool created with Jacobi preconditioning: every request, with a nonzero
    x0, equals the oracle's right-Jacobi solve bit for bit; a request whose
    diagonal has a zero finishes INVALID without touching the others."""
    from paper_2404_13216_gb300 import pbcg
    syst = systems(31 + alg, 6)
    if alg == 2:
        ctx.set_option(pbcg.OPT_RR_PERIOD, 7)
    pool = pbcg.Pool(ctx, max_rows=6 * 2048, max_entries=6 * 2048 * 16, max_slots=4, maxit=2000, alg=alg,
                     mode=pbcg.EXACT, precond=pbcg.PRECOND_JACOBI)
    rng = np.random.default_rng(3)
    x0s = [rng.standard_normal(A.n) for A in syst]
    # a request whose row 3 has no diagonal entry
    bad = inputs.convdiff2d(12, 4.0)
    keep = [k for k in range(bad.row_ptr[3], bad.row_ptr[4]) if bad.col_idx[k] != 3]
    rows = [list(range(bad.row_ptr[i], bad.row_ptr[i + 1])) if i != 3 else keep for i in range(bad.n)]
    idx = [k for r in rows for k in r]
    rp = np.zeros(bad.n + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    bad = inputs.CSR(bad.n, rp, bad.col_idx[idx].astype(np.int32), bad.vals[idx])
    live, got, queue = {}, {}, list(range(len(syst))) + ["bad"]
    it = 0
    while queue or live:
        while queue:
            key = queue[0]
            A = bad if key == "bad" else syst[key]
            s = pool.admit(A, inputs.rhs_ones(A), tol=1e-10, maxit=2000, x0=None if key == "bad" else x0s[key])
            if s is None:
                break
            live[s] = queue.pop(0)
        pool.step(4)
        it += 1
        done, _ = pool.poll(wait=True)
        for s in done:
            key = live.pop(s)
            h = pool.history(s)
            x, r = pool.result(s)
            got[key] = (x, r, h)
        assert it < 20000
    pool.close()
    if alg == 2:
        ctx.set_option(pbcg.OPT_RR_PERIOD, 50)
    assert got["bad"][1].status == -1 and got["bad"][1].iters == 0, got["bad"][1]      # PBCG_ERR_INVALID
    for k, A in enumerate(syst):
        ref = orc.solve(A.row_ptr, A.col_idx, A.vals, inputs.rhs_ones(A), x0=x0s[k], tol=1e-10, maxit=2000,
                        alg=min(alg, 1), mode=1, jacobi=True, rr_period=7 if alg == 2 else 0)
        x, r, h = got[k]
        assert r.status == ref.status and r.iters == ref.iters, (k, r, ref.status, ref.iters)
        assert same(h, ref.history), k
        assert same(x, ref.x), k
