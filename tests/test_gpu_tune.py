"""Launch variants and the autotuner (pbcg_set_variant, pbcg_tune).

Every variant -- staged or streamed matrix entries, round-robin or claimed
tiles, one or more resident CTAs per SM, longer or shorter chunks of the
batched tile list -- keeps each SpMV row's fma chain and rounds every exact
dot once from the same integer sum, so exact-mode histories, iteration
counts and x must be bit-identical across variants, on the 128^3 system, a
power-law matrix (wide rows, sorted by length) and a batch of systems.  The
tuner must keep the fastest candidate (never slower than the default as
measured), record it in its JSON-lines cache and take it from there again.
"""
import json

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


def _variants(narrow):
    from paper_2404_13216_gb300 import pbcg
    out = []
    for staged in ((1, 0) if narrow else (1,)):
        for order in (0, 1, 2, 3):
            for ctas in (0, 1):
                out.append(pbcg.Variant(staged, order, ctas, 0))
    return out


def _solve(ctx, M, b, maxit, alg=1, mode=1, tol=1e-300):
    x = np.zeros(M.n)
    r = ctx.solve(M, b, x, tol, maxit, alg, mode)
    return r, ctx.history(), x


@pytest.mark.parametrize("alg", [0, 1])
def test_variants_bitwise_128cubed(ctx, alg):
    A = inputs.convdiff3d(128, 50.0, (1.0, 0.5, 0.25))
    b = inputs.rhs_ones(A)
    M = ctx.upload_csr(A)
    ctx.set_variant(M, None)
    r0, h0, x0 = _solve(ctx, M, b, 40, alg)
    for v in _variants(True):
        ctx.set_variant(M, v)
        assert ctx.get_variant(M).staged == v.staged
        r, h, x = _solve(ctx, M, b, 40, alg)
        assert r.iters == r0.iters == 40 and same(h, h0) and same(x, x0), v
    ctx.set_variant(M, None)
    M.free()


def test_variants_bitwise_powerlaw_and_oracle(ctx, orc):
    A = inputs.powerlaw(n=1 << 17, mean_len=30, max_len=2000, seed=11)
    b = inputs.rhs_ones(A)
    ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-300, maxit=8, alg=1, mode=1, nthreads=16)
    M = ctx.upload_csr(A)
    for v in _variants(False):
        ctx.set_variant(M, v)
        r, h, x = _solve(ctx, M, b, 8)
        assert r.iters == ref.iters and same(h, ref.history) and same(x, ref.x), v
    M.free()


def test_batched_variants_bitwise(ctx):
    from paper_2404_13216_gb300 import pbcg
    B = inputs.batched_convdiff(nsys=48, seed=4)
    b = inputs.rhs_ones(B.A)
    M = ctx.upload_csr(B.A)
    tols = np.full(48, 1e-10)
    got = []
    for c in (0, 1, 3):
        ctx.set_variant(M, pbcg.Variant(1, 0, 0, c))
        x = np.zeros(B.A.n)
        res = ctx.solve_batched(M, B.sys_row_ptr, b, x, tols, 300, pbcg.PIPELINED, pbcg.EXACT)
        got.append(([(r.status, r.iters) for r in res], [ctx.history(k) for k in range(48)], x))
    for st, hs, x in got[1:]:
        assert st == got[0][0] and same(x, got[0][2])
        assert all(same(h, h0) for h, h0 in zip(hs, got[0][1]))
    M.free()


def test_tune_keeps_the_fastest_and_caches(ctx, tmp_path):
    from paper_2404_13216_gb300 import pbcg
    A = inputs.convdiff3d(96, 50.0, (1.0, 0.5, 0.25))
    b = inputs.rhs_ones(A)
    M = ctx.upload_csr(A)
    r0, h0, x0 = _solve(ctx, M, b, 30)
    cache = str(tmp_path / "tune.jsonl")
    chosen, tried = ctx.tune(M, pbcg.PIPELINED, pbcg.EXACT, iters=20, cache_path=cache)
    assert len(tried) == 12
    default = tried[0]
    assert (default.staged, default.order, default.ctas_per_sm) == (1, 0, 0)
    assert chosen.us_per_iter == min(t.us_per_iter for t in tried) <= default.us_per_iter
    cur = ctx.get_variant(M)
    assert (cur.staged, cur.order, cur.ctas_per_sm) == (chosen.staged, chosen.order, chosen.ctas_per_sm)
    r, h, x = _solve(ctx, M, b, 30)
    assert same(h, h0) and same(x, x0)
    rec = [json.loads(line) for line in open(cache)]
    assert len(rec) == 1 and rec[0]["staged"] == chosen.staged and "mode=1" in rec[0]["key"]
    # the cache answers the same key without timing anything
    ctx.set_variant(M, None)
    again, tried2 = ctx.tune(M, pbcg.PIPELINED, pbcg.EXACT, iters=20, cache_path=cache)
    assert tried2 == [] and (again.staged, again.order, again.ctas_per_sm) == \
        (chosen.staged, chosen.order, chosen.ctas_per_sm)
    # plain mode is a key of its own
    pc, pt = ctx.tune(M, pbcg.PIPELINED, pbcg.PLAIN, iters=20, cache_path=cache)
    assert len(pt) == 12 and len(open(cache).readlines()) == 2
    M.free()


def test_tune_batched(ctx, tmp_path):
    from paper_2404_13216_gb300 import pbcg
    B = inputs.batched_convdiff(nsys=32, seed=4)
    M = ctx.upload_csr(B.A)
    chosen, tried = ctx.tune(M, pbcg.PIPELINED, pbcg.EXACT, iters=30, sys_row_ptr=B.sys_row_ptr,
                             cache_path=str(tmp_path / "t.jsonl"))
    assert [t.batched_ctas_per_sm for t in tried] == [0, 1]
    assert chosen.us_per_iter == min(t.us_per_iter for t in tried)
    assert ctx.get_variant(M).batched_ctas_per_sm == chosen.batched_ctas_per_sm
    M.free()


def test_variant_validation(ctx):
    from paper_2404_13216_gb300 import pbcg
    A = inputs.convdiff2d(20, 5.0)
    M = ctx.upload_csr(A)
    for bad in (pbcg.Variant(2, 0, 0, 0), pbcg.Variant(1, 4, 0, 0), pbcg.Variant(1, 0, -1, 0)):
        with pytest.raises(pbcg.PbcgError):
            ctx.set_variant(M, bad)
    with pytest.raises(pbcg.PbcgError):
        ctx.tune(M, pbcg.PIPELINED, pbcg.EXACT, iters=0)
    # a system run by the one-cluster loop keeps its launch: only the default is a candidate
    chosen, tried = ctx.tune(M, pbcg.PIPELINED, pbcg.EXACT, iters=5)
    assert len(tried) == 1 and (chosen.staged, chosen.order, chosen.ctas_per_sm) == (1, 0, 0)
    M.free()
