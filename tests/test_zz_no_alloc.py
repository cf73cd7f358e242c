"""pbcg_dot_noalloc: the dot product for callers that cannot allocate device
memory (inside another allocator's arena, under a fixed memory budget, or in
a loop that must not enter the allocator).  It takes device inputs and a
device output, keeps its merge state in a fixed static device array, and must
agree with the context-based pbcg_dot: bit for bit in exact mode, within the
plain-dot tolerance of the other tests in plain mode, on two calls in a row.
In exact mode it is also held to the CPU oracle's correctly rounded dot on
the adversarial cases and the random exponent sweep of the parity tests.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2404_13216_gb300 import build
    build.build_library()
    from paper_2404_13216_gb300 import pbcg
    ctx = pbcg.Context(0)
    yield torch, pbcg, ctx
    ctx.close()


def _inputs(torch, seed, n):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(n) * np.ldexp(1.0, rng.integers(-60, 60, n))
    b = rng.standard_normal(n) * np.ldexp(1.0, rng.integers(-200, 200, n))
    return a, b, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()


@pytest.mark.parametrize("n", [0, 1, 33, 4097, 1_000_003])
def test_noalloc_matches_context_dot_twice(env, n):
    torch, pbcg, ctx = env
    for call in range(2):
        a, b, da, db = _inputs(torch, 100 + call, n)
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        assert pbcg.dot_noalloc(da, db, out[0:1], pbcg.EXACT, stream) == 0
        assert pbcg.dot_noalloc(da, db, out[1:2], pbcg.PLAIN, stream) == 0
        torch.cuda.synchronize()
        got_exact, got_plain = out.cpu().numpy()
        want_exact = ctx.dot(da, db, pbcg.EXACT)
        want_plain = ctx.dot(da, db, pbcg.PLAIN)
        assert np.array_equal(np.array([got_exact]).view(np.int64), np.array([want_exact]).view(np.int64))
        assert abs(got_plain - want_plain) <= 1e-12 * float(np.abs(a * b).sum()) + 0.0


def _exact_noalloc(torch, pbcg, a, b):
    da = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    db = torch.from_numpy(np.ascontiguousarray(b, dtype=np.float64)).cuda()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    assert pbcg.dot_noalloc(da, db, out, pbcg.EXACT) == 0
    torch.cuda.synchronize()
    return float(out.item())


def _same(got, want):
    if math.isnan(want):
        return math.isnan(got)
    return np.array_equal(np.array([got]).view(np.int64), np.array([want]).view(np.int64))


def test_noalloc_exact_matches_oracle_adversarial(env, orc):
    """Cancellation, ties, subnormal results, products whose FMA error term
    underflows, overflow: every case correctly rounded, as the oracle's
    big-integer sum gives it."""
    from tests import dotcases
    torch, pbcg, ctx = env
    for name, a, b in dotcases.cases(0):
        got = _exact_noalloc(torch, pbcg, a, b)
        assert _same(got, orc.dot_exact(a, b)), name


def test_noalloc_exact_matches_oracle_sweep(env, orc):
    """60 seeded cases: ragged lengths, exponent spans from narrow to the
    whole double range, exact zeros and planted cancellation."""
    torch, pbcg, ctx = env
    rng = np.random.default_rng(77)
    for case in range(60):
        n = int(rng.integers(1, 5000))
        lo = int(rng.integers(-1074, 900))
        hi = int(min(1000, lo + rng.integers(0, 2000)))
        ea = rng.integers(lo, hi + 1, n) // 2
        eb = rng.integers(lo, hi + 1, n) - ea
        a = np.ldexp(rng.uniform(0.5, 1.0, n), ea) * rng.choice([-1.0, 1.0], n)
        b = np.ldexp(rng.uniform(0.5, 1.0, n), np.clip(eb, -1074, 1000)) * rng.choice([-1.0, 1.0], n)
        a[rng.random(n) < 0.05] = 0.0
        if case % 3 == 0 and n > 1:
            h = n // 2
            a[h:2 * h] = -a[:h]
            b[h:2 * h] = b[:h]
        got = _exact_noalloc(torch, pbcg, a, b)
        want = orc.dot_exact(a, b, nthreads=4)
        assert _same(got, want) or (got == 0.0 and want == 0.0), (case, n, got, want)


def test_noalloc_nonfinite_then_clean(env):
    torch, pbcg, ctx = env
    a = torch.ones(100, dtype=torch.float64, device="cuda")
    a[7] = float("inf")
    b = torch.ones(100, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert pbcg.dot_noalloc(a, b, out, pbcg.EXACT) == 0
    torch.cuda.synchronize()
    assert math.isnan(out.item())
    a[7] = 1.0
    assert pbcg.dot_noalloc(a, b, out, pbcg.EXACT) == 0
    torch.cuda.synchronize()
    assert out.item() == 100.0


def test_noalloc_rejects_bad_arguments(env):
    torch, pbcg, ctx = env
    import ctypes
    lib = pbcg._lib
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    a = torch.ones(4, dtype=torch.float64, device="cuda")
    assert lib.pbcg_dot_noalloc(-1, pbcg._ptr(a), pbcg._ptr(a), 1, pbcg._ptr(out), None) == pbcg.ERR_INVALID
    assert lib.pbcg_dot_noalloc(1 << 31, pbcg._ptr(a), pbcg._ptr(a), 1, pbcg._ptr(out), None) == pbcg.ERR_INVALID
    assert lib.pbcg_dot_noalloc(4, None, pbcg._ptr(a), 1, pbcg._ptr(out), None) == pbcg.ERR_INVALID
    assert lib.pbcg_dot_noalloc(4, pbcg._ptr(a), pbcg._ptr(a), 1, None, None) == pbcg.ERR_INVALID
    assert lib.pbcg_dot_noalloc(4, pbcg._ptr(a), pbcg._ptr(a), 5, pbcg._ptr(out), None) == pbcg.ERR_INVALID
    # host memory is refused by the library itself (checked before any launch)
    h = np.ones(4)
    hp = h.ctypes.data_as(ctypes.c_void_p)
    assert lib.pbcg_dot_noalloc(4, hp, pbcg._ptr(a), 1, pbcg._ptr(out), None) == pbcg.ERR_INVALID
    assert lib.pbcg_dot_noalloc(4, pbcg._ptr(a), hp, 1, pbcg._ptr(out), None) == pbcg.ERR_INVALID
    ho = np.zeros(1)
    assert lib.pbcg_dot_noalloc(4, pbcg._ptr(a), pbcg._ptr(a), 1, ho.ctypes.data_as(ctypes.c_void_p),
                                None) == pbcg.ERR_INVALID
    assert ho[0] == 0.0
    # the binding refuses what the library would misread
    with pytest.raises(TypeError):
        pbcg.dot_noalloc(a.float(), a.float(), out)
    with pytest.raises(TypeError):
        pbcg.dot_noalloc(torch.ones(8, dtype=torch.float64, device="cuda")[::2], a, out)
    with pytest.raises(ValueError):
        pbcg.dot_noalloc(a, a[:3], out)
    with pytest.raises(ValueError):
        pbcg.dot_noalloc(a, a, out[:0])
    # and the entry point still works after the refusals
    assert pbcg.dot_noalloc(a, a, out, pbcg.EXACT) == 0
    torch.cuda.synchronize()
    assert out.item() == 4.0
