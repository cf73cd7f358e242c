"""pbcg_dot_noalloc: the dot product for callers that cannot allocate device
memory (inside another allocator's arena, under a fixed memory budget, or in
a loop that must not enter the allocator).  It takes device inputs and a
device output, keeps its merge state in a fixed static device array, and must
agree with the context-based pbcg_dot: bit for bit in exact mode, within the
plain-dot tolerance of the other tests in plain mode, on two calls in a row.

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
    del ctypes
