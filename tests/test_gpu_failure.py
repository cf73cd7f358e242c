"""Failure detection on the GPU without a fault.

The staged passes wait on shared-memory barriers for their bulk copies with a
bounded wait; when it gives up, the pass raises the control block's error
flag and the solve returns PBCG_ERR_TIMEOUT.  Here the same wait runs on a
barrier phase that nothing completes (pbcg_check_wait): it must give up,
report it, and leave the context usable.
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


def test_bounded_wait_expires_and_context_survives(ctx, orc):
    t = {}
    for probes in (1 << 10, 1 << 14):
        expired, sec = ctx.check_wait(probes)
        assert expired, probes
        assert sec > 0.0
        t[probes] = sec
    # the time grows with the limit (the wait really probes, it does not return at once)
    assert t[1 << 14] > t[1 << 10]
    print(f"bounded wait: {t[1 << 14] / (1 << 14) * 1e9:.0f} ns per probe; "
          f"the passes' limit of 2^18 probes gives up after about {t[1 << 14] / (1 << 14) * (1 << 18):.2f} s")
    # the context still solves, bit-identical to the oracle
    A = inputs.convdiff2d(20, 5.0)
    b = inputs.rhs_ones(A)
    ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-10, maxit=300, alg=1, mode=1)
    M = ctx.upload_csr(A)
    x = np.zeros(A.n)
    r = ctx.solve(M, b, x, 1e-10, 300, 1, 1)
    M.free()
    assert r.status == ref.status == 0 and r.iters == ref.iters
    assert np.array_equal(x, ref.x)


def test_check_wait_arguments(ctx):
    from paper_2404_13216_gb300 import pbcg
    for bad in (0, -1, (1 << 22) + 1):
        with pytest.raises(pbcg.PbcgError):
            ctx.check_wait(bad)
