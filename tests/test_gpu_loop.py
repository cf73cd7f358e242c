"""The loop graph: 16 iterations per execution of the WHILE body.

After a stop (maxit, a proposed convergence, a breakdown) the rest of the
body's passes return at their first status check, so a solve that stops at
any point inside a body must give what the host-driven loop of
pbcg_profile_solve gives (one kernel launch at a time, a host read between
launches): the same status, iteration count, residual history and x, bit
for bit, for both algorithms and both dot modes.  The launch count reports
whole body executions.
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
    c.set_option(pbcg.OPT_SMALL_CLUSTER, 0)      # the passes and their graph at every size
    yield c
    c.set_option(pbcg.OPT_SMALL_CLUSTER, 1)
    c.close()


def same(a, b):
    return np.array_equal(np.asarray(a).view(np.int64), np.asarray(b).view(np.int64))


@pytest.mark.parametrize("mode", [1, 0], ids=["exact", "plain"])
@pytest.mark.parametrize("alg", [0, 1, 2], ids=["bicgstab", "pipelined", "pipelined_rr"])
def test_stops_inside_a_body_match_the_host_loop(ctx, alg, mode):
    A = inputs.convdiff3d(20, 40.0, (1.0, 0.5, 0.25))
    b = inputs.rhs_ones(A)
    M = ctx.upload_csr(A)
    # maxit stops at every offset in and around the first bodies, and a
    # solve that stops by convergence (tol 1e-10)
    for tol, maxit in [(1e-300, 1), (1e-300, 2), (1e-300, 15), (1e-300, 16), (1e-300, 17),
                       (1e-300, 31), (1e-300, 33), (1e-10, 500)]:
        xg = np.zeros(A.n)
        rg = ctx.solve(M, b, xg, tol, maxit, alg, mode)
        hg = ctx.history()
        xh = np.zeros(A.n)
        rh, _ = ctx.profile_solve(M, b, xh, tol, maxit, alg, mode)
        hh = ctx.history()
        assert (rg.status, rg.iters) == (rh.status, rh.iters), (tol, maxit)
        assert same(hg, hh) and same(xg, xh), (tol, maxit)
        if tol == 1e-300:
            assert rg.status == 1 and rg.iters == maxit
    M.free()


def test_launch_count_counts_whole_bodies(ctx):
    from paper_2404_13216_gb300 import pbcg
    A = inputs.convdiff3d(20, 40.0, (1.0, 0.5, 0.25))
    b = inputs.rhs_ones(A)
    M = ctx.upload_csr(A)
    for maxit in (1, 16, 17, 40):
        x = np.zeros(A.n)
        r = ctx.solve(M, b, x, 1e-300, maxit, pbcg.PIPELINED, pbcg.EXACT)
        bodies = -(-maxit // 16)
        # setup (3 launches), 16 X/Y pairs per body, the true-residual pass
        assert r.launches == 3 + 32 * bodies + 1, (maxit, r.launches)
    M.free()
