"""The serving loop end to end on the GPU: a short Poisson stream through two
pools (exact and plain dots) on two contexts; every request finishes, and a
converged request's true residual meets its own tolerance."""
import numpy as np
import pytest

from paper_2404_13216_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2404_13216_gb300 import build
    build.build_library()
    from paper_2404_13216_gb300 import pbcg
    return pbcg


@pytest.mark.parametrize("alg", [1, 2], ids=["pbicgstab", "pbicgstab_rr"])
def test_serving_stream_on_gpu(lib, alg):
    from paper_2404_13216_gb300 import serve
    pbcg = lib
    reqs = inputs.serving_requests(count=40, rate=400.0, n_lo=1000, n_hi=30000, seed=7)
    templates = serve.make_templates(reqs, 10)
    ce, cp = pbcg.Context(0), pbcg.Context(0)
    for c in (ce, cp):
        c.set_option(pbcg.OPT_RR_PERIOD, 50)
    pools = serve.make_pools(ce, cp, templates, 1 << 20, 1 << 23, 16, 1500, alg)
    try:
        out = serve.serve(reqs, templates, pools, K=6, maxit=1500, time_limit=120.0)
    finally:
        for p in pools.values():
            p.close()
        ce.close()
        cp.close()
    st = out["status"]
    assert np.all(st != -99), "a request did not finish"
    assert np.all(out["latency"] > 0)
    for i, r in enumerate(reqs):
        if st[i] == 0:
            assert out["relres"][i] <= r.tol, (i, out["relres"][i], r.tol)
    summ = serve.summarize(reqs, templates, out, 400.0)
    assert summ["finished"] == len(reqs) and summ["failed"] == 0
    if alg == 2:
        assert summ["converged"] >= 0.9 * len(reqs)
