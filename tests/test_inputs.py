"""Shape checks of the synthetic generators (sizes quoted for the workloads)."""
import numpy as np

from paper_2404_13216_gb300 import inputs


def test_convdiff_sizes_and_rowsums():
    A = inputs.convdiff2d(64, 10.0)
    assert A.n == 4096 and A.nnz == 20224
    assert np.all(np.diff(A.row_ptr) >= 3)
    for i in (0, 100, 4095):
        cols = A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0)
    b = inputs.rhs_ones(A)
    assert np.allclose(b, [A.vals[A.row_ptr[i]:A.row_ptr[i + 1]].sum() for i in range(A.n)])
    A3 = inputs.convdiff3d(16, 50.0)
    assert A3.n == 4096 and A3.nnz == 7 * 4096 - 6 * 256


def test_convdiff_upwind_values():
    N, Pe = 8, 20.0
    A = inputs.convdiff2d(N, Pe, (1.0, 0.5))
    h = 1.0 / (N + 1)
    i = 3 * N + 4          # interior row: -y, -x, diag, +x, +y
    v = A.vals[A.row_ptr[i]:A.row_ptr[i + 1]]
    c = A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]
    assert list(c) == [i - N, i - 1, i, i + 1, i + N]
    assert np.isclose(v[2], 4 + Pe * h * 1.5)
    assert np.isclose(v[1], -1 - Pe * h * 1.0) and np.isclose(v[0], -1 - Pe * h * 0.5)
    assert v[3] == -1.0 and v[4] == -1.0


def test_powerlaw_small():
    A = inputs.powerlaw(n=20000, mean_len=30, max_len=2000, seed=1)
    lens = np.diff(A.row_ptr)
    assert lens.max() <= 2000 and lens.min() >= 2
    assert 25 < lens.mean() < 33
    for i in (0, 5, 19999):
        cols = A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0) and i in cols
        d = A.vals[A.row_ptr[i]:A.row_ptr[i + 1]][cols == i][0]
        off = np.abs(A.vals[A.row_ptr[i]:A.row_ptr[i + 1]][cols != i]).sum()
        assert np.isclose(abs(d), 1.1 * off)


def test_batched_blockdiag():
    B = inputs.batched_convdiff(nsys=12, seed=2)
    assert B.nsys == 12 and B.sys_row_ptr[-1] == B.A.n
    for k in range(B.nsys):
        r0, r1 = B.sys_row_ptr[k], B.sys_row_ptr[k + 1]
        cols = B.A.col_idx[B.A.row_ptr[r0]:B.A.row_ptr[r1]]
        assert cols.min() >= r0 and cols.max() < r1
        assert r1 - r0 == B.sides[k] ** 2


def test_serving_stream():
    reqs = inputs.serving_requests(count=500, rate=2000.0, seed=5)
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert 0.15 < t[-1] < 0.35
    ns = np.array([r.n for r in reqs])
    assert ns.min() >= 2 ** 2 and ns.max() <= 1.2 * (1 << 20)


def test_recipe_distributions():
    """The stated recipes: batched sides log-uniform in [32, 256] with Peclet
    U(1, 100); power-law off-diagonal magnitudes spread over about eight
    decades (N(0,1) * 10^U(-4,4)) with diagonal signs +-1 at random; the
    serving stream half 2D / half 3D, tolerances 1e-8 or 1e-10 and exact or
    plain dots at about one half each, n log-uniform in [4k, 1M]."""
    B = inputs.batched_convdiff(nsys=512, seed=4)
    s = B.sides.astype(float)
    assert s.min() >= 32 and s.max() <= 256
    # log-uniform: the median side sits near the geometric mean sqrt(32 * 256) = 90.5
    assert 75 < np.median(s) < 110
    assert B.peclet.min() >= 1.0 and B.peclet.max() <= 100.0 and 40 < B.peclet.mean() < 60

    A = inputs.powerlaw(n=20000, mean_len=30, max_len=2000, seed=1)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    off = np.abs(A.vals[A.col_idx != rows])
    lo, hi = np.percentile(np.log10(off), [5, 95])
    assert lo < -3 and hi > 3                      # about eight decades
    diag = A.vals[A.col_idx == rows]
    assert diag.size == A.n and 0.45 < np.mean(diag < 0) < 0.55

    reqs = inputs.serving_requests(count=2000, rate=2000.0, seed=5)
    dims = np.array([r.dim for r in reqs])
    tols = np.array([r.tol for r in reqs])
    ex = np.array([r.exact for r in reqs])
    assert set(dims) == {2, 3} and 0.45 < np.mean(dims == 3) < 0.55
    assert set(tols) == {1e-8, 1e-10} and 0.45 < np.mean(tols == 1e-8) < 0.55
    assert 0.45 < np.mean(ex) < 0.55
    ln = np.log(np.array([r.n for r in reqs], dtype=float))
    # log-uniform over [4096, 2^20] (rounded to whole grid sides): median near sqrt(4096 * 2^20) = 65536
    assert 40000 < np.exp(np.median(ln)) < 100000
