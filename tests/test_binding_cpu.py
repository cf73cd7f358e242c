"""The Python binding checks what it hands to the C ABI: lengths, dtypes,
contiguity and, for buffers written in place, writability.  Every check
raises before the library is called, so these run without a GPU (the
objects below have no library handle)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def pbcg():
    from paper_2404_13216_gb300 import build
    build.build_library()
    from paper_2404_13216_gb300 import pbcg
    return pbcg


@pytest.fixture
def ctx(pbcg):
    return object.__new__(pbcg.Context)        # no device: every call below must fail before the library


@pytest.fixture
def mat(pbcg, ctx):
    return pbcg.Matrix(ctx, None, 10, 28)


def test_solve_checks_b_and_x(pbcg, ctx, mat):
    with pytest.raises(ValueError):
        ctx.solve(mat, np.ones(9), np.zeros(10), 1e-8, 10)
    with pytest.raises(ValueError):
        ctx.solve(mat, np.ones(10), np.zeros(11), 1e-8, 10)
    with pytest.raises(TypeError):                          # converting would lose the in-place result
        ctx.solve(mat, np.ones(10), np.zeros(10, dtype=np.float32), 1e-8, 10)
    with pytest.raises(TypeError):
        ctx.solve(mat, np.ones(10), np.zeros(20)[::2], 1e-8, 10)
    x = np.zeros(10)
    x.flags.writeable = False
    with pytest.raises(TypeError):
        ctx.solve(mat, np.ones(10), x, 1e-8, 10)
    with pytest.raises(ValueError):
        ctx.profile_solve(mat, np.ones(10), np.zeros(9), 1e-8, 10)


def test_tensors_must_be_contiguous_and_typed(pbcg, ctx, mat):
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        ctx.solve(mat, torch.ones(10, dtype=torch.float32), np.zeros(10), 1e-8, 10)
    with pytest.raises(TypeError):
        ctx.solve(mat, np.ones(10), torch.zeros(20, dtype=torch.float64)[::2], 1e-8, 10)
    with pytest.raises(TypeError):
        ctx.upload(torch.zeros(11, dtype=torch.int64), np.zeros(28, np.int32), np.zeros(28))


def test_batched_dot_spmv_upload_lengths(pbcg, ctx, mat):
    with pytest.raises(ValueError):
        ctx.solve_batched(mat, np.array([0, 4, 10], np.int32), np.ones(10), np.zeros(10), np.full(3, 1e-8), 10)
    with pytest.raises(ValueError):
        ctx.solve_batched(mat, np.array([0], np.int32), np.ones(10), np.zeros(10), np.full(1, 1e-8), 10)
    with pytest.raises(ValueError):
        ctx.solve_batched(mat, np.array([0, 4, 10], np.int32), np.ones(9), np.zeros(10), np.full(2, 1e-8), 10)
    with pytest.raises(ValueError):                         # b shorter than a would be read past its end
        ctx.dot(np.ones(8), np.ones(7))
    with pytest.raises(ValueError):
        ctx.spmv(mat, np.ones(9))
    with pytest.raises(ValueError):
        ctx.spmv(mat, np.ones(10), np.zeros(9))
    with pytest.raises(ValueError):
        ctx.upload(np.array([0, 2, 3], np.int32), np.array([0, 1], np.int32), np.ones(3))


def test_pool_admit_and_result_lengths(pbcg):
    from paper_2404_13216_gb300 import inputs
    pool = object.__new__(pbcg.Pool)
    pool.sizes = {0: 25}
    A = inputs.convdiff2d(5, 3.0)
    with pytest.raises(ValueError):
        pool.admit(A, np.ones(24))
    with pytest.raises(ValueError):
        pool.admit(A, np.ones(25), x0=np.zeros(26))
    bad = inputs.CSR(A.n, A.row_ptr, A.col_idx[:-1], A.vals)
    with pytest.raises(ValueError):
        pool.admit(bad, np.ones(25))
    with pytest.raises(ValueError):
        pool.result(0, np.zeros(24))


def test_dot_noalloc_takes_device_tensors_only(pbcg):
    """pbcg_dot_noalloc reads and writes device memory in place: host arrays
    and host tensors are refused before the library is called."""
    torch = pytest.importorskip("torch")
    a = np.ones(8)
    with pytest.raises(TypeError):
        pbcg.dot_noalloc(a, a, np.zeros(1))
    t = torch.ones(8, dtype=torch.float64)
    with pytest.raises(TypeError):
        pbcg.dot_noalloc(t, t, torch.zeros(1, dtype=torch.float64))
