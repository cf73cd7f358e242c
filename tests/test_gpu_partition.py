"""Row-partitioned solves (pbcg_part_*) on the GPU.

Section 2 of the paper runs the method over processes that each own a block
of rows, and Tables 2 and 3 show that with ExBLAS dots the iteration counts
do not depend on the number of processes.  Here every rank runs the passes on
its block, exchanges the halo of each gathered vector, and adds its share of
every dot (the integer digits of its long accumulator) into one total that
every rank rounds once.  In exact mode the history, iteration count, status
and the concatenated x must be bit-identical to the one-grid solve and to the
CPU oracle, for any number of ranks and any split of the rows.

The ranks are separate processes on one GPU, connected by gloo; no kernel of
one rank waits on another rank (every exchange goes through the host).
"""
import datetime
import os
import socket

import numpy as np
import pytest

from paper_2404_13216_gb300 import inputs

pytestmark = pytest.mark.gpu


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2404_13216_gb300 import build
    build.build_library()


def same(a, b):
    return np.array_equal(np.asarray(a).view(np.int64), np.asarray(b).view(np.int64))


def _system(name):
    if name == "3d24":
        return inputs.convdiff3d(24, 50.0)
    if name == "2d40":
        return inputs.convdiff2d(40, 25.0)
    return inputs.powerlaw(n=6000, mean_len=20, max_len=300, seed=7)


def _block(A, rs, r):
    lo, hi = int(rs[r]), int(rs[r + 1])
    rp = A.row_ptr[lo:hi + 1] - A.row_ptr[lo]
    sl = slice(int(A.row_ptr[lo]), int(A.row_ptr[hi]))
    return rp.astype(np.int32), A.col_idx[sl].astype(np.int32), A.vals[sl]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, name, rs, jobs, out):
    """One rank: its block of system `name`, then every (tol, maxit, alg,
    mode) job of `jobs` as a partitioned solve from x0 = 0."""
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2404_13216_gb300 import comm as pcomm
    from paper_2404_13216_gb300 import pbcg
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=180))
    try:
        torch.cuda.set_device(0)
        A = _system(name)
        b = inputs.rhs_ones(A)
        rp, ci, va = _block(A, rs, rank)
        lo, hi = int(rs[rank]), int(rs[rank + 1])
        got = []
        with pbcg.Context(0) as ctx:
            part = pbcg.Partition(ctx, pcomm.TorchComm(), rs, rp, ci, va)
            for tol, maxit, alg, mode in jobs:
                x = np.zeros(hi - lo)
                res = part.solve(b[lo:hi], x, tol, maxit, alg, mode)
                got.append((res.status, res.iters, res.relres_true, ctx.history().tobytes(), x.tobytes()))
            part.close()
        out[rank] = got
    finally:
        dist.destroy_process_group()


def _run_ranks(name, rs, jobs):
    """Per job: ([(status, iters, relres_true) per rank], [history per rank], concatenated x)."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    world = len(rs) - 1
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, np.asarray(rs), jobs, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=400)
        if p.exitcode is None:
            p.kill()
            p.join()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    per_job = []
    for j in range(len(jobs)):
        res = [out[r][j] for r in range(world)]
        hist = [np.frombuffer(t[3], dtype=np.float64) for t in res]
        x = np.concatenate([np.frombuffer(t[4], dtype=np.float64) for t in res])
        per_job.append(([t[:3] for t in res], hist, x))
    return per_job


@pytest.fixture(scope="module")
def single():
    """One-grid solves through pbcg_solve, the reference of the partitioned ones."""
    _gpu()
    from paper_2404_13216_gb300 import pbcg
    ctx = pbcg.Context(0)
    ctx.set_option(pbcg.OPT_SMALL_CLUSTER, 0)
    cache = {}

    def run(name, tol, maxit, alg, mode):
        key = (name, tol, maxit, alg, mode)
        if key not in cache:
            A = _system(name)
            b = inputs.rhs_ones(A)
            M = ctx.upload_csr(A)
            x = np.zeros(A.n)
            r = ctx.solve(M, b, x, tol, maxit, alg, mode)
            cache[key] = (r, ctx.history(), x)
            M.free()
        return cache[key]
    yield run
    ctx.close()


@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_one_rank_partition_is_the_single_solve(single, orc, alg, mode):
    """nranks = 1 (no exchange): the partition path itself, host-driven with
    the dist merges, against pbcg_solve and the oracle."""
    from paper_2404_13216_gb300 import comm as pcomm
    from paper_2404_13216_gb300 import pbcg
    A = _system("3d24")
    b = inputs.rhs_ones(A)
    rs = np.array([0, A.n], np.int32)
    with pbcg.Context(0) as ctx:
        part = pbcg.Partition(ctx, pcomm.LocalComm(), rs, A.row_ptr, A.col_idx, A.vals)
        x = np.zeros(A.n)
        res = part.solve(b, x, 1e-10, 400, alg, mode)
        hist = ctx.history()
        part.close()
    r1, h1, x1 = single("3d24", 1e-10, 400, alg, mode)
    assert res.status == r1.status and res.iters == r1.iters
    if mode == 1:
        ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=1e-10, maxit=400, alg=alg, mode=1, nthreads=8)
        assert res.iters == ref.iters and same(hist, ref.history) and same(x, ref.x)
        assert same(hist, h1) and same(x, x1)
    else:
        # one rank adds one partial per dot: the one-grid plain sums, up to the last bits
        assert np.allclose(hist[:20], h1[:20], rtol=1e-8, atol=0)
        assert res.status != 0 or res.relres_true <= 1e-10


SPLITS = {
    "3d24": [[0, 6912, 13824], [0, 4000, 9001, 13824]],      # halves; uneven thirds (ragged against tiles)
    "2d40": [[0, 803, 1600], [0, 1, 900, 1600]],              # a one-row rank
    "powerlaw": [[0, 3000, 6000], [0, 1500, 2500, 6000]],     # random columns: every rank talks to every rank
}


@pytest.mark.parametrize("name", ["3d24", "2d40", "powerlaw"])
def test_exact_partitioned_bitwise_for_any_rank_count(single, orc, name):
    """The paper's process-count invariance, bit for bit: 2 and 3 ranks,
    even and uneven splits, both algorithms, against one grid and the
    oracle.  On the 2D system the same ranks also run plain dots: added in
    rank order, deterministic for a split, within the plain tolerance of the
    one-grid history, and converged to the tolerance."""
    A = _system(name)
    b = inputs.rhs_ones(A)
    tol, maxit = (1e-10, 400) if name != "powerlaw" else (1e-10, 60)
    jobs = [(tol, maxit, 0, 1), (tol, maxit, 1, 1)]
    if name == "2d40":
        jobs.append((1e-8, 800, 1, 0))
    refs = []
    for alg in (0, 1):
        ref = orc.solve(A.row_ptr, A.col_idx, A.vals, b, tol=tol, maxit=maxit, alg=alg, mode=1, nthreads=8)
        r1, h1, x1 = single(name, tol, maxit, alg, 1)
        assert r1.iters == ref.iters and same(h1, ref.history) and same(x1, ref.x)
        refs.append(ref)
    for rs in SPLITS[name]:
        results = _run_ranks(name, rs, jobs)
        for alg in (0, 1):
            ranks, hist, x = results[alg]
            ref = refs[alg]
            for (st, its, _), h in zip(ranks, hist):
                assert st == ref.status and its == ref.iters, (rs, alg, st, its)
                assert same(h, ref.history), (rs, alg)
            assert same(x, ref.x), (rs, alg)
            assert len({r[2] for r in ranks}) == 1           # every rank formed the same true residual
        if name == "2d40":
            r1, h1, _ = single(name, 1e-8, 800, 1, 0)
            ranks, hist, x = results[2]
            assert all(r[0] == 0 and r[2] <= 1e-8 for r in ranks), ranks
            k = min(20, len(h1), len(hist[0]))
            assert np.allclose(hist[0][:k], h1[:k], rtol=1e-8, atol=0)
            assert all(same(h, hist[0]) for h in hist)          # the same history on every rank
