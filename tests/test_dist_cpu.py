"""Multi-rank paths on CPU with the gloo backend (world size 2).

1. bench.py's reduction: whole-job time is the slowest rank's, work is summed.
2. The row-partition seam of the exact dot: each rank accumulates the exact
   integer sum of its half of the rows (the oracle's fixed-point big integer,
   as base-2^32 digits in int64), the digits are all-reduced, and one rounding
   gives the same double as the unsplit dot -- the process-count invariance of
   the exact method (Tables 2-3).
"""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    ms, its = bench.reduce_over_ranks(dist, 10.0 + rank, 100 * (rank + 1), torch.device("cpu"))
    # exact dot over a row split
    rng = np.random.default_rng(0)
    n = 5000
    a = rng.standard_normal(n) * np.ldexp(1.0, rng.integers(-300, 300, n))
    b = rng.standard_normal(n)
    a[::7] = -a[1::7][: a[::7].size] if a[1::7].size >= a[::7].size else a[::7]
    lo, hi = (0, n // 3) if rank == 0 else (n // 3, n)
    N = oracle.dot_exact_fixed(a[lo:hi], b[lo:hi])
    mag = abs(N)
    digits = [(mag >> (32 * k)) & 0xFFFFFFFF for k in range(oracle.LIMBS)]
    t = torch.tensor([d if N >= 0 else -d for d in digits], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    total = sum(int(v) << (32 * k) for k, v in enumerate(t.tolist()))
    got = oracle.round_fixed(total)
    want = oracle.dot_exact(a, b)
    out[rank] = (ms, its, got, want)
    dist.destroy_process_group()


def test_two_rank_reduction_and_exact_split():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    for r in range(2):
        ms, its, got, want = out[r]
        assert ms == 11.0 and its == 300
        assert np.array_equal(np.array([got]).view(np.int64), np.array([want]).view(np.int64))
