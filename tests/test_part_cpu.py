"""Host side of row-partitioned solves, without a GPU.

1. pbcg_part_plan (host-only C): the halo of a rank's block (external columns,
   sorted, grouped by owning rank), the per-rank counts and each entry's
   local column, against a numpy computation, and its validation.
2. The communicator the GPU path uses: TorchComm's two collectives over gloo
   (world size 2), called through the same C callbacks the library calls,
   carrying out the library's halo protocol (counts, then requested rows,
   then values) and an int64 sum of carry-save digits with negative entries.
"""
import ctypes
import os
import socket

import numpy as np
import pytest

from paper_2404_13216_gb300 import inputs


@pytest.fixture(scope="module")
def pbcg():
    from paper_2404_13216_gb300 import build
    build.build_library()
    from paper_2404_13216_gb300 import pbcg
    return pbcg


def _block(A, rs, r):
    lo, hi = int(rs[r]), int(rs[r + 1])
    rp = (A.row_ptr[lo:hi + 1] - A.row_ptr[lo]).astype(np.int32)
    sl = slice(int(A.row_ptr[lo]), int(A.row_ptr[hi]))
    return rp, A.col_idx[sl].astype(np.int32)


def _numpy_plan(A, rs, r):
    lo, hi = int(rs[r]), int(rs[r + 1])
    rp, ci = _block(A, rs, r)
    ext = np.unique(ci[(ci < lo) | (ci >= hi)])
    owner = np.searchsorted(rs, ext, side="right") - 1
    counts = np.bincount(owner, minlength=len(rs) - 1)
    local = np.where((ci >= lo) & (ci < hi), ci - lo, (hi - lo) + np.searchsorted(ext, ci))
    return ext, counts, local


@pytest.mark.parametrize("gen", ["3d12", "powerlaw"])
def test_plan_matches_numpy(pbcg, gen):
    A = inputs.convdiff3d(12, 20.0) if gen == "3d12" else inputs.powerlaw(n=3000, mean_len=15, max_len=200, seed=3)
    rng = np.random.default_rng(5)
    for P in (1, 2, 3, 5):
        cuts = np.sort(rng.choice(np.arange(1, A.n), P - 1, replace=False)) if P > 1 else np.zeros(0, int)
        rs = np.concatenate([[0], cuts, [A.n]]).astype(np.int32)
        for r in range(P):
            rp, ci = _block(A, rs, r)
            halo, counts, local = pbcg.part_plan(P, r, rs, rp, ci)
            e_halo, e_counts, e_local = _numpy_plan(A, rs, r)
            assert np.array_equal(halo, e_halo) and np.array_equal(counts, e_counts)
            assert np.array_equal(local, e_local)
            assert counts[r] == 0 and counts.sum() == halo.size


def test_plan_validation(pbcg):
    A = inputs.convdiff2d(6, 2.0)
    rs = np.array([0, 20, 36], np.int32)
    rp, ci = _block(A, rs, 0)
    with pytest.raises(pbcg.PbcgError):
        pbcg.part_plan(2, 2, rs, rp, ci)                              # no such rank
    with pytest.raises(pbcg.PbcgError):
        pbcg.part_plan(2, 0, np.array([0, 20, 10], np.int32), rp, ci)  # row_starts decreases
    with pytest.raises(pbcg.PbcgError):
        pbcg.part_plan(2, 0, np.array([1, 20, 36], np.int32), rp, ci)  # does not start at 0
    bad = ci.copy()
    bad[3] = 36
    with pytest.raises(pbcg.PbcgError):
        pbcg.part_plan(2, 0, rs, rp, bad)                              # column beyond the global rows
    with pytest.raises(pbcg.PbcgError):
        pbcg.part_plan(2, 0, np.array([0, 0, 36], np.int32), rp[:1], ci[:0])   # empty block


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from paper_2404_13216_gb300 import comm as pcomm
    from paper_2404_13216_gb300 import pbcg
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = pcomm.TorchComm()
        c, keep = pbcg._c_comm(comm)
        A = inputs.powerlaw(n=2000, mean_len=12, max_len=100, seed=9)
        rs = np.array([0, 700, 2000], np.int32)
        rp, ci = _block(A, rs, rank)
        halo, counts, _ = pbcg.part_plan(world, rank, rs, rp, ci)
        I64 = ctypes.c_int64 * world

        def a2a(send, sb, sd, recv, rb, rd):
            return c.alltoallv(None, send.ctypes.data_as(ctypes.c_void_p), I64(*sb), I64(*sd),
                               recv.ctypes.data_as(ctypes.c_void_p), I64(*rb), I64(*rd))
        # 1. counts: how many of my rows each rank wants
        cs = counts.astype(np.int64)
        cr = np.zeros(world, np.int64)
        eight = [8] * world
        assert a2a(cs, eight, [8 * k for k in range(world)], cr, eight, [8 * k for k in range(world)]) == 0
        # 2. the requested global rows
        qb = [4 * int(v) for v in counts]
        qd = np.concatenate([[0], np.cumsum(qb)[:-1]]).tolist()
        ab = [4 * int(v) for v in cr]
        ad = np.concatenate([[0], np.cumsum(ab)[:-1]]).tolist()
        wanted = np.zeros(max(1, int(cr.sum())), np.int32)
        assert a2a(halo.astype(np.int32), qb, qd, wanted, ab, ad) == 0
        wanted = wanted[:int(cr.sum())]
        # 3. values: x_global[i] = 0.5 * i, sent for the wanted rows
        vals = (0.5 * wanted).astype(np.float64)
        recv = np.zeros(max(1, halo.size), np.float64)
        assert a2a(vals, [2 * v for v in ab], [2 * v for v in ad], recv, [2 * v for v in qb], [2 * v for v in qd]) == 0
        # 4. carry-save digits with negative entries, summed in place
        dig = np.array([(-1) ** (rank + k) * (1 << 40) * (k + 1) + rank for k in range(8)], np.int64)
        buf = (ctypes.c_int64 * dig.size)(*dig.tolist())
        assert c.allreduce_sum_i64(None, buf, dig.size) == 0
        out[rank] = (halo.tolist(), wanted.tolist(), recv[:halo.size].tolist(), list(buf), counts.tolist(),
                     cr.tolist())
    finally:
        dist.destroy_process_group()


def test_two_rank_halo_protocol_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        if p.exitcode is None:
            p.kill()
            p.join()
    assert all(p.exitcode == 0 for p in procs)
    rs = [0, 700, 2000]
    for r in range(2):
        halo, wanted, recv, digits, counts, cr = out[r]
        o = 1 - r
        # what I was asked for is exactly the other rank's halo inside my rows
        other_halo = np.array(out[o][0])
        mine = other_halo[(other_halo >= rs[r]) & (other_halo < rs[r + 1])]
        assert wanted == mine.tolist() and cr[o] == len(mine) and out[o][4][r] == len(mine)
        # and the values arrive at the right halo positions
        assert recv == (0.5 * np.array(halo)).tolist()
        want = [sum((-1) ** (q + k) * (1 << 40) * (k + 1) + q for q in range(2)) for k in range(8)]
        assert digits == want
