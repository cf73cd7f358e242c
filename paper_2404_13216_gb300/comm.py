"""Collectives of a row-partitioned solve over torch.distributed.

pbcg_part_create and pbcg_part_solve (include/pbcg.h) leave the transport to
the caller: they ask for an in-place int64 sum over all ranks and for a
personalised byte exchange (alltoallv), both on host memory.  TorchComm
provides the two over an initialised torch.distributed process group -- gloo
on host tensors, or NCCL through a copy to the rank's GPU -- and
pbcg.Partition hands them to the library as C callbacks.  Nothing here
computes any part of the method: the callbacks move integers and bytes.
"""
from __future__ import annotations

import numpy as np


class TorchComm:
    """The two collectives over `group` (None: the default process group)."""

    def __init__(self, group=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist, self.group = torch, dist, group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)
        self.backend = str(dist.get_backend(group)).lower()
        self.device = (torch.device("cuda", torch.cuda.current_device())
                       if self.backend == "nccl" else torch.device("cpu"))

    def _dev(self, t):
        return t if self.device.type == "cpu" else t.to(self.device)

    def allreduce_sum_i64(self, buf: np.ndarray) -> None:
        """buf (int64, host) := its sum over the ranks, in place."""
        t = self._dev(self.torch.from_numpy(buf))
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        if t.device.type != "cpu":
            buf[:] = t.cpu().numpy()

    def alltoallv(self, send: np.ndarray, send_bytes, send_displs, recv: np.ndarray, recv_bytes,
                  recv_displs) -> None:
        """Rank r's bytes send[send_displs[k]:+send_bytes[k]] go to rank k,
        which receives them at recv[recv_displs[r]:+recv_bytes[r]]."""
        torch = self.torch
        sb, sd = [int(v) for v in send_bytes], [int(v) for v in send_displs]
        rb, rd = [int(v) for v in recv_bytes], [int(v) for v in recv_displs]
        # pack the segments contiguously in rank order, exchange, unpack
        sbuf = np.concatenate([send[sd[k]:sd[k] + sb[k]] for k in range(self.size)]) if sum(sb) else \
            np.zeros(0, np.uint8)
        rbuf = np.empty(sum(rb), np.uint8)
        ts, tr = self._dev(torch.from_numpy(sbuf)), self._dev(torch.from_numpy(rbuf))
        self.dist.all_to_all_single(tr, ts, output_split_sizes=rb, input_split_sizes=sb, group=self.group)
        if tr.device.type != "cpu":
            rbuf = tr.cpu().numpy()
        off = 0
        for k in range(self.size):
            recv[rd[k]:rd[k] + rb[k]] = rbuf[off:off + rb[k]]
            off += rb[k]


class LocalComm:
    """A one-rank communicator (nothing to exchange)."""
    rank, size = 0, 1

    def allreduce_sum_i64(self, buf):
        pass

    def alltoallv(self, send, send_bytes, send_displs, recv, recv_bytes, recv_displs):
        for k in range(len(send_bytes)):
            n = int(send_bytes[k])
            recv[int(recv_displs[k]):int(recv_displs[k]) + n] = send[int(send_displs[k]):int(send_displs[k]) + n]
