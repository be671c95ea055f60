"""One table sharded over the ranks of a torch.distributed process group.

Each rank owns one shard: an ordinary table (HashTable) of the keys whose
partition hash g(k) = ((a_g k + c_g) mod p) mod G names that rank (see
ght_partition in include/ght.h; g's constants are independent of the
tables'). A build partitions each rank's pairs by g, moves every pair to
its shard with one all-to-all, and builds the shard; a find partitions the
queries (remembering their positions), sends them to their shards, finds
them there, sends the answers back with the reverse all-to-all and returns
them to query order. Every step on the data runs in the library's kernels;
this module moves buffers between ranks with torch.distributed collectives
(NCCL for device tensors; a gloo group exchanges device tensors through
host memory).

The partition, the return to query order and the local tables come from an
``ops`` object (by default the library's kernels on the current device); it
is a parameter so that the exchange protocol can also run over other local
implementations.
"""

from __future__ import annotations

import numpy as np

from ._binding import BCHT_SET, GhtError, HashTable, ght_partition, ght_unpermute


class DeviceOps:
    """Partition, unpermute and local tables on the current CUDA device."""

    def __init__(self, seed: int, shards: int, device=None):
        import torch

        self.seed = int(seed)
        self.shards = int(shards)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())

    def _stream(self) -> int:
        import torch
        return torch.cuda.current_stream(self.device).cuda_stream

    def partition(self, keys, values):
        """(keys by shard, values or input positions by shard, per-shard counts)."""
        import torch
        out_k = torch.empty_like(keys)
        out_v = torch.empty_like(keys)
        counts = np.zeros(self.shards, dtype=np.uint64)
        with torch.cuda.device(self.device):
            ght_partition(keys, values, keys.numel(), self.seed, self.shards, out_k, out_v, counts, self._stream())
        return out_k, out_v, [int(c) for c in counts]

    def unpermute(self, src, pos, out=None):
        import torch
        if out is None:
            out = torch.empty_like(src)
        with torch.cuda.device(self.device):
            ght_unpermute(src, pos, src.numel(), out, self._stream())
        return out

    def make_table(self, scheme, capacity: int, load_factor: float, seed: int, **config):
        return HashTable(scheme, capacity, load_factor, seed=seed, device=self.device, **config)


class ShardedTable:
    """A table of up to ``capacity`` keys over all ranks of ``group``; each
    rank calls build and find collectively with its own part of the input
    and gets the answers to its own queries."""

    def __init__(self, scheme, capacity: int, load_factor: float, seed: int = 0, group=None, ops=None, **config):
        import torch.distributed as dist

        self.group = group
        on = dist.is_available() and dist.is_initialized()
        self.world = dist.get_world_size(group) if on else 1
        self.rank = dist.get_rank(group) if on else 0
        self.backend = dist.get_backend(group) if on else None
        self.scheme = scheme
        self.capacity = int(capacity)
        self.load_factor = float(load_factor)
        self.seed = int(seed)
        self.config = config
        self.ops = ops if ops is not None else DeviceOps(seed, self.world)
        self.table = None
        self.n_local = 0

    # -- collectives -------------------------------------------------------------
    def _exchange_counts(self, send_counts: list[int]) -> list[int]:
        import torch
        import torch.distributed as dist
        if self.world == 1:
            return list(send_counts)
        s = torch.tensor(send_counts, dtype=torch.int64)
        r = torch.empty_like(s)
        if self.backend == "nccl":
            s, r = s.cuda(), r.cuda()
        dist.all_to_all_single(r, s, group=self.group)
        return [int(x) for x in r.cpu()]

    def _all_to_all(self, send, send_counts: list[int], recv_counts: list[int]):
        import torch
        import torch.distributed as dist
        if self.world == 1:
            return send
        staged = send.is_cuda and self.backend != "nccl"  # gloo moves host tensors
        src = send.cpu() if staged else send
        dst = torch.empty(sum(recv_counts), dtype=send.dtype, device=src.device)
        dist.all_to_all_single(dst, src, recv_counts, send_counts, group=self.group)
        return dst.to(send.device) if staged else dst

    def _sum(self, x: int) -> int:
        import torch
        import torch.distributed as dist
        if self.world == 1:
            return x
        t = torch.tensor([x], dtype=torch.int64)
        if self.backend == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return int(t.item())

    def _agree(self, code: int) -> int:
        """The largest error code over the ranks (0: every rank succeeded)."""
        import torch
        import torch.distributed as dist
        if self.world == 1:
            return code
        t = torch.tensor([code], dtype=torch.int64)
        if self.backend == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=self.group)
        return int(t.item())

    # -- operations --------------------------------------------------------------
    def build(self, keys, values=None) -> None:
        """Collective: every rank passes its own pairs (values may be None for
        a keys-only set); the pairs of all ranks form the table."""
        keys_only = self.scheme in ("bcht_set", BCHT_SET)
        if values is None and not keys_only:
            raise ValueError("values are required except for a keys-only set")
        if self.world == 1:  # one shard: nothing to partition or exchange
            k, v, send = keys, values if values is not None else keys, [keys.numel()]
        else:
            k, v, send = self.ops.partition(keys, values)
        recv = self._exchange_counts(send)
        rk = self._all_to_all(k, send, recv)
        rv = self._all_to_all(v, send, recv)
        n_total = self._sum(sum(recv))
        code, msg = 0, ""
        if n_total > self.capacity:
            code, msg = 8, f"{n_total} keys exceed the capacity {self.capacity}"
        else:
            try:
                # each shard sized for the keys it received, at the table's load factor
                self.table = self.ops.make_table(self.scheme, max(sum(recv), 1), self.load_factor,
                                                 self.seed + 7919 * (self.rank + 1), **self.config)
                self.table.build(rk, None if keys_only else rv)
            except GhtError as e:
                code, msg = e.code, str(e)
        agreed = self._agree(code)
        if agreed:
            self.table = None
            self.n_local = 0
            raise GhtError(agreed, msg or f"a shard's build failed on another rank (status {agreed})")
        self.n_local = sum(recv)

    def find(self, queries, out=None):
        """Collective: every rank passes its own queries and receives their answers."""
        if self.table is None:
            raise GhtError(5, "the sharded table has no successful build")
        if self.world == 1:
            return self.table.find(queries, out)
        q, pos, send = self.ops.partition(queries, None)
        recv = self._exchange_counts(send)
        rq = self._all_to_all(q, send, recv)
        answers = self.table.find(rq) if rq.numel() else rq.clone()
        back = self._all_to_all(answers, recv, send)
        return self.ops.unpermute(back, pos, out)
