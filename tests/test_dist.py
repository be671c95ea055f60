"""The benchmark's multi-rank logic on CPU with two gloo ranks: each rank
works on its own inputs (distinct seeds, disjoint key sets), the timing is
the maximum over ranks, and the reported value is the whole job's keys over
that time. No GPU: the data path has no collective, only the timing does."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seed = bench.rank_seed(bench.SEED, rank)
    keys = W.make_keys(4096, seed)
    local_ms = 10.0 + 5.0 * rank  # rank 1 is slower
    mx = bench.reduce_max(local_ms, world)
    value = bench.whole_job_value(1000, 3, world, mx)
    gathered = [torch.zeros(4096, dtype=torch.int32) for _ in range(world)]
    dist.all_gather(gathered, keys)
    q.put((rank, seed, mx, value, [g.clone() for g in gathered]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_own_inputs():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    seeds = {r[1] for r in res}
    assert len(seeds) == world
    for rank, seed, mx, value, gathered in res:
        assert mx == 15.0  # the slower rank's time
        assert value == pytest.approx(world * 1000 * 3 / 0.015 / 1e9)
    k0, k1 = res[0][4]
    assert len(set(k0.tolist()) & set(k1.tolist())) < 5  # independent random key sets


def test_single_rank_is_the_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.whole_job_value(10, 2, 1, 1000.0) == pytest.approx(20 / 1e9)


# ---------------------------------------------------------------------------
# One table sharded over the ranks (paper_2108_07232_gb300.sharded): the
# exchange protocol over two gloo ranks on the CPU. The partition and the
# shards' local tables are host stand-ins built on the oracle (a partition by
# the oracle's hash, a shard whose find is the definitional lookup), so the
# test checks what the protocol adds: every pair reaches exactly one shard,
# every query is answered by the shard that holds its key, and every answer
# returns to its query's position.

class _OracleShard:
    def build(self, keys, values):
        import numpy as np
        self.keys = keys.clone()
        self.values = values.clone() if values is not None else torch.ones_like(keys)
        self.n = keys.numel()
        assert len(np.unique(keys.numpy())) == self.n  # no pair reached two shards twice

    def find(self, queries, out=None):
        import numpy as np
        import oracle as O
        res = torch.from_numpy(O.lookup(self.keys, self.values, queries).view(np.int32).copy())
        if out is None:
            return res
        out.copy_(res)
        return out


class _OracleOps:
    def __init__(self, shards, a, c):
        self.shards, self.a, self.c = shards, a, c
        self.tables = []

    def partition(self, keys, values):
        import numpy as np
        import oracle as O
        g = np.array([O.hash_value(self.a, self.c, self.shards, int(k)) for k in O._u32(keys)], dtype=np.int64)
        order = np.argsort(g, kind="stable")
        counts = np.bincount(g, minlength=self.shards)
        idx = torch.from_numpy(order)
        out_v = values[idx] if values is not None else torch.from_numpy(order.astype(np.int32))
        return keys[idx].contiguous(), out_v.contiguous(), [int(x) for x in counts]

    def unpermute(self, src, pos, out=None):
        out = torch.empty_like(src) if out is None else out
        out[pos.long()] = src
        return out

    def make_table(self, scheme, capacity, load_factor, seed, **config):
        t = _OracleShard()
        self.tables.append(t)
        return t


def _sharded_worker(rank: int, world: int, port: int, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import numpy as np
        import oracle as O
        from paper_2108_07232_gb300.sharded import ShardedTable
        n_rank = 3000
        all_k, all_v = W.make_keys(world * n_rank, 41), W.make_values(world * n_rank, 41)
        mine = slice(rank * n_rank, (rank + 1) * n_rank)
        ops = _OracleOps(world, 2654435761, 12345)
        t = ShardedTable("bcht", world * n_rank, 0.9, seed=3, ops=ops)
        t.build(all_k[mine].contiguous(), all_v[mine].contiguous())
        shard = ops.tables[-1]
        # the keys this rank holds are exactly those whose partition hash names it
        g = np.array([O.hash_value(ops.a, ops.c, world, int(k)) for k in O._u32(all_k)])
        want_keys = set(O._u32(all_k)[g == rank].tolist())
        held = set(O._u32(shard.keys).tolist())
        # queries of both ranks' keys and of keys in no rank, in a random order
        queries = W.make_queries(all_k, 5000 + 17 * rank, 0.6, seed=50 + rank)
        got = t.find(queries)
        want = O.lookup(all_k, all_v, queries)
        empty = t.find(torch.empty(0, dtype=torch.int32))
        q.put((rank, held == want_keys, t.n_local, bool((O._u32(got) == want).all()), empty.numel(), None))
    except Exception as e:  # report, so the parent fails with the reason
        q.put((rank, False, 0, False, -1, repr(e)))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_sharded_table_over_two_gloo_ranks_answers_like_the_lookup():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sum(r[2] for r in res) == world * 3000  # every pair in exactly one shard
    for rank, keys_ok, n_local, answers_ok, n_empty, err in res:
        assert err is None, err
        assert keys_ok and answers_ok and n_empty == 0, rank
        assert 0.4 * 3000 < n_local < 0.6 * world * 3000


def test_sharded_table_on_one_rank_is_the_local_table():
    """Without a process group there is one shard: no partition, no exchange."""
    import oracle as O
    from paper_2108_07232_gb300.sharded import ShardedTable

    class _NoPartition(_OracleOps):
        def partition(self, keys, values):
            raise AssertionError("one rank needs no partition")

    ops = _NoPartition(1, 3, 5)
    t = ShardedTable("bcht", 500, 0.9, seed=1, ops=ops)
    k, v = W.make_keys(500, 3), W.make_values(500, 3)
    t.build(k, v)
    q = W.make_queries(k, 700, 0.5, seed=4)
    assert (O._u32(t.find(q)) == O.lookup(k, v, q)).all() and t.n_local == 500
    import pytest as _pt
    with _pt.raises(ValueError):
        t.build(k, None)
