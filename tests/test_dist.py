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
