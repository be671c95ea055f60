"""Sharding one table over ranks, on the GPU: the partition kernel against
the oracle's hash, the return to query order, and a sharded table over two
ranks (two processes on one GPU, exchanging through gloo on the host)
answering like the definitional lookup."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_07232_gb300 import build
    build.build()
    import paper_2108_07232_gb300 as G
    return G


@pytest.mark.parametrize("shards", [1, 2, 3, 8, 1000])
@pytest.mark.parametrize("with_values", [True, False])
def test_partition_follows_the_partition_hash(G, shards, with_values):
    """Every key lands in the segment of shard g(k) = ((a_g k + c_g) mod p) mod G
    (the oracle's hash with the partition constants), the per-shard counts
    are exact, and the values (or input positions) travel with their keys."""
    from paper_2108_07232_gb300 import _binding as B
    n, seed = 100003, 77
    keys = W.make_keys(n, 5)
    keys[123] = -1  # the sentinel goes to shard 0
    vals = W.make_values(n, 5)
    a, c = B.ght_partition_constants(seed)
    ku = O._u32(keys)
    g = np.array([0 if k == O.EMPTY else O.hash_value(a, c, shards, int(k)) for k in ku])
    dk, dv = keys.cuda(), vals.cuda()
    ok, ov = torch.empty_like(dk), torch.empty_like(dk)
    counts = np.zeros(shards, dtype=np.uint64)
    B.ght_partition(dk, dv if with_values else None, n, seed, shards, ok, ov, counts)
    assert counts.tolist() == np.bincount(g, minlength=shards).tolist()
    got_k, got_v = O._u32(ok.cpu()), O._u32(ov.cpu())
    ends = np.cumsum(counts.astype(np.int64))
    starts = ends - counts.astype(np.int64)
    for s in range(shards):
        seg = slice(int(starts[s]), int(ends[s]))
        assert set(got_k[seg].tolist()) == set(ku[g == s].tolist())
    if with_values:
        pairs = sorted(zip(got_k.tolist(), got_v.tolist()))
        assert pairs == sorted(zip(ku.tolist(), O._u32(vals).tolist()))
    else:
        assert sorted(got_v.tolist()) == list(range(n))
        assert (ku[got_v.astype(np.int64)] == got_k).all()
    # empty input
    z = torch.empty(0, dtype=torch.int32, device="cuda")
    counts = np.full(shards, 9, dtype=np.uint64)
    B.ght_partition(z, None, 0, seed, shards, z, z, counts)
    assert (counts == 0).all()


def test_partition_rejects_bad_arguments(G):
    from paper_2108_07232_gb300 import _binding as B
    k = torch.zeros(8, dtype=torch.int32, device="cuda")
    counts = np.zeros(8, dtype=np.uint64)
    for shards in (0, 4097):
        with pytest.raises(G.GhtError):
            B.ght_partition(k, None, 8, 1, shards, k, k, counts)
    with pytest.raises(G.GhtError):  # keys off a 16-byte boundary
        B.ght_partition(k[1:], None, 7, 1, 2, k, k, counts)


def test_unpermute_returns_answers_to_query_order(G):
    from paper_2108_07232_gb300 import _binding as B
    n = 70001
    perm = torch.randperm(n, generator=torch.Generator().manual_seed(3)).to(torch.int32)
    src = W.make_values(n, 8)
    dst = torch.empty_like(src).cuda()
    B.ght_unpermute(src.cuda(), perm.cuda(), n, dst)
    want = torch.empty_like(src)
    want[perm.long()] = src
    assert torch.equal(dst.cpu(), want)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q, sentinel: bool):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        import paper_2108_07232_gb300 as G
        from paper_2108_07232_gb300.sharded import ShardedTable
        n_rank = 150000
        all_k, all_v = W.make_keys(world * n_rank, 61), W.make_values(world * n_rank, 61)
        mine = slice(rank * n_rank, (rank + 1) * n_rank)
        k, v = all_k[mine].clone(), all_v[mine].clone()
        if sentinel and rank == 1:
            k[77] = -1
        t = ShardedTable("bcht", world * n_rank, 0.95, seed=9)
        try:
            t.build(k.cuda(), v.cuda())
        except G.GhtError as e:
            q.put((rank, "error", e.status))
            return
        queries = W.make_queries(all_k, 200000 + 31 * rank, 0.5, seed=70 + rank)
        got = t.find(queries.cuda()).cpu()
        ok = bool((O._u32(got) == O.lookup(all_k, all_v, queries)).all())
        q.put((rank, "ok", (ok, t.n_local, t.table.stats()["n_stored"])))
    except Exception as e:
        q.put((rank, "exception", repr(e)))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def _run_ranks(world, sentinel):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q, sentinel)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=600) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return res


def test_sharded_table_over_two_ranks_answers_like_the_lookup(G):
    """Two ranks (two processes on this GPU; gloo moves the buffers through
    host memory) build one table from their own halves of the pairs, each
    keeps the shard its partition hash names, and every rank's queries --
    keys of either rank and keys of none -- are answered bit-exactly."""
    res = _run_ranks(2, sentinel=False)
    for rank, kind, payload in res:
        assert kind == "ok", payload
        ok, n_local, n_stored = payload
        assert ok and n_local == n_stored
    assert sum(r[2][1] for r in res) == 2 * 150000


def test_sharded_build_error_reaches_every_rank(G):
    """A sentinel key in one rank's input fails the shard that receives it;
    every rank raises the same error, none keeps a half-built table."""
    res = _run_ranks(2, sentinel=True)
    assert [(kind, payload) for _, kind, payload in res] == [("error", "GHT_ERR_SENTINEL_KEY")] * 2
