"""Keys-only BCHT (membership set, 32 four-byte keys per 128-byte bucket)
against the oracle: the set is the oracle's BCHT with b = 32 over pairs
(key, 0), so a find must answer 1 exactly for the keys the definitional
lookup finds, the exported keys must pass the validator as such a table, and
find probe counts must equal the oracle's on the exported table."""

import numpy as np
import pytest
import torch

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


def _as_pairs(keys32: np.ndarray) -> np.ndarray:
    k = keys32.astype(np.uint64)
    return np.where(keys32 == O.EMPTY, np.uint64(O.EMPTY_PAIR), k)  # value 0 in the high word


@pytest.mark.parametrize("lf", [0.8, 0.95, 0.99])
@pytest.mark.parametrize("kpl", [1, 2])
def test_keys_only_set_parity(G, lf, kpl):
    n = (1 << 16) + 29
    keys = W.make_keys(n, 61)
    zeros = torch.zeros(n, dtype=torch.int32)
    t = G.HashTable("bcht_set", n, lf, seed=3, count_probes=1, keys_per_lane=kpl, build_keys_per_lane=kpl)
    t.build(keys.cuda())  # no values
    st = t.stats()
    assert st["slot_bytes"] == 4 and st["bucket_size"] == 32 and st["built"] == 1
    assert st["num_buckets"] == O.num_buckets(n, lf, 32)
    slots = t.export()
    assert slots.dtype == np.uint32 and slots.size == st["num_slots"]
    T = O.Table(O.BCHT, n, lf, b=32, m=st["num_buckets"])
    T.set_constants(st["hash_a"], st["hash_c"])
    pairs = _as_pairs(slots)
    ok, msg = T.validate(keys, zeros, slots=pairs)
    assert ok, msg
    for f in (0.0, 0.5, 1.0):
        q = W.make_queries(keys, n + 7, f, seed=5)
        t.reset_counters()
        got = O._u32(t.find(q.cuda()).cpu())
        want = (O.lookup(keys, zeros, q) != O.EMPTY).astype(np.uint32)
        assert (got == want).all(), f
        assert t.stats()["find_probes"] == T.find(q, slots=pairs)[2]


def test_keys_only_set_edges(G):
    t = G.HashTable("bcht_set", 100, 0.9, seed=1)
    k = torch.tensor([5, 6, 7], dtype=torch.int32)
    t.build(k.pin_memory())  # host path, no values
    got = t.find(torch.tensor([5, 8, -1, 7], dtype=torch.int32).cuda()).cpu().tolist()
    assert got == [1, 0, 0, 1]
    with pytest.raises(G.GhtError):
        t.build(torch.tensor([1, -1], dtype=torch.int32).cuda())
    with pytest.raises(G.GhtError):
        G.HashTable("bcht_set", 100, 0.9, bucket_size=16)


@pytest.mark.parametrize("lf", [0.9, 0.99])
@pytest.mark.parametrize("kpl", [4, 6])
def test_keys_only_set_staged_find(G, lf, kpl):
    """The staged find (bucket parts in shared memory, 4-lane tiles) on the
    set's 32-key buckets: membership bit-exact against the definitional
    lookup, probe counts equal to the oracle's on the exported table, the
    sentinel answered absent."""
    n = (1 << 16) + 29
    keys = W.make_keys(n, 67)
    zeros = torch.zeros(n, dtype=torch.int32)
    t = G.HashTable("bcht_set", n, lf, seed=3, count_probes=1, find_async=1, keys_per_lane=kpl)
    t.build(keys.cuda())
    st = t.stats()
    assert (st["find_staged"], st["tile_lanes"], st["keys_per_lane"]) == (1, 4, kpl)
    T = O.Table(O.BCHT, n, lf, b=32, m=st["num_buckets"])
    T.set_constants(st["hash_a"], st["hash_c"])
    pairs = _as_pairs(t.export())
    for f in (0.0, 0.5, 1.0):
        q = W.make_queries(keys, n + 7, f, seed=11)
        t.reset_counters()
        got = O._u32(t.find(q.cuda()).cpu())
        want = (O.lookup(keys, zeros, q) != O.EMPTY).astype(np.uint32)
        assert (got == want).all(), f
        assert t.stats()["find_probes"] == T.find(q, slots=pairs)[2]
    q = torch.cat([keys[:3], torch.tensor([-1], dtype=torch.int32), W.make_negatives(n, 2, 3)])
    assert O._u32(t.find(q.cuda()).cpu()).tolist() == [1, 1, 1, 0, 0, 0]


def test_keys_only_set_find_selection(G):
    """Small sets find through the 8-lane register find, sets whose slots
    exceed the L2 through the staged one; the forms that cannot run are
    rejected."""
    small = G.HashTable("bcht_set", 1 << 16, 0.9).stats()
    assert (small["find_staged"], small["tile_lanes"]) == (0, 8)
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    big = G.HashTable("bcht_set", (l2 // 4) + (1 << 20), 1.0)
    assert (big.stats()["find_staged"], big.stats()["tile_lanes"], big.stats()["keys_per_lane"]) == (1, 4, 6)
    del big
    with pytest.raises(G.GhtError):
        G.HashTable("bcht_set", 1000, 0.9, find_async=1, tile_lanes=8)
    with pytest.raises(G.GhtError):
        G.HashTable("bcht_set", 1000, 0.9, find_async=-1, tile_lanes=4)
