"""GPU parity of the grouped find (queries grouped by table range, round by
round, answers returned to query order), called through the C ABI, against
the CPU oracle on the same seeded inputs:

* results equal the definitional lookup bit for bit, for every scheme with
  16-pair buckets, at positive fractions 0, 0.5 and 1, with ragged batch
  sizes, sentinel queries and crowded batches (one key asked millions of
  times, which overflows the grouping regions into the spill path);
* probe counts equal the oracle's find evaluated on the GPU's own table:
  the grouped schedule makes exactly the per-query probes of Sec. V;
* batches or arrays the grouped find does not take fall back to the
  per-query find, with the same results; the per-query find stays the
  default.
"""

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

NQ = (1 << 22) + 37  # ragged: not a multiple of a tile, a window or a group region


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_07232_gb300 import build
    build.build()
    import paper_2108_07232_gb300 as G
    return G


def oracle_view(st, scheme, capacity, lf):
    T = O.Table(scheme, capacity, lf, b=st["bucket_size"], h=st["num_hashes"],
                t=st["threshold"] or None, m=st["num_buckets"])
    T.set_constants(st["hash_a"], st["hash_c"])
    return T


def build_table(G, scheme, n, lf, seed=13, data_seed=3, **cfg):
    keys = W.make_keys(n, data_seed)
    vals = W.make_values(n, data_seed)
    t = G.HashTable(scheme, n, lf, seed=seed, count_probes=1, **cfg)
    t.build(keys.cuda(), vals.cuda())
    assert t.stats()["built"] == 1
    return t, keys, vals


def check_batch(G, t, T, slots, keys, vals, q, grouped=True):
    t.reset_counters()
    got = O._u32(t.find(q.cuda()).cpu())
    st = t.stats()
    assert st["last_find_grouped"] == (1 if grouped else 0)
    assert (got == O.lookup(keys, vals, q)).all()
    assert st["find_queries"] == q.numel()
    assert st["find_probes"] == T.find(q, slots=slots)[2]


@pytest.mark.parametrize("scheme,lf,n", [
    (O.BCHT, 0.9, 1 << 20), (O.BCHT, 0.99, 1 << 20),   # 256-bucket sub-groups, one level
    (O.BCHT, 0.95, 1 << 22),                           # 512-bucket sub-groups, two per group
    (O.P2BHT, 0.8, 1 << 20), (O.IHT, 0.86, 1 << 20),
    (O.BCHT_LB, 0.95, 1 << 20), (O.BCHT_LB, 0.99, 1 << 20),
])
def test_grouped_find_parity(G, scheme, lf, n):
    """Bit-exact results and exact probe counts of the grouped find (forced
    on) for each scheme's stop rule: BCHT stops at a bucket with an empty
    slot (Sec. V-B), P2BHT, IHT and the load-balanced BCHT read on until the
    key is found (Sec. V-C, V-D, III-A)."""
    t, keys, vals = build_table(G, scheme, n, lf, find_grouped=1)
    st = t.stats()
    assert st["find_grouped"] == 1
    T = oracle_view(st, scheme, n, lf)
    slots = t.export()
    ok, msg = T.validate(keys, vals, slots=slots)
    assert ok, msg
    for f in (0.0, 0.5, 1.0):
        check_batch(G, t, T, slots, keys, vals, W.make_queries(keys, NQ, f, seed=17))


def test_grouped_find_sub_groups_across_eight_splits(G):
    """A table of 2^24 keys (2^20 buckets: groups of 4096 buckets split in
    eight 512-bucket sub-groups) with 2^23 + 5 queries."""
    n, lf = 1 << 24, 0.95
    t, keys, vals = build_table(G, O.BCHT, n, lf, find_grouped=1)
    st = t.stats()
    T = oracle_view(st, O.BCHT, n, lf)
    slots = t.export()
    for f in (0.0, 0.7):
        check_batch(G, t, T, slots, keys, vals, W.make_queries(keys, (1 << 23) + 5, f, seed=19))


def test_grouped_find_edge_cases(G):
    """Sentinel queries (answered as misses without a probe), one key asked
    for every query of a batch (its group and sub-group overflow their
    regions: the spill path answers the rest), a missing key asked likewise,
    and the fallbacks: an unaligned query array and a batch too small for the
    grouping regions run the per-query find."""
    n, lf = 1 << 20, 0.99
    t, keys, vals = build_table(G, O.BCHT, n, lf, find_grouped=1)
    st = t.stats()
    T = oracle_view(st, O.BCHT, n, lf)
    slots = t.export()
    q = W.make_queries(keys, NQ, 0.5, seed=23).clone()
    q[::97] = -1  # sentinel queries spread over the batch
    check_batch(G, t, T, slots, keys, vals, q)
    # a key stored past its first bucket, asked NQ times (crowded: spills)
    _, per_key, _ = T.find(keys[:4096], slots=slots)
    hot = keys[:4096][int(np.argmax(per_key))]
    assert int(per_key.max()) >= 2
    q = hot.repeat(NQ)
    check_batch(G, t, T, slots, keys, vals, q)
    neg = W.make_negatives(n, 1, 5)
    check_batch(G, t, T, slots, keys, vals, neg.repeat(NQ))
    # half the batch one key, half ordinary queries
    q = W.make_queries(keys, NQ, 0.5, seed=29).clone()
    q[: NQ // 2] = keys[7]
    check_batch(G, t, T, slots, keys, vals, q)
    # unaligned queries: the per-query find, same answers
    qq = W.make_queries(keys, NQ + 1, 0.5, seed=31).cuda()
    t.reset_counters()
    got = O._u32(t.find(qq[1:]).cpu())
    assert t.stats()["last_find_grouped"] == 0
    assert (got == O.lookup(keys, vals, qq[1:].cpu())).all()
    # a small batch (regions below the grouping's minimum): per query
    q = W.make_queries(keys, 5000, 0.5, seed=37)
    check_batch(G, t, T, slots, keys, vals, q, grouped=False)


def test_grouped_find_off_and_other_shapes(G):
    """find_grouped = -1 (like 0, the default) keeps the per-query find on a
    batch the grouped find would take; 32-pair buckets, CUCKOO1 and the
    keys-only set reject find_grouped = 1."""
    n, lf = 1 << 20, 0.9
    t, keys, vals = build_table(G, O.BCHT, n, lf, find_grouped=-1)
    q = W.make_queries(keys, NQ, 0.5, seed=41)
    got = O._u32(t.find(q.cuda()).cpu())
    assert t.stats()["last_find_grouped"] == 0
    assert (got == O.lookup(keys, vals, q)).all()
    for scheme, cfg in (("bcht", {"bucket_size": 32}), ("cuckoo1", {}), ("bcht_set", {})):
        with pytest.raises(G.GhtError):
            G.HashTable(scheme, 1 << 16, 0.8, seed=1, find_grouped=1, **cfg)


def test_grouped_find_at_scale_matches_the_per_query_find(G):
    """2^26 keys at LF 0.9 (596 MB of slots, beyond the L2; 4.7 M buckets,
    groups of 16384 buckets split in 64 sub-groups) and 2^25 queries: the
    grouped find (opt-in) matches the per-query find of the same table (the
    default, also for this batch) and the definitional lookup."""
    n, lf = 1 << 26, 0.9
    free, _ = torch.cuda.mem_get_info()
    if free < 8 * 2**30:
        pytest.skip("needs about 8 GB of free device memory")
    keys = W.make_keys(n, 43, device="cuda")
    vals = W.make_values(n, 43, device="cuda")
    a = G.HashTable("bcht", n, lf, seed=3, find_grouped=1)
    b = G.HashTable("bcht", n, lf, seed=3)
    a.build(keys, vals)
    b.build(keys, vals)
    assert b.stats()["find_grouped"] == 0
    q = W.make_queries(keys, 1 << 25, 0.5, seed=47)
    got_a = a.find(q)
    assert a.stats()["last_find_grouped"] == 1
    got_b = b.find(q)
    assert b.stats()["last_find_grouped"] == 0
    assert torch.equal(got_a, got_b)
    want = O.lookup(keys.cpu(), vals.cpu(), q.cpu())
    assert (O._u32(got_a.cpu()) == want).all()
