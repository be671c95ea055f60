"""Served pool (continuous batching under an HBM budget), through the C ABI:
each find request's answer is the same whether it runs alone or packed with
others in the mix, and equals the definitional lookup; builds are admitted
only when they fit the budget; trace replay works in pool and serial modes."""

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


@pytest.fixture(scope="module")
def tables():
    sizes = [1000, 37, 20000, 65536, 3000, 150000]
    out = []
    for i, n in enumerate(sizes):
        k, v = W.make_keys(n, 100 + i), W.make_values(n, 100 + i)
        out.append((n, k.cuda(), v.cuda()))
    return out


def _requests(tables, count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for j in range(count):
        t = int(rng.integers(0, len(tables)))
        n, k, _ = tables[t]
        size = int(2 ** rng.uniform(0, 16))  # 1 .. 65536 queries
        q = W.make_queries(k.cpu(), size, 0.7, seed=1000 * seed + j).cuda()
        reqs.append((t, q))
    return reqs


def test_pool_results_same_alone_and_in_the_mix(G, tables):
    pool = G.Pool(1 << 30)
    ids = []
    for i, (n, k, v) in enumerate(tables):
        tk, tid = pool.submit_build(n, 0.95, 7 + i, k, v)
        ids.append((tk, tid))
    for tk, _ in ids:
        assert pool.wait(tk)["status"] == 0
    reqs = _requests(tables, 300, seed=1)
    # alone: one request at a time
    alone = []
    for t, q in reqs:
        out = torch.full_like(q, 7)
        pool.wait(pool.submit_find(ids[t][1], q, out))
        alone.append(out)
    # in the mix: all submitted at once, waited on afterwards. Requests that
    # arrive while the pool's launches are busy are packed together; a queue
    # of large finds submitted first keeps them busy for tens of ms, longer
    # than the submissions take, so the mix does not depend on how fast this
    # host submits against how fast the GPU answers.
    big_t = len(tables) - 1
    big_q = W.make_queries(tables[big_t][1].cpu(), 1 << 22, 0.5, seed=77).cuda()
    big_out = torch.empty_like(big_q)
    blockers = [pool.submit_find(ids[big_t][1], big_q, big_out) for _ in range(300)]
    launches_before = pool.stats()["find_launches"]
    mixed, tickets = [], []
    for t, q in reqs:
        out = torch.full_like(q, 9)
        tickets.append(pool.submit_find(ids[t][1], q, out))
        mixed.append(out)
    packed = [pool.wait(tk)["launch_requests"] for tk in tickets]
    for tk in blockers:
        assert pool.wait(tk)["status"] == 0
    st = pool.stats()
    # the blockers take one launch each (each is a full launch's worth of
    # queries); the 300 mixed requests far fewer than one each
    assert st["find_launches"] - launches_before < len(reqs) // 2 + len(blockers)
    assert max(packed) > 1
    for (t, q), a, m in zip(reqs, alone, mixed):
        assert torch.equal(a, m)
        n, k, v = tables[t]
        assert (O._u32(m.cpu()) == O.lookup(k.cpu(), v.cpu(), q.cpu())).all()
    pool.close()


def test_pool_admits_builds_within_the_budget(G, tables):
    n, k, v = tables[3]
    one = G.ght_table_bytes(G.BCHT, n, 0.95)
    pool = G.Pool(2 * one + 1000)  # room for two such tables
    t1, a = pool.submit_build(n, 0.95, 1, k, v)
    t2, b = pool.submit_build(n, 0.95, 2, k, v)
    t3, c = pool.submit_build(n, 0.95, 3, k, v)
    assert pool.wait(t1)["status"] == 0 and pool.wait(t2)["status"] == 0
    with pytest.raises(G.GhtError) as e:  # the third waits for room
        pool.wait(t3, timeout=0.5)
    assert e.value.status == "GHT_ERR_DEVICE_TIMEOUT"
    st = pool.stats()
    assert st["pending_builds"] == 1 and st["used_bytes"] <= 2 * one + 1000
    pool.drop(a)
    assert pool.wait(t3, timeout=60)["status"] == 0
    q = W.make_queries(k.cpu(), 5000, 0.5, seed=3).cuda()
    out = torch.empty_like(q)
    pool.wait(pool.submit_find(c, q, out))
    assert (O._u32(out.cpu()) == O.lookup(k.cpu(), v.cpu(), q.cpu())).all()
    # a finds on a dropped table is refused, a table larger than the budget is refused
    with pytest.raises(G.GhtError):
        pool.wait(pool.submit_find(a, q, out))
    big, _ = pool.submit_build(1 << 24, 0.5, 4, k, v)
    with pytest.raises(G.GhtError) as e:
        pool.wait(big)
    assert e.value.status == "GHT_ERR_OOM"
    assert pool.stats()["builds_refused"] == 1
    pool.close()


def test_pool_replay_pool_and_serial(G, tables):
    pool = G.Pool(1 << 30)
    ids = []
    for i, (n, k, v) in enumerate(tables):
        tk, tid = pool.submit_build(n, 0.95, 30 + i, k, v)
        pool.wait(tk)
        ids.append(tid)
    reqs = _requests(tables, 120, seed=2)
    arrivals = np.cumsum(np.random.default_rng(4).exponential(20e-6, len(reqs)))
    outs = {m: [torch.empty_like(q) for _, q in reqs] for m in ("pool", "serial")}
    res = {}
    for mode in ("pool", "serial"):
        trace = [{"kind": "find", "table": ids[t], "queries": q, "out": outs[mode][i], "arrival_s": arrivals[i]}
                 for i, (t, q) in enumerate(reqs)]
        k2, v2 = W.make_keys(4000, 55), W.make_values(4000, 55)
        trace.append({"kind": "build", "keys": k2.cuda(), "values": v2.cuda(), "capacity": 4000,
                      "load_factor": 0.9, "seed": 5, "arrival_s": float(arrivals[len(reqs) // 2])})
        lat, st, mk = pool.replay(trace, serial=(mode == "serial"))
        assert (st == 0).all() and (lat > 0).all() and mk > 0
        res[mode] = lat
    for a, b in zip(outs["pool"], outs["serial"]):
        assert torch.equal(a, b)
    pool.close()


def test_pool_finds_exact_while_builds_are_admitted(G, tables):
    """Builds of new tables are admitted and run on the build worker's
    stream while find launches are in flight: every find answer is the same
    as when it ran alone and equals the definitional lookup, and finds
    submitted on a new table before its build completed wait for it and
    answer from it."""
    pool = G.Pool(1 << 30)
    ids = []
    for i, (n, k, v) in enumerate(tables):
        tk, tid = pool.submit_build(n, 0.95, 60 + i, k, v)
        assert pool.wait(tk)["status"] == 0
        ids.append(tid)
    reqs = _requests(tables, 240, seed=5)
    alone = []
    for t, q in reqs:
        out = torch.full_like(q, 3)
        pool.wait(pool.submit_find(ids[t], q, out))
        alone.append(out)
    fresh = []
    for j, n in enumerate((200000, 50000, 1000)):
        k, v = W.make_keys(n, 300 + j), W.make_values(n, 300 + j)
        fresh.append((n, k.cuda(), v.cuda(), k, v))
    mixed, tickets, new_finds = [], [], []
    builds = []
    for i, (t, q) in enumerate(reqs):
        if i % 80 == 0:  # a build request arrives among the finds
            n, dk, dv, hk, hv = fresh[i // 80]
            btk, bid = pool.submit_build(n, 0.9, 400 + i, dk, dv)
            builds.append(btk)
            nq = W.make_queries(hk, 20000, 0.5, seed=500 + i).cuda()
            nout = torch.full_like(nq, 11)
            new_finds.append((pool.submit_find(bid, nq, nout), nq, nout, hk, hv))
        out = torch.full_like(q, 5)
        tickets.append(pool.submit_find(ids[t], q, out))
        mixed.append(out)
    for tk in tickets:
        assert pool.wait(tk, timeout=120)["status"] == 0
    for btk in builds:
        assert pool.wait(btk, timeout=120)["status"] == 0
    assert pool.stats()["builds_done"] >= len(tables) + len(builds)
    for (t, q), a, m in zip(reqs, alone, mixed):
        assert torch.equal(a, m)
        n, k, v = tables[t]
        assert (O._u32(m.cpu()) == O.lookup(k.cpu(), v.cpu(), q.cpu())).all()
    for ftk, nq, nout, hk, hv in new_finds:
        assert pool.wait(ftk, timeout=120)["status"] == 0
        assert (O._u32(nout.cpu()) == O.lookup(hk, hv, nq.cpu())).all()
    pool.close()
