"""The allocation-free host find (ght_find_host_noalloc) against the existing
host find (ght_find_host), both called through the C ABI.

Callers that may not use the CUDA allocator while they run -- a plugin's
execute step in an inference server, or code running while another pool
owns device memory -- use the allocation-free entry point; it must return
exactly what the allocating one returns. Two calls in a row check that the
shared static staging array carries nothing from one call into the next.
This file is collected last so that a failure here stops a `-x` run only
after every other test has run."""

import ctypes as C

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


def _raw_find(lib, fn, handle, q: np.ndarray) -> tuple[int, np.ndarray]:
    out = np.full(q.size, 0x12345678, dtype=np.uint32)
    rc = getattr(lib, fn)(C.c_void_p(handle), q.ctypes.data_as(C.c_void_p),
                          out.ctypes.data_as(C.c_void_p), C.c_uint64(q.size))
    return rc, out


def test_no_alloc_find_matches_the_allocating_host_find(G):
    lib = G.lib()
    n = 1 << 20
    keys, vals = W.make_keys(n, 77), W.make_values(n, 77)
    t = G.HashTable("bcht", n, 0.97, seed=5)
    t.build(keys.cuda(), vals.cuda())
    torch.cuda.synchronize()
    # two calls in a row with different sizes and query mixes; the second is
    # shorter, so stale entries of the first would show in its results
    for call, (nq, frac, seed) in enumerate([((1 << 20) + 3, 0.5, 1), (5000, 0.9, 2)]):
        q = W.make_queries(keys, nq, frac, seed).numpy().view(np.uint32).copy()
        rc_na, out_na = _raw_find(lib, "ght_find_host_noalloc", t._t, q)
        assert rc_na == 0, lib.ght_last_error().decode()
        rc_ref, out_ref = _raw_find(lib, "ght_find_host", t._t, q)
        assert rc_ref == 0, lib.ght_last_error().decode()
        assert np.array_equal(out_na, out_ref), call
        # every answer is the value stored with the query's key, or the
        # sentinel for a key that was not inserted
        assert np.array_equal(out_na, O.lookup(keys, vals, q)), call


@pytest.mark.parametrize("cfg", [{}, {"find_grouped": 1}])
def test_no_alloc_find_allocates_nothing_on_the_device(G, cfg):
    """After a first call (and the table's creation, which reserves the
    staging array), further calls leave the device's free memory unchanged:
    nothing is allocated from the driver, torch or the library's pool. On a
    table set for the grouped find, whose scratch would come from an
    allocator, this entry point still finds per query."""
    lib = G.lib()
    n = 1 << 18
    keys, vals = W.make_keys(n, 79), W.make_values(n, 79)
    t = G.HashTable("bcht", n, 0.9, seed=6, **cfg)
    t.build(keys.cuda(), vals.cuda())
    q = W.make_queries(keys, 1 << 21, 0.5, 3).numpy().view(np.uint32).copy()
    rc, _ = _raw_find(lib, "ght_find_host_noalloc", t._t, q)
    assert rc == 0, lib.ght_last_error().decode()
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    reserved_before = torch.cuda.memory_reserved()
    for _ in range(2):
        rc, out = _raw_find(lib, "ght_find_host_noalloc", t._t, q)
        assert rc == 0, lib.ght_last_error().decode()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    assert torch.cuda.memory_reserved() == reserved_before
    assert np.array_equal(out, O.lookup(keys, vals, q))
    assert t.stats()["last_find_grouped"] == 0


def test_no_alloc_find_rejects_batches_beyond_the_staging_array(G):
    lib = G.lib()
    n = 1000
    keys, vals = W.make_keys(n, 78), W.make_values(n, 78)
    t = G.HashTable("bcht", n, 0.9, seed=5)
    t.build(keys.cuda(), vals.cuda())
    too_many = np.zeros(G.NOALLOC_MAX_QUERIES + 1, dtype=np.uint32)
    rc, out = _raw_find(lib, "ght_find_host_noalloc", t._t, too_many)
    assert rc == 8  # GHT_ERR_CAPACITY
    assert "static staging array" in lib.ght_last_error().decode()
    assert (out == 0x12345678).all()  # nothing was written
    rc, _ = _raw_find(lib, "ght_find_host_noalloc", t._t, np.zeros(0, dtype=np.uint32))
    assert rc == 0
