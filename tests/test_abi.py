"""CPU-side checks of the C-ABI library: it builds, loads, exports every entry
point include/ght.h declares, and its host-side arithmetic (sizing, the hash
family with its divide-free remainders) agrees with the oracle. No GPU call."""

import os
import random
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2108_07232_gb300 import build
    build.build()
    import paper_2108_07232_gb300 as G
    return G


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"\b(ght_[a-z_0-9]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(L):
    lib = L.lib()
    declared = _declared()
    assert {"ght_create", "ght_build", "ght_find", "ght_stats", "ght_destroy"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), name


def test_version_and_defaults(L):
    assert "sm_103a" in L.ght_version()
    c = L.ght_default_config(L.BCHT)
    assert (c.bucket_size, c.num_hashes, c.max_chain, c.max_attempts) == (16, 3, 1000, 50)
    c = L.ght_default_config(L.IHT)
    assert (c.bucket_size, c.num_hashes, c.threshold) == (16, 3, 13)
    c = L.ght_default_config(L.CUCKOO1)
    assert (c.bucket_size, c.num_hashes) == (1, 3)
    with pytest.raises(L.GhtError):
        L.ght_default_config(9)


@pytest.mark.parametrize("scheme,b", [(0, 16), (1, 16), (2, 16), (3, 1), (4, 16)])
def test_table_bytes_follow_the_oracle_sizing(L, scheme, b):
    for n, lf in [(1 << 20, 0.9), (268435456, 0.99), (1000, 0.6), (0, 0.5), (17, 1.0)]:
        m = O.num_buckets(n, lf, b)
        slots = m * b * 8
        assert L.ght_table_bytes(scheme, n, lf) == 256 + ((slots + 255) // 256) * 256


def test_keys_only_set_uses_four_byte_slots(L):
    for n, lf in [(1 << 20, 0.9), (1000, 0.99), (0, 0.5)]:
        m = O.num_buckets(n, lf, 32)
        assert L.ght_table_bytes(5, n, lf) == 256 + ((m * 32 * 4 + 255) // 256) * 256
    assert L.ght_table_bytes(5, 100, 0.9, {"bucket_size": 16}) == 0


def test_table_bytes_rejects_bad_shapes(L):
    assert L.ght_table_bytes(0, 100, 0.0) == 0
    assert L.ght_table_bytes(0, 100, 1.01) == 0
    assert L.ght_table_bytes(0, 100, 0.9, {"bucket_size": 8}) == 0
    assert L.ght_table_bytes(1, 100, 0.9, {"num_hashes": 3}) == 0
    assert L.ght_table_bytes(3, 2**40, 0.5) == 0
    assert L.ght_table_bytes(0, 100, 0.9, {"tile_lanes": 2}) == 0
    assert L.ght_table_bytes(0, 100, 0.9, {"bucket_size": 32, "tile_lanes": 4}) == 0
    assert L.ght_table_bytes(2, 100, 0.9, {"bucket_size": 32}) > 0  # IHT b = 32, t = 26


def test_staged_find_shapes(L):
    """The staged find applies to 128-byte buckets read by 4-lane tiles with
    2..8 query sets per lane; every other combination is refused before any
    device call (the sizing itself is unchanged by it)."""
    ok = L.ght_table_bytes(0, 1000, 0.9)
    for kpl in range(2, 9):
        assert L.ght_table_bytes(0, 1000, 0.9, {"find_async": 1, "keys_per_lane": kpl}) == ok
    assert L.ght_table_bytes(0, 1000, 0.9, {"find_async": 1, "keys_per_lane": 1}) == 0
    assert L.ght_table_bytes(0, 1000, 0.9, {"find_async": 1, "keys_per_lane": 9}) == 0
    assert L.ght_table_bytes(0, 1000, 0.9, {"find_async": 1, "tile_lanes": 16}) == 0
    assert L.ght_table_bytes(0, 1000, 0.9, {"find_async": 1, "bucket_size": 32, "tile_lanes": 8}) == 0
    for scheme in (0, 1, 2, 4):  # BCHT, P2BHT, IHT, load-balanced BCHT; 4-lane tiles
        for b, most in ((16, 8), (32, 6)):  # sets in flight: 2..8, or 2..6 for 256-byte buckets
            base = L.ght_table_bytes(scheme, 1000, 0.8, {"bucket_size": b})
            assert base > 0
            assert L.ght_table_bytes(scheme, 1000, 0.8, {"find_async": 1, "bucket_size": b}) == base
            assert L.ght_table_bytes(scheme, 1000, 0.8, {"find_async": 1, "bucket_size": b,
                                                         "keys_per_lane": most}) == base
            assert L.ght_table_bytes(scheme, 1000, 0.8, {"find_async": 1, "bucket_size": b,
                                                         "keys_per_lane": most + 1}) == 0
            assert L.ght_table_bytes(scheme, 1000, 0.8, {"find_async": 1, "bucket_size": b, "tile_lanes": 8}) == 0
        if scheme:
            assert L.ght_table_bytes(scheme, 1000, 0.8, {"tile_lanes": 4}) == 0  # register find: 8-lane tiles
    assert L.ght_table_bytes(3, 1000, 0.8, {"find_async": 1}) == 0  # 1CHT
    # the register find keeps 1..2 sets per lane
    assert L.ght_table_bytes(0, 1000, 0.9, {"find_async": -1, "keys_per_lane": 3}) == 0
    # the keys-only set: 4-lane find tiles only with the staged find
    set_ok = L.ght_table_bytes(5, 1000, 0.9)
    assert L.ght_table_bytes(5, 1000, 0.9, {"find_async": 1}) == set_ok
    assert L.ght_table_bytes(5, 1000, 0.9, {"find_async": 1, "tile_lanes": 4, "keys_per_lane": 8}) == set_ok
    assert L.ght_table_bytes(5, 1000, 0.9, {"find_async": 1, "tile_lanes": 8}) == 0
    assert L.ght_table_bytes(5, 1000, 0.9, {"find_async": -1, "tile_lanes": 4}) == 0
    assert L.ght_table_bytes(5, 1000, 0.9, {"tile_lanes": 4}) == 0  # small: no staged find by default


def _host_hash(L, a, c, m, keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    out = np.empty_like(keys)
    L.ght_hash_host(a, c, m, keys, out, keys.size)
    return out


def test_host_hash_matches_golden_vectors(L, golden_dir):
    for line in open(os.path.join(golden_dir, "hash_vectors.txt")):
        body = line.split("#", 1)[0].split()
        if body:
            a, c, m, k, want = map(int, body)
            assert _host_hash(L, a, c, m, [k])[0] == want, (a, c, m, k)


def test_host_hash_matches_oracle_on_random_and_edge_operands(L):
    """The library's divide-free remainders (fold mod p, Lemire mod m) against
    the oracle's plain 64-bit `%`, over random and boundary operands."""
    rng = random.Random(5)
    ms = [1, 2, 3, 5, 7, 16, 72818, 1 << 20, 16946683, 2**31 - 1, 2**31, 2**31 + 1,
          2**32 - 5, 2**32 - 2, 2**32 - 1] + [rng.randrange(1, 2**32) for _ in range(20)]
    edge_k = [0, 1, 2, 3, 4, 5, 2**31 - 1, 2**31, 2**32 - 6, 2**32 - 5, 2**32 - 4, 2**32 - 2, 2**32 - 1]
    keys = np.array(edge_k + [rng.randrange(0, 2**32) for _ in range(3000)], dtype=np.uint32)
    consts = [(1, 0), (O.PRIME - 1, O.PRIME - 1), (2**32 - 1, 2**32 - 1), (2**31, 5)] + \
             [(rng.randrange(1, O.PRIME), rng.randrange(0, O.PRIME)) for _ in range(6)]
    for m in ms:
        for a, c in consts:
            got = _host_hash(L, a, c, m, keys)
            want = [O.hash_value(a, c, m, int(k)) for k in keys[:400]]
            assert got[:400].tolist() == want, (a, c, m)
            # the rest in bulk with numpy's exact uint64 arithmetic on small products
            if a < 2**16:
                x = (np.uint64(a) * keys.astype(np.uint64) + np.uint64(c)) % np.uint64(O.PRIME) % np.uint64(m)
                assert (got == x.astype(np.uint32)).all()


def test_host_hash_rejects_zero_buckets(L):
    with pytest.raises(L.GhtError):
        L.ght_hash_host(1, 0, 0, np.zeros(1, np.uint32), np.zeros(1, np.uint32), 1)


def test_probe_lines_rejects_bad_arguments_before_any_device_call(L):
    """The access-pattern probe validates mode, pointer alignment and line
    count on the host; with ops = 0 a valid call is a no-op. No GPU call."""
    aligned, misaligned = 1 << 20, (1 << 20) + 8  # never dereferenced: rejected or no-op
    for mode, ptr, lines in [(-1, aligned, 16), (6, aligned, 16), (0, 0, 16), (0, misaligned, 16),
                             (0, aligned, 0), (0, aligned, 2**32)]:
        with pytest.raises(L.GhtError) as e:
            L.ght_probe_lines(mode, ptr, lines, 1, 1, 0)
        assert e.value.status == "GHT_ERR_INVALID_ARG", (mode, ptr, lines)
    for mode in range(6):
        L.ght_probe_lines(mode, aligned, 16, 0, 1, 0)  # ops = 0: nothing to do



def test_unknown_table_options_are_rejected(L):
    """A misspelt option must not be dropped silently: the binding refuses
    names that are not fields of ght_config (before any device call)."""
    with pytest.raises(TypeError):
        L.ght_table_bytes(0, 1000, 0.9, {"find_asynk": 1})
    with pytest.raises(TypeError):
        L.ght_table_bytes(0, 1000, 0.9, {"reserved": 0})
    assert L.ght_table_bytes(0, 1000, 0.9, {"check_duplicates": 1}) == L.ght_table_bytes(0, 1000, 0.9)


def _header():
    return open(os.path.join(ROOT, "include", "ght.h")).read()


def test_noalloc_capacity_matches_the_header(L):
    """The binding's copy of GHT_NOALLOC_MAX_QUERIES is the header's value."""
    m = re.search(r"#define\s+GHT_NOALLOC_MAX_QUERIES\s+\((\d+)u\s*<<\s*(\d+)\)", _header())
    assert m, "GHT_NOALLOC_MAX_QUERIES not found in ght.h"
    assert L.NOALLOC_MAX_QUERIES == int(m.group(1)) << int(m.group(2))


def _struct_fields(src, name):
    end = re.search(r"\}\s*" + name + ";", src).start()
    body = src[src.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        typ, ptr, names = re.match(r"(?:const\s+)?(\w+)\s*(\*?)\s*(.*)", decl, re.S).groups()
        for nm in names.split(","):
            nm = nm.strip()
            arr = re.match(r"(\w+)\[(\d+)\]", nm)
            t = "pointer" if ptr else typ
            fields.append((arr.group(1), t, int(arr.group(2))) if arr else (nm, t, 1))
    return fields


@pytest.mark.parametrize("cname,pyname", [("ght_config", "GhtConfig"), ("ght_stats_t", "GhtStats"),
                                          ("ght_batch_stats_t", "GhtBatchStats"),
                                          ("ght_pool_result_t", "GhtPoolResult"),
                                          ("ght_pool_stats_t", "GhtPoolStats"),
                                          ("ght_pool_request_t", "GhtPoolRequest")])
def test_binding_structs_follow_the_header(L, cname, pyname):
    """Each ctypes structure of the binding lists the header's fields in the
    header's order with the same sizes, so no field is read from the wrong
    offset."""
    import ctypes as C

    from paper_2108_07232_gb300 import _binding
    sizes = {"int32_t": 4, "uint32_t": 4, "uint64_t": 8, "double": 8, "pointer": C.sizeof(C.c_void_p)}
    want = _struct_fields(_header(), cname)
    got = getattr(_binding, pyname)._fields_
    assert [f[0] for f in want] == [g[0] for g in got]
    for (name, typ, count), (_, ctype) in zip(want, got):
        assert C.sizeof(ctype) == sizes[typ] * count, name
