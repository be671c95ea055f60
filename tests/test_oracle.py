"""Pins of the CPU oracle against facts fixed outside the oracle itself:
hand-derived hash values, primality, published generator outputs, the paper's
worked example (Fig. 1), the paper's printed probe counts, closed forms,
invariants and brute force on tiny inputs. CPU only."""

import json
import math
import os
import random

import numpy as np
import pytest

import oracle as O
import workloads as W

P = O.PRIME
EMPTY = O.EMPTY


def _read_rows(path):
    rows = []
    with open(path) as f:
        for line in f:
            body = line.split("#", 1)[0].strip()
            if body:
                rows.append(body.split())
    return rows


# --------------------------------------------------------------------- hash ---

def test_prime_is_the_largest_32bit_prime():
    """Section VII uses p = 4294967291: prime, and no prime lies above it below 2^32."""
    def is_prime(x):
        return x > 1 and all(x % d for d in range(2, math.isqrt(x) + 1))
    assert P == 2**32 - 5
    assert is_prime(P)
    assert not any(is_prime(q) for q in range(P + 1, 2**32))


def test_hash_hand_derived_vectors(golden_dir):
    for a, c, m, k, want in _read_rows(os.path.join(golden_dir, "hash_vectors.txt")):
        assert O.hash_value(int(a), int(c), int(m), int(k)) == int(want), (a, c, m, k)


def test_hash_identity_reduces_to_mod():
    """a = 1, c = 0 and k < p: h(k) = k mod m (a textbook remainder)."""
    rng = random.Random(1)
    for m in (1, 2, 3, 16, 72818, 2**31 - 1, 2**32 - 1):
        for _ in range(200):
            k = rng.randrange(0, P)
            assert O.hash_value(1, 0, m, k) == k % m


def test_hash_is_affine_mod_p():
    """With m >= p the outer mod is the identity, so h(k1) - h(k2) == a (k1 - k2) mod p
    and (for a != 0) h is injective on [0, p). A dropped term, a wrong sign or a
    swapped operand breaks one of these."""
    rng = random.Random(2)
    m = 2**32 - 1
    for _ in range(50):
        a, c = rng.randrange(1, P), rng.randrange(0, P)
        ks = [rng.randrange(0, 2**32) for _ in range(40)]
        hs = [O.hash_value(a, c, m, k) for k in ks]
        assert all(0 <= h < P for h in hs)
        for i in range(1, len(ks)):
            assert (hs[i] - hs[0] - a * (ks[i] - ks[0])) % P == 0
        assert (hs[0] - c - a * ks[0]) % P == 0
    a, c = 2654435761 % P, 12345
    ks = rng.sample(range(0, P), 20000)
    assert len({O.hash_value(a, c, m, k) for k in ks}) == len(ks)


def test_hash_collides_on_k_and_k_plus_p():
    for k in range(5):  # k + p < 2^32 only for k <= 4
        assert O.hash_value(123456789, 987654321, 1000, k) == O.hash_value(123456789, 987654321, 1000, k + P)


def test_hash_is_uniform_enough():
    """Chi-square over 97 buckets for 97,000 seeded random keys (loose bound)."""
    keys = O._u32(W.make_keys(97000, 11))
    a, c = O.derive_constants(3, 0, 1)
    counts = np.zeros(97)
    for k in keys[:97000]:
        counts[O.hash_value(a[0], c[0], 97, int(k))] += 1
    chi2 = ((counts - 1000.0) ** 2 / 1000.0).sum()
    assert chi2 < 96 + 6 * math.sqrt(2 * 96)


def test_splitmix64_published_vector(golden_dir):
    want = [int(r[0], 16) for r in _read_rows(os.path.join(golden_dir, "splitmix64_seed0.txt"))]
    assert O.splitmix64_stream(0, 3) == want


def test_derive_constants_ranges_and_attempts():
    seen = set()
    for seed in (0, 1, 0x676874):
        for attempt in range(5):
            a, c = O.derive_constants(seed, attempt, 4)
            assert all(1 <= x < P for x in a)
            assert all(0 <= x < P for x in c)
            seen.add(tuple(a + c))
    assert len(seen) == 15
    # attempt 0 draws straight from the generator seeded with the seed itself
    s = O.splitmix64_stream(42, 2)
    a, c = O.derive_constants(42, 0, 1)
    assert a[0] == 1 + s[0] % (P - 1) and c[0] == s[1] % P


def test_xorshift32_is_a_permutation_of_nonzero_states():
    xs = O.xorshift32_stream(2463534242, 200000)
    assert 0 not in xs
    assert len(set(xs)) == len(xs)


def test_xorshift32_hand_derived_vector(golden_dir):
    rows = _read_rows(os.path.join(golden_dir, "xorshift32_seed1.txt"))
    assert O.xorshift32_stream(1, len(rows)) == [int(r[0]) for r in rows]


def test_xorshift32_has_full_period():
    """Marsaglia (2003) lists (13, 17, 5) among the shift triples whose 32-bit
    xorshift generator has period 2^32 - 1. The step is linear over GF(2):
    its matrix T (column j = the step applied to bit j) must satisfy
    T^(2^32-1) = I and T^((2^32-1)/q) != I for every prime q dividing
    2^32 - 1 = 3 * 5 * 17 * 257 * 65537. A wrong shift amount or direction
    breaks this."""
    def step(x):
        return O.xorshift32_stream(x, 1)[0]

    rng = random.Random(5)
    for _ in range(100):
        x, y = rng.randrange(1, 2**32), rng.randrange(1, 2**32)
        if x != y:
            assert step(x ^ y) == step(x) ^ step(y)
    cols = [step(1 << j) for j in range(32)]

    def apply(m, v):
        r, j = 0, 0
        while v:
            if v & 1:
                r ^= m[j]
            v >>= 1
            j += 1
        return r

    def mul(a, b):  # a after b
        return [apply(a, bc) for bc in b]

    def power(m, e):
        r = [1 << j for j in range(32)]
        while e:
            if e & 1:
                r = mul(m, r)
            m = mul(m, m)
            e >>= 1
        return r

    ident = [1 << j for j in range(32)]
    order = 2**32 - 1
    assert power(cols, order) == ident
    for q in (3, 5, 17, 257, 65537):
        assert power(cols, order // q) != ident, q


def test_sizing(golden_dir):
    for n, lf, b, m in _read_rows(os.path.join(golden_dir, "sizing.txt")):
        assert O.num_buckets(int(n), float(lf), int(b)) == int(m), (n, lf, b)
    assert O.num_buckets(10, 0.0, 16) == 0
    assert O.num_buckets(10, 1.5, 16) == 0
    assert O.num_buckets(2**40, 0.5, 1) == 0  # more than 2^32 - 1 buckets


# ------------------------------------------------------- definitional lookup ---

def test_lookup_matches_a_dictionary():
    rng = np.random.default_rng(3)
    for n in (0, 1, 7, 1000):
        keys = rng.choice(2**32 - 1, size=n, replace=False).astype(np.uint32)
        vals = rng.integers(0, 2**32 - 1, size=n, dtype=np.uint64).astype(np.uint32)
        extra = rng.integers(0, 2**32, size=300, dtype=np.uint64).astype(np.uint32)
        q = np.concatenate([keys, keys[: n // 2], extra, np.array([EMPTY], np.uint32)])
        rng.shuffle(q)
        d = dict(zip(keys.tolist(), vals.tolist()))
        got = O.lookup(keys, vals, q)
        assert got.tolist() == [d.get(int(x), EMPTY) for x in q]


def test_lookup_rejects_sentinel_key():
    with pytest.raises(ValueError):
        O.lookup(np.array([1, EMPTY], np.uint32), np.array([1, 2], np.uint32), np.array([1], np.uint32))


# ------------------------------------------------------------ worked example ---

_SCHEMES = {"bcht": O.BCHT, "p2bht": O.P2BHT, "iht": O.IHT, "cuckoo1": O.CUCKOO1, "bcht_lb": O.BCHT_LB}


def _fixture_table(case):
    h, b, m = case["h"], case["b"], case["m"]
    top = max(int(k) for k in case["hashes"]) + 1
    eb = np.zeros((top, h), dtype=np.uint32)
    for k, hs in case["hashes"].items():
        eb[int(k)] = hs
    T = O.Table(_SCHEMES[case["scheme"]], 16, 1.0, b=b, h=h, m=m, t=case.get("t"),
                explicit_buckets=eb, max_chain=case.get("max_chain", 8))
    T.slots[:] = O.EMPTY_PAIR
    for bi, ks in enumerate(case["initial"]):
        for s, k in enumerate(ks):
            T.slots[bi * b + s] = (np.uint64(1000 + k) << np.uint64(32)) | np.uint64(k)
    return T


def _bucket_of(T, key):
    for i, pair in enumerate(T.slots):
        if int(pair) & 0xFFFFFFFF == key:
            return i // T.b
    return None


def test_fig1_worked_examples(golden_dir):
    with open(os.path.join(golden_dir, "fig1_examples.json")) as f:
        spec = json.load(f)
    for case in spec["cases"]:
        T = _fixture_table(case)
        before = {int(p) & 0xFFFFFFFF: i // T.b for i, p in enumerate(T.slots) if int(p) != O.EMPTY_PAIR}
        ok = T.insert(case["insert"], 1000 + case["insert"], rng_state=12345)
        e = case["expect"]
        assert ok == e["ok"], case["name"]
        assert T.stats.probes == e["probes"], case["name"]
        assert T.stats.evictions == e["evictions"], case["name"]
        assert [T.load(i) for i in range(T.m)] == e["bucket_loads"], case["name"]
        for k, bkt in e.get("key_in_bucket", {}).items():
            assert _bucket_of(T, int(k)) == bkt, case["name"]
        if "moved_from" in e:
            moved = [k for k, bkt in before.items() if _bucket_of(T, k) != bkt]
            assert len(moved) == 1 and before[moved[0]] == e["moved_from"]
            assert _bucket_of(T, moved[0]) == e["moved_to"]
        if "moves" in e:  # (from, to) of every key that changed bucket
            moves = sorted([before[k], _bucket_of(T, k)] for k in before if _bucket_of(T, k) != before[k])
            assert moves == sorted(e["moves"]), case["name"]
        # values travel with their keys
        for pair in T.slots:
            if int(pair) != O.EMPTY_PAIR:
                assert (int(pair) >> 32) == 1000 + (int(pair) & 0xFFFFFFFF)


# --------------------------------------------------- paper's probe counts ---

@pytest.fixture(scope="module")
def probe_inputs():
    n = 1 << 20
    keys, vals = W.make_keys(n, 1), W.make_values(n, 1)
    qpos = W.make_queries(keys, n, 1.0, 3)
    qneg = W.make_negatives(n, n, 1)
    return n, keys, vals, qpos, qneg


def test_probe_counts_match_the_paper(golden_dir, probe_inputs):
    n, keys, vals, qpos, qneg = probe_inputs
    schemes = {"bcht": O.BCHT, "p2bht": O.P2BHT, "iht": O.IHT, "cuckoo1": O.CUCKOO1}
    built = {}
    for row in _read_rows(os.path.join(golden_dir, "paper_probe_counts.txt")):
        scheme, b, h, t, lf, op, want, tol = row[:8]
        key = (scheme, b, h, t, lf)
        if key not in built:
            T = O.Table(schemes[scheme], n, float(lf), seed=5, b=int(b), h=int(h),
                        t=int(t) if scheme == "iht" else None)
            assert T.build(keys, vals) == 1, key
            built[key] = T
        T = built[key]
        if op == "insert":
            got = T.stats.probes / n
        elif op == "find_pos":
            got = T.find(qpos)[2] / n
        else:
            got = T.find(qneg)[2] / n
        assert abs(got - float(want)) <= float(tol) + 1e-9, (row, got)


def test_find_closed_forms(probe_inputs):
    """Negative finds: exactly 2 probes for P2BHT and 3 for IHT and the
    load-balanced BCHT (no early exit, Sec. III-A last paragraph), at most h
    for BCHT; 50 % positive = mean of 0 % and 100 %."""
    n, keys, vals, qpos, qneg = probe_inputs
    for scheme, lf, neg_exact in ((O.P2BHT, 0.8, 2), (O.IHT, 0.86, 3), (O.BCHT, 0.95, None),
                                  (O.BCHT_LB, 0.95, 3)):
        T = O.Table(scheme, n, lf, seed=9)
        assert T.build(keys, vals) == 1
        vpos, pp, tp = T.find(qpos)
        vneg, pn, tn = T.find(qneg)
        assert (vneg == EMPTY).all()
        if neg_exact:
            assert (pn == neg_exact).all()
        else:
            assert pn.max() <= 3 and pn.min() >= 1
        assert pp.min() >= 1 and pp.max() <= T.h
        half = np.concatenate([O._u32(qpos)[: n // 2], O._u32(qneg)[: n // 2]])
        th = T.find(half)[2]
        assert th == pp[: n // 2].sum() + pn[: n // 2].sum()


def test_bcht_reaches_098_on_every_seed():
    """Section VII-C: BCHT builds at load factor 0.98 in about 99 % of runs."""
    n = 1 << 16
    keys, vals = W.make_keys(n, 21), W.make_values(n, 21)
    ok = sum(O.Table(O.BCHT, n, 0.98, seed=s).build(keys, vals) == 1 for s in range(20))
    assert ok >= 19


def test_schemes_fail_beyond_their_reach():
    """Section VII-A2/A3: b = 16 P2BHT and IHT cannot reach load factor 0.9+;
    1CHT with three hash functions cannot reach 0.95 (the h = 3, b = 1
    orientability threshold is about 0.918)."""
    n = 1 << 16
    keys, vals = W.make_keys(n, 4), W.make_values(n, 4)
    assert O.Table(O.P2BHT, n, 0.95, seed=1).build(keys, vals) == 0
    assert O.Table(O.IHT, n, 0.95, seed=1).build(keys, vals) == 0
    assert O.Table(O.CUCKOO1, n, 0.95, seed=1).build(keys, vals) == 0
    T = O.Table(O.BCHT, n, 0.99, seed=1, max_chain=0)
    assert T.build(keys, vals) == 0 and T.stats.failed_at >= 0


def test_sentinel_key_is_rejected():
    T = O.Table(O.BCHT, 4, 0.5, seed=1)
    assert T.build(np.array([1, EMPTY], np.uint32), np.array([5, 6], np.uint32)) == -1


def test_sentinel_query_returns_empty_without_probes():
    T = O.Table(O.BCHT, 4, 0.5, seed=1)
    T.build(np.array([1, 2], np.uint32), np.array([5, 6], np.uint32))
    v, pe, tot = T.find(np.array([EMPTY, 1], np.uint32))
    assert v.tolist() == [EMPTY, 5] and pe[0] == 0


# --------------------------------------------------------------- invariants ---

@pytest.mark.parametrize("scheme,lf", [(O.BCHT, 0.99), (O.P2BHT, 0.8), (O.IHT, 0.86),
                                       (O.CUCKOO1, 0.85), (O.BCHT_LB, 0.99)])
def test_builds_pass_the_validator_and_find_matches_lookup(scheme, lf):
    n = 1 << 16
    keys, vals = W.make_keys(n, 8), W.make_values(n, 8)
    T = O.Table(scheme, n, lf, seed=2)
    assert T.build(keys, vals) == 1
    ok, msg = T.validate(keys, vals)
    assert ok, msg
    q = W.make_queries(keys, 5000, 0.5, 4)
    assert (T.find(q)[0] == O.lookup(keys, vals, q)).all()


def _corrupt(T, how):
    s = T.slots
    full = np.flatnonzero(s != np.uint64(O.EMPTY_PAIR))
    empty = np.flatnonzero(s == np.uint64(O.EMPTY_PAIR))
    i = int(full[0])
    if how == "half_empty":
        s[i] = np.uint64(O.EMPTY_PAIR) & ~np.uint64(1 << 40)
    elif how == "wrong_bucket":
        k = int(s[i]) & 0xFFFFFFFF
        cands = {T.bucket(j, k) for j in range(T.h)}
        dest = next(int(e) for e in empty if int(e) // T.b not in cands)
        s[dest], s[i] = s[i], np.uint64(O.EMPTY_PAIR)
    elif how == "duplicate":
        s[int(empty[0])] = s[i]
    elif how == "lost":
        s[i] = np.uint64(O.EMPTY_PAIR)
    elif how == "value":
        s[i] = s[i] ^ np.uint64(1 << 33)


@pytest.mark.parametrize("how", ["half_empty", "wrong_bucket", "duplicate", "lost", "value"])
def test_validator_catches_planted_mistakes(how):
    n = 2000
    keys, vals = W.make_keys(n, 5), W.make_values(n, 5)
    T = O.Table(O.BCHT, n, 0.8, seed=1)
    assert T.build(keys, vals) == 1
    _corrupt(T, how)
    ok, msg = T.validate(keys, vals)
    assert not ok and msg


def test_validator_catches_broken_early_exit_invariant():
    """A key stored at H_1 while H_0 still has room would make early-exit find miss it."""
    n = 3000
    keys, vals = W.make_keys(n, 6), W.make_values(n, 6)
    T = O.Table(O.BCHT, n, 0.5, seed=1)
    assert T.build(keys, vals) == 1
    s = T.slots
    for i, pair in enumerate(s):
        k = int(pair) & 0xFFFFFFFF
        if int(pair) == O.EMPTY_PAIR:
            continue
        b0, b1 = T.bucket(0, k), T.bucket(1, k)
        if b0 != b1 and T.load(b1) < T.b:
            dest = b1 * T.b + T.load(b1)
            s[dest], s[i] = pair, np.uint64(O.EMPTY_PAIR)
            break
    ok, msg = T.validate(keys, vals)
    assert not ok and "not full" in msg


def test_validator_catches_broken_iht_threshold_invariant():
    """Sec. III-C: a key goes to a secondary bucket only when its primary
    would reach t keys. A key moved from its primary (holding fewer than
    t - 1 keys) to a secondary with room breaks this, and the validator says
    so."""
    n = 3000
    keys, vals = W.make_keys(n, 6), W.make_values(n, 6)
    T = O.Table(O.IHT, n, 0.6, seed=1)
    assert T.build(keys, vals) == 1 and T.params.t == 13
    assert T.validate(keys, vals)[0]
    s = T.slots
    for i, pair in enumerate(s):
        if int(pair) == O.EMPTY_PAIR:
            continue
        k = int(pair) & 0xFFFFFFFF
        bp, bs = T.bucket(0, k), T.bucket(1, k)
        if i // T.b == bp and bs != bp and T.load(bp) <= T.params.t - 1 and T.load(bs) < T.b:
            dest = bs * T.b + next(j for j in range(T.b) if int(s[bs * T.b + j]) == O.EMPTY_PAIR)
            s[dest], s[i] = pair, np.uint64(O.EMPTY_PAIR)
            break
    else:
        pytest.fail("no key to move")
    ok, msg = T.validate(keys, vals)
    assert not ok and "primary" in msg


# -------------------------------------------------------------- brute force ---

def _orientable(cands, m, b):
    """Exhaustive search: can every key take one of its candidate buckets
    without any bucket exceeding b keys?"""
    loads = [0] * m
    order = sorted(range(len(cands)), key=lambda i: len(set(cands[i])))

    def rec(j):
        if j == len(order):
            return True
        for bkt in sorted(set(cands[order[j]])):
            if loads[bkt] < b:
                loads[bkt] += 1
                if rec(j + 1):
                    return True
                loads[bkt] -= 1
        return False
    return rec(0)


def _independent_layout_check(T, cands, n):
    where = {}
    for i, pair in enumerate(T.slots):
        if int(pair) == O.EMPTY_PAIR:
            continue
        k = int(pair) & 0xFFFFFFFF
        assert k not in where
        where[k] = i // T.b
    assert sorted(where) == list(range(n))
    for k, bkt in where.items():
        assert bkt in cands[k]


def test_bcht_brute_force_tiny_tables():
    rng = random.Random(7)
    solvable = solved = 0
    for trial in range(400):
        m, b, h = rng.randint(1, 4), rng.randint(1, 3), rng.randint(2, 3)
        n = rng.randint(1, min(12, m * b))
        cands = [[rng.randrange(m) for _ in range(h)] for _ in range(n)]
        T = O.Table(O.BCHT, 16, 1.0, b=b, h=h, m=m, explicit_buckets=np.array(cands, np.uint32),
                    max_chain=2000)
        T.params.rng_seed = rng.randrange(1, 2**32)
        ok = T.build(np.arange(n, dtype=np.uint32), np.arange(n, dtype=np.uint32) + 7)
        orientable = _orientable(cands, m, b)
        if ok == 1:
            assert orientable
            _independent_layout_check(T, cands, n)
            assert T.validate(np.arange(n, dtype=np.uint32), np.arange(n, dtype=np.uint32) + 7)[0]
        else:
            assert ok == 0
        if orientable and b >= 2:
            solvable += 1
            solved += ok == 1
    assert solvable > 50 and solved >= 0.95 * solvable


@pytest.mark.parametrize("scheme", [O.P2BHT, O.IHT])
def test_stable_schemes_brute_force_tiny_tables(scheme):
    """Greedy schemes may fail on a solvable instance, never succeed on an
    unsolvable one, and every success is a valid layout."""
    rng = random.Random(11 + scheme)
    for trial in range(300):
        m, b = rng.randint(1, 4), rng.randint(1, 3)
        h = 2 if scheme == O.P2BHT else 3
        n = rng.randint(1, min(12, m * b))
        cands = [[rng.randrange(m) for _ in range(h)] for _ in range(n)]
        T = O.Table(scheme, 16, 1.0, b=b, h=h, m=m, t=rng.randint(1, b + 1),
                    explicit_buckets=np.array(cands, np.uint32))
        ok = T.build(np.arange(n, dtype=np.uint32), np.arange(n, dtype=np.uint32))
        if ok == 1:
            assert _orientable(cands, m, b)
            _independent_layout_check(T, cands, n)
        if not _orientable(cands, m, b):
            assert ok == 0


def test_chain_bound_is_exact(golden_dir):
    """Section III-A: the build fails once the maximum number of exchanges is
    reached. Fig. 1(b) needs exactly one exchange: a bound of 1 suffices, a
    bound of 0 fails after reading the one full bucket."""
    with open(os.path.join(golden_dir, "fig1_examples.json")) as f:
        case = next(c for c in json.load(f)["cases"] if c["name"] == "bcht_fig1b")
    for bound, ok, probes, evictions in ((0, 0, 1, 0), (1, 1, 2, 1)):
        T = _fixture_table(case)
        T.params.max_chain = bound
        assert T.insert(7, 1007, rng_state=99) == ok
        assert (T.stats.probes, T.stats.evictions) == (probes, evictions)


@pytest.mark.parametrize("lf", [0.9, 0.99])
def test_two_phase_order_is_a_bcht_insertion_order(lf):
    """The two-phase GPU build is sequential BCHT (Sec. III-A) with the keys
    permuted: first every key that reaches its first-choice bucket H_0 while
    fewer than b keys have (arrival rank < b), then the rest, each part in
    input order. In the first part no bucket is full, so each insert is one
    probe with no eviction and lands in slot `rank` of H_0; the whole order
    builds a valid table whose finds equal the definitional lookup, with an
    insert probe average close to input order's."""
    n = 1 << 16
    keys, vals = W.make_keys(n, 17), W.make_values(n, 17)
    k = O._u32(keys).astype(np.uint64)
    T = O.Table(O.BCHT, n, lf, seed=5)
    a, c = T.constants()
    h0 = ((np.uint64(a[0]) * k + np.uint64(c[0])) % np.uint64(O.PRIME)) % np.uint64(T.m)
    # arrival rank of each key at its H_0, in input order
    order = np.argsort(h0, kind="stable")
    sorted_h0 = h0[order]
    first = np.searchsorted(sorted_h0, sorted_h0, side="left")
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n) - first
    placed = rank < T.b
    assert 0.03 * n < (~placed).sum() < 0.15 * n  # the overflow of the first part
    # part one alone: one probe per key, no eviction, slot = arrival rank
    P = O.Table(O.BCHT, n, lf, seed=5)
    assert P.build(keys[placed], vals[placed]) == 1
    assert P.stats.probes == placed.sum() and P.stats.evictions == 0
    slots = P.slots.reshape(P.m, P.b)
    kp = O._u32(keys)[placed]
    assert (slots[h0[placed].astype(np.int64), rank[placed]] & np.uint64(0xFFFFFFFF) == kp).all()
    # the whole permuted order
    perm = np.concatenate([np.flatnonzero(placed), np.flatnonzero(~placed)])
    R = O.Table(O.BCHT, n, lf, seed=5)
    assert R.build(keys[perm], vals[perm]) == 1
    ok, msg = R.validate(keys, vals)
    assert ok, msg
    q = W.make_queries(keys, n, 0.5, seed=3)
    assert (R.find(q)[0] == O.lookup(keys, vals, q)).all()
    S = O.Table(O.BCHT, n, lf, seed=5)
    assert S.build(keys, vals) == 1
    assert abs(R.stats.probes - S.stats.probes) / n < 0.03, (R.stats.probes / n, S.stats.probes / n)
