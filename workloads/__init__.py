"""Seeded synthetic inputs for the static hash-table path.

This module is test-data generation only. It holds none of the hash table's
arithmetic (no table hash family, no sizing, no placement rule), so both the
CPU oracle's tests and the GPU path may consume its arrays without sharing any
of the method's code.

The paper's workload (Section VII) is 32-bit unique random keys and 32-bit random
values, with query streams that are 100 %, 50 % or 0 % positive. Here:

* keys      = F_s(i), i = 0, 1, ...: a seeded 6-round Feistel bijection on 32-bit
              words, so keys are unique by construction; the one index that
              maps to the sentinel 0xFFFFFFFF is skipped.
* negatives = F_s(i) for indices after the keys, hence disjoint from them.
* values    = G_s(i), an independent mixer; the sentinel is replaced by 0
              (a stored sentinel value would be indistinguishable from
              "not found").
* queries   = round(f * N) positives drawn uniformly with replacement from the
              keys, then negatives, then a seeded permutation of the positions.

Every step is a counter-based integer function evaluated with int64 torch ops,
so CPU and CUDA produce identical arrays for the same seed.
Arrays are returned as int32 tensors that carry the uint32 bit patterns.
"""

from __future__ import annotations

import torch

SENTINEL = 0xFFFFFFFF
_M32 = 0xFFFFFFFF
_M16 = 0xFFFF


def _splitmix64_stream(seed: int, count: int) -> list[int]:
    """Round keys for the generators (Steele, Lea, Flood 2014 SplitMix64)."""
    m64 = (1 << 64) - 1
    out = []
    s = seed & m64
    for _ in range(count):
        s = (s + 0x9E3779B97F4A7C15) & m64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m64
        out.append(z ^ (z >> 31))
    return out


def _round_fn(r: torch.Tensor, k: int) -> torch.Tensor:
    """Feistel round function on 16-bit halves; any function keeps the bijection."""
    x = (r ^ (k & _M16)) * 0x85EBCA6B  # < 2^48, exact in int64
    x = (x ^ (x >> 15)) & _M32
    x = ((x & _M16) * 0xC2B2AE35) ^ (x >> 16) ^ ((k >> 16) & _M16)
    return (x ^ (x >> 13)) & _M16


def feistel32(i: torch.Tensor, seed: int, rounds: int = 6) -> torch.Tensor:
    """Seeded bijection on [0, 2^32); ``i`` is an int64 tensor of values < 2^32."""
    ks = _splitmix64_stream(seed ^ 0x46656973746C, rounds)
    left = (i >> 16) & _M16
    right = i & _M16
    for r in range(rounds):
        left, right = right, left ^ _round_fn(right, ks[r] & _M32)
    return (left << 16) | right


def mix32(i: torch.Tensor, seed: int) -> torch.Tensor:
    """Counter-based 32-bit mixer (not a bijection); ``i`` int64 < 2^32."""
    k = _splitmix64_stream(seed ^ 0x6D69783332, 2)
    x = (i ^ (k[0] & _M32)) & _M32
    x = (((x & _M16) * 0x7FEB352D) + ((((x >> 16) * 0x7FEB352D) & _M16) << 16)) & _M32
    x = x ^ (x >> 15)
    x = (((x & _M16) * 0x846CA68B) + ((((x >> 16) * 0x846CA68B) & _M16) << 16)) & _M32
    x = x ^ (x >> 16) ^ (k[1] & _M32)
    return x & _M32


def to_u32_bits(x: torch.Tensor) -> torch.Tensor:
    """int64 values in [0, 2^32) -> int32 tensor with the same bit pattern."""
    return torch.where(x >= (1 << 31), x - (1 << 32), x).to(torch.int32)


def from_u32_bits(x: torch.Tensor) -> torch.Tensor:
    """int32 tensor carrying uint32 bits -> int64 values in [0, 2^32)."""
    return x.to(torch.int64) & _M32


def _unique_words(start: int, count: int, seed: int, device) -> torch.Tensor:
    """``count`` distinct non-sentinel words F_s(start), F_s(start+1), ..."""
    if count == 0:
        return torch.empty(0, dtype=torch.int64, device=device)
    idx = torch.arange(start, start + count + 1, dtype=torch.int64, device=device)
    w = feistel32(idx, seed)
    w = w[w != SENTINEL]
    return w[:count]


def make_keys(n: int, seed: int, device="cpu") -> torch.Tensor:
    """n unique uint32 keys (int32 bits), uniform over [0, 2^32) minus the sentinel."""
    return to_u32_bits(_unique_words(0, n, seed, device))


def make_negatives(n_keys: int, count: int, seed: int, device="cpu") -> torch.Tensor:
    """``count`` unique keys disjoint from ``make_keys(n_keys, seed)``."""
    return to_u32_bits(_unique_words(n_keys + 1, count, seed, device))


def make_values(n: int, seed: int, device="cpu") -> torch.Tensor:
    """n uint32 values (int32 bits); the sentinel never appears."""
    idx = torch.arange(n, dtype=torch.int64, device=device)
    v = mix32(idx, seed ^ 0x76616C)
    v = torch.where(v == SENTINEL, torch.zeros_like(v), v)
    return to_u32_bits(v)


def make_queries(keys: torch.Tensor, n_queries: int, positive_fraction: float,
                 seed: int, negatives: torch.Tensor | None = None) -> torch.Tensor:
    """Mixed query stream: round(f*N) positives drawn with replacement from
    ``keys``, the rest negatives, in a seeded random order."""
    device = keys.device
    n = keys.numel()
    n_pos = int(round(positive_fraction * n_queries))
    if n == 0:
        n_pos = 0
    n_neg = n_queries - n_pos
    parts = []
    if n_pos:
        j = torch.arange(n_pos, dtype=torch.int64, device=device)
        pick = mix32(j, seed ^ 0x706F73) % n
        parts.append(keys[pick])
    if n_neg:
        if negatives is None:
            negatives = make_negatives(n, n_neg, seed, device)
        if negatives.numel() < n_neg:
            raise ValueError("not enough negative keys")
        parts.append(negatives[:n_neg].to(device))
    if not parts:
        return torch.empty(0, dtype=torch.int32, device=device)
    q = torch.cat(parts)
    pos = torch.arange(n_queries, dtype=torch.int64, device=device)
    order = torch.argsort(((mix32(pos, seed ^ 0x7065726D) & 0x7FFFFFFF) << 32) | pos)
    return q[order].contiguous()


def make_workload(n: int, n_queries: int, positive_fraction: float, seed: int,
                  device="cpu"):
    """(keys, values, queries) for one table, all int32 tensors carrying uint32 bits."""
    keys = make_keys(n, seed, device)
    vals = make_values(n, seed, device)
    n_neg = n_queries - int(round(positive_fraction * n_queries))
    negs = make_negatives(n, n_neg, seed, device) if n_neg else None
    q = make_queries(keys, n_queries, positive_fraction, seed, negs)
    return keys, vals, q


def uniform01(index: int, seed: int) -> float:
    """Counter-based uniform draw in [0, 1) (53-bit), for per-table parameters."""
    z = _splitmix64_stream(seed ^ (index * 0x9E3779B97F4A7C15), 1)[0]
    return (z >> 11) / float(1 << 53)


def make_batch(num_tables: int, log2_min: int, log2_max: int, lf_lo: float, lf_hi: float,
               queries_per_key: float, positive_fraction: float, seed: int, device="cpu"):
    """Independent tables with key counts floor(2^(log2_min + (log2_max-log2_min) u)),
    u ~ U[0, 1), load factors ~ U[lf_lo, lf_hi], and round(queries_per_key * n)
    queries per table at the given positive fraction. Returns a dict with the
    per-table capacities and load factors, the concatenated keys, values and
    queries (int32 bits) and the (num_tables + 1) key and query offsets."""
    import numpy as np

    sizes, lfs = [], []
    for t in range(num_tables):
        u = uniform01(t, seed ^ 0x73697A65)
        sizes.append(int(2.0 ** (log2_min + (log2_max - log2_min) * u)))
        lfs.append(lf_lo + (lf_hi - lf_lo) * uniform01(t, seed ^ 0x6C66))
    keys, vals, qs = [], [], []
    for t, n in enumerate(sizes):
        k, v, q = make_workload(n, int(round(queries_per_key * n)), positive_fraction, seed + 7919 * (t + 1),
                                device)
        keys.append(k)
        vals.append(v)
        qs.append(q)
    key_offs = np.zeros(num_tables + 1, dtype=np.uint64)
    key_offs[1:] = np.cumsum(sizes)
    q_offs = np.zeros(num_tables + 1, dtype=np.uint64)
    q_offs[1:] = np.cumsum([q.numel() for q in qs])
    return {
        "capacities": np.array(sizes, dtype=np.uint64), "load_factors": np.array(lfs, dtype=np.float64),
        "keys": torch.cat(keys), "values": torch.cat(vals), "queries": torch.cat(qs),
        "key_offsets": key_offs, "query_offsets": q_offs,
    }
