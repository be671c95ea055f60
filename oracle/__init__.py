"""CPU oracle for the static bucketed hash tables (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
and reference legs may import this package. The product path (the CUDA
library and its Python binding) never imports, links or calls it.

The arithmetic lives in plain C (``ght_oracle.c``); this module compiles it
with gcc on first use and wraps it with ctypes over numpy arrays. Scheme
numbers, sizing and the hash family follow the paper's Sections III, V and
VII; see the C header for the per-function citations.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ght_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libght_oracle.so")

PRIME = 4294967291
EMPTY = 0xFFFFFFFF
EMPTY_PAIR = 0xFFFFFFFFFFFFFFFF

BCHT, P2BHT, IHT, CUCKOO1, BCHT_LB = 0, 1, 2, 3, 4
SCHEME_NAMES = {BCHT: "bcht", P2BHT: "p2bht", IHT: "iht", CUCKOO1: "cuckoo1", BCHT_LB: "bcht_lb"}


class Params(C.Structure):
    _fields_ = [
        ("scheme", C.c_int32), ("b", C.c_int32), ("h", C.c_int32), ("t", C.c_int32),
        ("m", C.c_uint64), ("a", C.c_uint32 * 4), ("c", C.c_uint32 * 4),
        ("max_chain", C.c_uint32), ("rng_seed", C.c_uint32),
        ("explicit_buckets", C.POINTER(C.c_uint32)), ("explicit_n", C.c_uint64),
    ]


class BuildStats(C.Structure):
    _fields_ = [
        ("probes", C.c_uint64), ("evictions", C.c_uint64), ("longest_chain", C.c_uint64),
        ("inserted", C.c_uint64), ("failed_at", C.c_int64),
    ]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, -O2, no vector intrinsics)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ght_oracle.h"))):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            u32p = C.POINTER(C.c_uint32)
            u64p = C.POINTER(C.c_uint64)
            L.orc_hash.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint32]
            L.orc_hash.restype = C.c_uint32
            L.orc_bucket.argtypes = [C.POINTER(Params), C.c_int, C.c_uint32]
            L.orc_bucket.restype = C.c_uint32
            L.orc_splitmix64.argtypes = [u64p]
            L.orc_splitmix64.restype = C.c_uint64
            L.orc_derive_constants.argtypes = [C.c_uint64, C.c_uint32, C.c_int, u32p, u32p]
            L.orc_num_buckets.argtypes = [C.c_uint64, C.c_double, C.c_int]
            L.orc_num_buckets.restype = C.c_uint64
            L.orc_default_params.argtypes = [C.c_int, C.c_uint64, C.c_double, C.c_uint64,
                                             C.c_uint32, C.POINTER(Params)]
            L.orc_bucket_load.argtypes = [C.POINTER(Params), u64p, C.c_uint64]
            L.orc_build.argtypes = [C.POINTER(Params), u64p, u32p, u32p, C.c_uint64,
                                    C.POINTER(BuildStats)]
            L.orc_insert.argtypes = [C.POINTER(Params), u64p, C.c_uint32, C.c_uint32, u32p,
                                     C.POINTER(BuildStats)]
            L.orc_find.argtypes = [C.POINTER(Params), u64p, u32p, u32p, C.c_uint64,
                                   C.POINTER(C.c_uint8)]
            L.orc_find.restype = C.c_uint64
            L.orc_lookup.argtypes = [u32p, u32p, C.c_uint64, u32p, u32p, C.c_uint64]
            L.orc_validate.argtypes = [C.POINTER(Params), u64p, u32p, u32p, C.c_uint64,
                                       C.c_char_p, C.c_int]
            L.orc_xorshift32.argtypes = [u32p]
            L.orc_xorshift32.restype = C.c_uint32
            _lib = L
    return _lib


def _u32(x) -> np.ndarray:
    """Accept numpy arrays or torch tensors (int32 bits) -> contiguous uint32 array."""
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    x = np.ascontiguousarray(x)
    if x.dtype in (np.int32, np.uint32):
        return x.view(np.uint32)
    return np.ascontiguousarray(x.astype(np.uint64) & 0xFFFFFFFF).astype(np.uint32)


def _p32(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_uint32))


def _p64(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


def hash_value(a: int, c: int, m: int, k: int) -> int:
    return lib().orc_hash(a, c, m, k)


def splitmix64_stream(seed: int, count: int) -> list[int]:
    st = C.c_uint64(seed)
    return [lib().orc_splitmix64(C.byref(st)) for _ in range(count)]


def derive_constants(seed: int, attempt: int, h: int):
    a = (C.c_uint32 * 4)()
    c = (C.c_uint32 * 4)()
    lib().orc_derive_constants(seed, attempt, h, a, c)
    return list(a)[:h], list(c)[:h]


def num_buckets(capacity: int, lf: float, b: int) -> int:
    return int(lib().orc_num_buckets(capacity, lf, b))


def xorshift32_stream(seed: int, count: int) -> list[int]:
    st = C.c_uint32(seed)
    return [lib().orc_xorshift32(C.byref(st)) for _ in range(count)]


class Table:
    """One oracle table: parameters plus a host slot array of m*b pairs."""

    def __init__(self, scheme: int, capacity: int, lf: float, seed: int = 0, attempt: int = 0,
                 b: int | None = None, h: int | None = None, t: int | None = None,
                 max_chain: int | None = None, explicit_buckets=None, m: int | None = None):
        self.params = Params()
        if lib().orc_default_params(scheme, capacity, lf, seed, attempt, C.byref(self.params)) != 0:
            raise ValueError("invalid table arguments")
        P = self.params
        if b is not None:
            P.b = b
        if h is not None:
            P.h = h
            a, c = derive_constants(seed, attempt, h)
            for i in range(h):
                P.a[i], P.c[i] = a[i], c[i]
        if b is not None and m is None:
            P.m = num_buckets(capacity, lf, b)
        if m is not None:
            P.m = m
        if t is not None:
            P.t = t
        if max_chain is not None:
            P.max_chain = max_chain
        self._explicit = None
        if explicit_buckets is not None:
            eb = np.ascontiguousarray(np.asarray(explicit_buckets, dtype=np.uint32).reshape(-1, P.h))
            self._explicit = eb
            P.explicit_buckets = _p32(eb)
            P.explicit_n = eb.shape[0]
        self.slots = np.full(P.m * P.b, EMPTY_PAIR, dtype=np.uint64)
        self.stats = BuildStats()

    # -- views ---------------------------------------------------------------
    @property
    def m(self) -> int:
        return int(self.params.m)

    @property
    def b(self) -> int:
        return int(self.params.b)

    @property
    def h(self) -> int:
        return int(self.params.h)

    def constants(self):
        h = self.h
        return list(self.params.a)[:h], list(self.params.c)[:h]

    def set_constants(self, a, c):
        for i in range(self.h):
            self.params.a[i], self.params.c[i] = int(a[i]), int(c[i])

    def bucket(self, i: int, k: int) -> int:
        return lib().orc_bucket(C.byref(self.params), i, k)

    def load(self, bucket: int) -> int:
        return lib().orc_bucket_load(C.byref(self.params), _p64(self.slots), bucket)

    # -- operations ----------------------------------------------------------
    def build(self, keys, values) -> int:
        k, v = _u32(keys), _u32(values)
        return lib().orc_build(C.byref(self.params), _p64(self.slots), _p32(k), _p32(v),
                               k.size, C.byref(self.stats))

    def insert(self, key: int, value: int, rng_state: int = 1) -> int:
        """Insert one pair into the current slots (no reset)."""
        st = C.c_uint32(rng_state)
        return lib().orc_insert(C.byref(self.params), _p64(self.slots), key, value, C.byref(st),
                                C.byref(self.stats))

    def find(self, queries, slots: np.ndarray | None = None):
        """(values, per-query probes, total probes) over this table's slots
        (or over ``slots``, e.g. a table exported from the GPU)."""
        q = _u32(queries)
        out = np.empty(q.size, dtype=np.uint32)
        pe = np.empty(q.size, dtype=np.uint8)
        s = self.slots if slots is None else np.ascontiguousarray(slots, dtype=np.uint64)
        total = lib().orc_find(C.byref(self.params), _p64(s), _p32(q), _p32(out), q.size,
                               pe.ctypes.data_as(C.POINTER(C.c_uint8)))
        return out, pe, int(total)

    def validate(self, keys=None, values=None, n: int | None = None, slots: np.ndarray | None = None):
        s = self.slots if slots is None else np.ascontiguousarray(slots, dtype=np.uint64)
        msg = C.create_string_buffer(512)
        if keys is not None:
            k, v = _u32(keys), _u32(values)
            ok = lib().orc_validate(C.byref(self.params), _p64(s), _p32(k), _p32(v), k.size, msg, 512)
        else:
            ok = lib().orc_validate(C.byref(self.params), _p64(s), None, None, n, msg, 512)
        return bool(ok), msg.value.decode()


def lookup(keys, values, queries) -> np.ndarray:
    """Definitional result: value of each query's pair, or the sentinel."""
    k, v, q = _u32(keys), _u32(values), _u32(queries)
    out = np.empty(q.size, dtype=np.uint32)
    if lib().orc_lookup(_p32(k), _p32(v), k.size, _p32(q), _p32(out), q.size) != 0:
        raise ValueError("invalid lookup input (sentinel key or out of memory)")
    return out
