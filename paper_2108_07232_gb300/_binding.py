"""ctypes binding of libght.so (argument marshalling only)."""

from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(HERE, "_build", "libght.so")

EMPTY = 0xFFFFFFFF
BCHT, P2BHT, IHT, CUCKOO1, BCHT_LB, BCHT_SET = 0, 1, 2, 3, 4, 5
SCHEMES = {"bcht": BCHT, "p2bht": P2BHT, "iht": IHT, "cuckoo1": CUCKOO1, "bcht_lb": BCHT_LB,
           "bcht_set": BCHT_SET}

STATUS = {
    0: "GHT_OK", 1: "GHT_ERR_INVALID_ARG", 2: "GHT_ERR_OOM", 3: "GHT_ERR_BUILD_FAILED",
    4: "GHT_ERR_SENTINEL_KEY", 5: "GHT_ERR_NOT_BUILT", 6: "GHT_ERR_CUDA",
    7: "GHT_ERR_DEVICE_TIMEOUT", 8: "GHT_ERR_CAPACITY", 9: "GHT_ERR_DUPLICATE_KEY",
}


class GhtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


class GhtConfig(C.Structure):
    _fields_ = [
        ("bucket_size", C.c_int32), ("num_hashes", C.c_int32), ("threshold", C.c_int32),
        ("max_chain", C.c_uint32), ("max_attempts", C.c_uint32), ("count_probes", C.c_int32),
        ("tile_lanes", C.c_int32), ("blocks_per_sm", C.c_int32), ("keys_per_lane", C.c_int32),
        ("build_tile_lanes", C.c_int32), ("build_keys_per_lane", C.c_int32),
        ("build_blocks_per_sm", C.c_int32), ("group_build", C.c_int32), ("ranked_build", C.c_int32),
        ("find_async", C.c_int32), ("check_duplicates", C.c_int32), ("max_steps", C.c_uint32),
        ("find_grouped", C.c_int32),
    ]


class GhtStats(C.Structure):
    _fields_ = [
        ("scheme", C.c_int32), ("bucket_size", C.c_int32), ("num_hashes", C.c_int32),
        ("threshold", C.c_int32), ("num_buckets", C.c_uint64), ("num_slots", C.c_uint64),
        ("capacity", C.c_uint64), ("n_stored", C.c_uint64), ("load_factor", C.c_double),
        ("attempts", C.c_uint32), ("max_chain", C.c_uint32), ("hash_a", C.c_uint32 * 4),
        ("hash_c", C.c_uint32 * 4), ("insert_probes", C.c_uint64), ("insert_retries", C.c_uint64),
        ("insert_evictions", C.c_uint64), ("longest_chain", C.c_uint64), ("find_probes", C.c_uint64), ("find_queries", C.c_uint64),
        ("table_bytes", C.c_uint64), ("built", C.c_int32), ("tile_lanes", C.c_int32),
        ("keys_per_lane", C.c_int32), ("build_tile_lanes", C.c_int32), ("build_keys_per_lane", C.c_int32),
        ("last_fill_ms", C.c_double), ("last_insert_ms", C.c_double), ("last_find_ms", C.c_double),
        ("last_group_ms", C.c_double), ("last_build_grouped", C.c_int32), ("slot_bytes", C.c_int32),
        ("last_build_ranked", C.c_int32), ("last_place_ms", C.c_double), ("place_overflow", C.c_uint64),
        ("find_staged", C.c_int32), ("last_build_split", C.c_int32),
        ("last_h2d_ms", C.c_double), ("last_h2d_bytes", C.c_uint64),
        ("find_grouped", C.c_int32), ("last_find_grouped", C.c_int32), ("last_split_ms", C.c_double),
    ]

    def as_dict(self) -> dict:
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        h = self.num_hashes
        d["hash_a"], d["hash_c"] = d["hash_a"][:h], d["hash_c"][:h]
        return d


class GhtBatchStats(C.Structure):
    _fields_ = [
        ("num_tables", C.c_uint32), ("tables_failed", C.c_uint32), ("total_keys", C.c_uint64),
        ("total_queries", C.c_uint64), ("total_slots", C.c_uint64), ("table_bytes", C.c_uint64),
        ("rebuilds", C.c_uint32), ("tuned", C.c_int32), ("tile_lanes", C.c_int32),
        ("keys_per_lane", C.c_int32), ("build_tile_lanes", C.c_int32), ("build_keys_per_lane", C.c_int32),
        ("last_run_ms", C.c_double), ("graph_launches", C.c_uint64),
        ("blocks_per_sm", C.c_int32), ("build_blocks_per_sm", C.c_int32),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class GhtPoolResult(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("kind", C.c_int32), ("table", C.c_uint32), ("launch_requests", C.c_int32),
        ("n", C.c_uint64), ("queue_s", C.c_double), ("latency_s", C.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class GhtPoolStats(C.Structure):
    _fields_ = [
        ("budget_bytes", C.c_uint64), ("used_bytes", C.c_uint64), ("tables", C.c_uint32),
        ("tables_ready", C.c_uint32), ("find_launches", C.c_uint64), ("finds_done", C.c_uint64),
        ("queries_done", C.c_uint64), ("builds_done", C.c_uint64), ("builds_refused", C.c_uint64),
        ("pending_finds", C.c_uint64), ("pending_builds", C.c_uint64), ("mean_requests_per_launch", C.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class GhtPoolRequest(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("table", C.c_uint32), ("d_in", C.c_void_p), ("d_values", C.c_void_p),
        ("d_out", C.c_void_p), ("n", C.c_uint64), ("capacity", C.c_uint64), ("load_factor", C.c_double),
        ("seed", C.c_uint64), ("arrival_s", C.c_double),
    ]


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB_PATH


def lib():
    """Load libght.so. Raises if it has not been built (no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(
                    f"{_LIB_PATH} is missing: build it with `python -m paper_2108_07232_gb300.build`")
            L = C.CDLL(_LIB_PATH)
            vp, u64, u32, i32 = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int
            sig = {
                "ght_version": ([], C.c_char_p),
                "ght_last_error": ([], C.c_char_p),
                "ght_default_config": ([i32, C.POINTER(GhtConfig)], i32),
                "ght_table_bytes": ([i32, u64, C.c_double, C.POINTER(GhtConfig)], u64),
                "ght_create": ([i32, u64, C.c_double, u64], vp),
                "ght_create_ex": ([i32, u64, C.c_double, u64, C.POINTER(GhtConfig), vp, u64], vp),
                "ght_set_stream": ([vp, vp], i32),
                "ght_build": ([vp, vp, vp, u64], i32),
                "ght_find": ([vp, vp, vp, u64], i32),
                "ght_build_host": ([vp, vp, vp, u64], i32),
                "ght_find_host": ([vp, vp, vp, u64], i32),
                "ght_find_host_noalloc": ([vp, vp, vp, u64], i32),
                "ght_stats": ([vp, C.POINTER(GhtStats)], i32),
                "ght_build_scratch_bytes": ([vp, u64], u64),
                "ght_find_scratch_bytes": ([vp, u64], u64),
                "ght_set_build_scratch": ([vp, vp, u64], i32),
                "ght_reset_counters": ([vp], i32),
                "ght_export": ([vp, vp, u64], i32),
                "ght_hash_device": ([vp, vp, vp, u64], i32),
                "ght_hash_host": ([u32, u32, u32, vp, vp, u64], i32),
                "ght_probe_lines": ([i32, vp, u64, u64, u32, vp], i32),
                "ght_partition_constants": ([u64, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)], i32),
                "ght_partition": ([vp, vp, u64, u64, u32, vp, vp, vp, vp], i32),
                "ght_unpermute": ([vp, vp, u64, vp, vp], i32),
                "ght_destroy": ([vp], None),
                "ght_batch_create": ([C.c_uint32, vp, vp, u64, C.POINTER(GhtConfig)], vp),
                "ght_batch_set_stream": ([vp, vp], i32),
                "ght_batch_set_layout": ([vp, vp, vp], i32),
                "ght_batch_build": ([vp, vp, vp], i32),
                "ght_batch_find": ([vp, vp, vp], i32),
                "ght_batch_run": ([vp, vp, vp, vp, vp], i32),
                "ght_batch_autotune": ([vp, vp, vp, vp, vp], i32),
                "ght_batch_stats": ([vp, C.POINTER(GhtBatchStats)], i32),
                "ght_batch_table_stats": ([vp, C.c_uint32, C.POINTER(GhtStats)], i32),
                "ght_batch_export": ([vp, C.c_uint32, vp, u64], i32),
                "ght_batch_destroy": ([vp], None),
                "ght_pool_create": ([u64, C.POINTER(GhtConfig)], vp),
                "ght_pool_submit_build": ([vp, u64, C.c_double, u64, vp, vp, u64, C.POINTER(C.c_uint32)], u64),
                "ght_pool_submit_find": ([vp, C.c_uint32, vp, vp, u64], u64),
                "ght_pool_wait": ([vp, u64, C.c_double, C.POINTER(GhtPoolResult)], i32),
                "ght_pool_drop_table": ([vp, C.c_uint32], i32),
                "ght_pool_stats": ([vp, C.POINTER(GhtPoolStats)], i32),
                "ght_pool_replay": ([vp, vp, u64, i32, vp, vp, C.POINTER(C.c_double)], i32),
                "ght_pool_destroy": ([vp], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(rc: int) -> None:
    if rc != 0:
        raise GhtError(rc, lib().ght_last_error().decode())


def _ptr(x) -> int | None:
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    return int(x)


def _config(cfg) -> GhtConfig | None:
    if cfg is None or isinstance(cfg, GhtConfig):
        return cfg
    c = GhtConfig()
    names = {f for f, _ in GhtConfig._fields_}
    for k, v in dict(cfg).items():
        if k not in names:
            raise TypeError(f"unknown table option {k!r}")
        if v is not None:
            setattr(c, k, int(v))
    return c


# --- names of the C ABI -------------------------------------------------------

def ght_version() -> str:
    return lib().ght_version().decode()


def ght_last_error() -> str:
    return lib().ght_last_error().decode()


def ght_default_config(scheme: int) -> GhtConfig:
    c = GhtConfig()
    _check(lib().ght_default_config(scheme, C.byref(c)))
    return c


def ght_table_bytes(scheme: int, capacity: int, load_factor: float, cfg=None) -> int:
    c = _config(cfg)
    return int(lib().ght_table_bytes(scheme, capacity, load_factor, C.byref(c) if c else None))


def ght_create(scheme: int, capacity: int, load_factor: float, seed: int) -> int:
    t = lib().ght_create(scheme, capacity, load_factor, seed)
    if not t:
        raise GhtError(1, ght_last_error())
    return t


def ght_create_ex(scheme: int, capacity: int, load_factor: float, seed: int, cfg=None,
                  d_storage=None, storage_bytes: int = 0) -> int:
    c = _config(cfg)
    t = lib().ght_create_ex(scheme, capacity, load_factor, seed, C.byref(c) if c else None,
                            _ptr(d_storage), storage_bytes)
    if not t:
        raise GhtError(1, ght_last_error())
    return t


def ght_set_stream(t: int, stream) -> None:
    _check(lib().ght_set_stream(t, stream))


def ght_build(t: int, d_keys, d_values, n: int) -> None:
    _check(lib().ght_build(t, _ptr(d_keys), _ptr(d_values), n))


def ght_find(t: int, d_queries, d_out, n: int) -> None:
    _check(lib().ght_find(t, _ptr(d_queries), _ptr(d_out), n))


def ght_build_host(t: int, h_keys, h_values, n: int) -> None:
    _check(lib().ght_build_host(t, _ptr(h_keys), _ptr(h_values), n))


def ght_find_host(t: int, h_queries, h_out, n: int) -> None:
    _check(lib().ght_find_host(t, _ptr(h_queries), _ptr(h_out), n))


def ght_find_host_noalloc(t: int, h_queries, h_out, n: int) -> None:
    _check(lib().ght_find_host_noalloc(t, _ptr(h_queries), _ptr(h_out), n))


NOALLOC_MAX_QUERIES = 1 << 22


def ght_build_scratch_bytes(t: int, n: int) -> int:
    return int(lib().ght_build_scratch_bytes(t, n))


def ght_find_scratch_bytes(t: int, n: int) -> int:
    return int(lib().ght_find_scratch_bytes(t, n))


def ght_set_build_scratch(t: int, d_scratch, nbytes: int) -> None:
    _check(lib().ght_set_build_scratch(t, _ptr(d_scratch), nbytes))


def ght_stats(t: int) -> GhtStats:
    s = GhtStats()
    _check(lib().ght_stats(t, C.byref(s)))
    return s


def ght_reset_counters(t: int) -> None:
    _check(lib().ght_reset_counters(t))


def ght_export(t: int, h_slots, n_slots: int) -> None:
    _check(lib().ght_export(t, _ptr(h_slots), n_slots))


def ght_hash_device(t: int, d_keys, d_buckets, n: int) -> None:
    _check(lib().ght_hash_device(t, _ptr(d_keys), _ptr(d_buckets), n))


def ght_hash_host(a: int, c: int, m: int, h_keys, h_out, n: int) -> None:
    _check(lib().ght_hash_host(a, c, m, _ptr(h_keys), _ptr(h_out), n))


def ght_probe_lines(mode: int, d_lines, num_lines: int, ops: int, seed: int = 1, stream: int = 0) -> None:
    """Memory-system ceiling probe on random 128-byte lines (asynchronous on `stream`)."""
    _check(lib().ght_probe_lines(mode, _ptr(d_lines), num_lines, ops, seed, stream))


def ght_partition_constants(seed: int) -> tuple[int, int]:
    a, c = C.c_uint32(0), C.c_uint32(0)
    _check(lib().ght_partition_constants(seed, C.byref(a), C.byref(c)))
    return a.value, c.value


def ght_partition(d_keys, d_values, n: int, seed: int, shards: int, d_out_keys, d_out_values, h_counts,
                  stream: int = 0) -> None:
    _check(lib().ght_partition(_ptr(d_keys), _ptr(d_values), n, seed, shards, _ptr(d_out_keys),
                               _ptr(d_out_values), _ptr(h_counts), stream))


def ght_unpermute(d_src, d_pos, n: int, d_dst, stream: int = 0) -> None:
    _check(lib().ght_unpermute(_ptr(d_src), _ptr(d_pos), n, _ptr(d_dst), stream))


def ght_destroy(t: int) -> None:
    lib().ght_destroy(t)


# --- tensor-level wrapper -----------------------------------------------------

class HashTable:
    """One static table whose storage is a torch tensor on the current CUDA
    device. Work follows torch's current stream at each call."""

    def __init__(self, scheme, capacity: int, load_factor: float, seed: int = 0, device=None,
                 **config):
        import torch

        self.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        self.capacity = int(capacity)
        self.load_factor = float(load_factor)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._cfg = _config(config) if config else None
        nbytes = ght_table_bytes(self.scheme, self.capacity, self.load_factor, self._cfg)
        if nbytes == 0:
            raise GhtError(1, ght_last_error())
        # torch's allocator hands out blocks aligned far beyond 256 bytes; the
        # extra 256 bytes cover any allocator that does not
        self._storage = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self._storage.data_ptr()
        aligned = (base + 255) & ~255
        with torch.cuda.device(self.device):
            self._t = ght_create_ex(self.scheme, self.capacity, self.load_factor, seed, self._cfg,
                                    aligned, nbytes)
        self.nbytes = nbytes
        self._offset = aligned - base

    def slots_view(self):
        """The table's slot array as a device int64 tensor (no copy)."""
        n = ght_stats(self._t).num_slots
        lo = self._offset + 256
        return self._storage[lo:lo + n * 8].view(__import__("torch").int64)

    # the table handle is freed with the object
    def close(self) -> None:
        if getattr(self, "_t", None):
            ght_destroy(self._t)
            self._t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        import torch
        ght_set_stream(self._t, torch.cuda.current_stream(self.device).cuda_stream)

    @staticmethod
    def _u32(x):
        import torch
        if x.dtype not in (torch.int32, torch.uint32):
            raise TypeError("keys, values and queries must be int32 (uint32 bits) tensors")
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x

    def build(self, keys, values=None) -> None:
        """Build from keys and values (values may be None for a keys-only set)."""
        k = self._u32(keys)
        if values is None:
            if self.scheme != BCHT_SET:
                raise ValueError("values are required except for a keys-only set")
            v = None
        else:
            v = self._u32(values)
            if k.numel() != v.numel():
                raise ValueError("keys and values differ in length")
        with _device_of(self.device):
            self._stream()
            self._ensure_scratch(k.numel())
            if k.is_cuda:
                ght_build(self._t, k, v, k.numel())
            else:
                ght_build_host(self._t, k, v, k.numel())

    def _ensure_scratch(self, n: int) -> None:
        """Two-phase and grouped builds need scratch; it is a torch tensor kept with the table."""
        self._ensure_bytes(ght_build_scratch_bytes(self._t, n))

    def _ensure_find_scratch(self, n: int) -> None:
        """A grouped find (find_grouped = 1) needs scratch too: the same buffer, grown."""
        self._ensure_bytes(ght_find_scratch_bytes(self._t, n))

    def _ensure_bytes(self, need: int) -> None:
        import torch
        have = getattr(self, "_scratch_bytes", 0)
        if need and need > have:
            self._scratch = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
            base = self._scratch.data_ptr()
            ght_set_build_scratch(self._t, (base + 255) & ~255, need)
            self._scratch_bytes = need

    def release_scratch(self) -> None:
        """Drop the build scratch (later builds insert every key with the cuckoo insert until re-set)."""
        if getattr(self, "_scratch_bytes", 0):
            ght_set_build_scratch(self._t, None, 0)
            self._scratch = None
            self._scratch_bytes = 0

    def find(self, queries, out=None):
        import torch
        q = self._u32(queries)
        if out is None:
            out = torch.empty_like(q)
        with _device_of(self.device):
            self._stream()
            if q.is_cuda:
                self._ensure_find_scratch(q.numel())
                ght_find(self._t, q, out, q.numel())
            else:
                ght_find_host(self._t, q, out, q.numel())
        return out

    def stats(self) -> dict:
        with _device_of(self.device):
            self._stream()
            return ght_stats(self._t).as_dict()

    def reset_counters(self) -> None:
        self._stream()
        ght_reset_counters(self._t)

    def export(self):
        """Raw slots, bucket-major, as a numpy array: uint64 pairs, or uint32
        keys for a keys-only set."""
        import numpy as np
        s = ght_stats(self._t)
        out = np.empty(s.num_slots * s.slot_bytes // 8, dtype=np.uint64)
        with _device_of(self.device):
            self._stream()
            ght_export(self._t, out, out.size)
        return out.view(np.uint32) if s.slot_bytes == 4 else out

    def hash_device(self, keys):
        """(n, h) int64 tensor of bucket indices computed on the device."""
        import torch
        k = self._u32(keys)
        h = ght_stats(self._t).num_hashes
        out = torch.empty(k.numel() * h, dtype=torch.int32, device=k.device)
        with _device_of(self.device):
            self._stream()
            ght_hash_device(self._t, k, out, k.numel())
        return (out.to(torch.int64) & 0xFFFFFFFF).view(-1, h)


def _device_of(dev):
    import torch
    return torch.cuda.device(dev)


# --- batched tables -------------------------------------------------------------

class Batch:
    """Many independent BCHT tables (b = 16, h = 3) built and queried by shared
    launches. Inputs are concatenated int32 (uint32 bits) tensors with per-table
    offsets set once by :meth:`set_layout`."""

    def __init__(self, capacities, load_factors, seed: int = 0, device=None, **config):
        import numpy as np
        import torch

        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        caps = np.ascontiguousarray(capacities, dtype=np.uint64)
        lfs = np.ascontiguousarray(load_factors, dtype=np.float64)
        if caps.size != lfs.size or caps.size == 0:
            raise ValueError("capacities and load_factors must have the same non-zero length")
        self.num_tables = int(caps.size)
        cfg = _config(config) if config else None
        with torch.cuda.device(self.device):
            b = lib().ght_batch_create(self.num_tables, caps.ctypes.data, lfs.ctypes.data, seed,
                                       C.byref(cfg) if cfg else None)
        if not b:
            raise GhtError(1, ght_last_error())
        self._b = b
        self.key_offsets = None
        self.query_offsets = None

    def close(self) -> None:
        if getattr(self, "_b", None):
            lib().ght_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        import torch
        _check(lib().ght_batch_set_stream(self._b, torch.cuda.current_stream(self.device).cuda_stream))

    def set_layout(self, key_offsets, query_offsets) -> None:
        import numpy as np
        ko = np.ascontiguousarray(key_offsets, dtype=np.uint64)
        qo = np.ascontiguousarray(query_offsets, dtype=np.uint64)
        if ko.size != self.num_tables + 1 or qo.size != self.num_tables + 1:
            raise ValueError("offsets need num_tables + 1 entries")
        _check(lib().ght_batch_set_layout(self._b, ko.ctypes.data, qo.ctypes.data))
        self.key_offsets, self.query_offsets = ko, qo

    def build(self, keys, values) -> None:
        import torch
        with torch.cuda.device(self.device):
            self._stream()
            _check(lib().ght_batch_build(self._b, _ptr(keys), _ptr(values)))

    def find(self, queries, out=None):
        import torch
        if out is None:
            out = torch.empty_like(queries)
        with torch.cuda.device(self.device):
            self._stream()
            _check(lib().ght_batch_find(self._b, _ptr(queries), _ptr(out)))
        return out

    def run(self, keys, values, queries, out=None):
        """Build and find in one CUDA-graph launch."""
        import torch
        if out is None:
            out = torch.empty_like(queries)
        with torch.cuda.device(self.device):
            self._stream()
            _check(lib().ght_batch_run(self._b, _ptr(keys), _ptr(values), _ptr(queries), _ptr(out)))
        return out

    def autotune(self, keys, values, queries, out=None) -> dict:
        import torch
        if out is None:
            out = torch.empty_like(queries)
        with torch.cuda.device(self.device):
            self._stream()
            _check(lib().ght_batch_autotune(self._b, _ptr(keys), _ptr(values), _ptr(queries), _ptr(out)))
        return self.stats()

    def stats(self) -> dict:
        s = GhtBatchStats()
        _check(lib().ght_batch_stats(self._b, C.byref(s)))
        return s.as_dict()

    def table_stats(self, t: int) -> dict:
        s = GhtStats()
        _check(lib().ght_batch_table_stats(self._b, t, C.byref(s)))
        return s.as_dict()

    def export(self, t: int):
        import numpy as np
        n = self.table_stats(t)["num_slots"]
        out = np.empty(n, dtype=np.uint64)
        _check(lib().ght_batch_export(self._b, t, out.ctypes.data, n))
        return out


# --- served pool -----------------------------------------------------------------

class Pool:
    """Device-resident BCHT tables under an HBM budget, serving find and build
    requests with continuous batching (see include/ght.h). Tensors passed to
    submit calls are kept alive until their request is waited on."""

    def __init__(self, budget_bytes: int, device=None, **config):
        import torch

        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        cfg = _config(config) if config else None
        with torch.cuda.device(self.device):
            p = lib().ght_pool_create(int(budget_bytes), C.byref(cfg) if cfg else None)
        if not p:
            raise GhtError(1, ght_last_error())
        self._p = p
        self._keep = {}

    def close(self) -> None:
        if getattr(self, "_p", None):
            lib().ght_pool_destroy(self._p)
            self._p = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit_build(self, capacity: int, load_factor: float, seed: int, keys, values):
        tid = C.c_uint32(0)
        tk = lib().ght_pool_submit_build(self._p, int(capacity), float(load_factor), int(seed), _ptr(keys),
                                         _ptr(values), keys.numel(), C.byref(tid))
        if not tk:
            raise GhtError(1, ght_last_error())
        self._keep[tk] = (keys, values)
        return tk, tid.value

    def submit_find(self, table: int, queries, out):
        tk = lib().ght_pool_submit_find(self._p, int(table), _ptr(queries), _ptr(out), queries.numel())
        if not tk:
            raise GhtError(1, ght_last_error())
        self._keep[tk] = (queries, out)
        return tk

    def wait(self, ticket: int, timeout: float = 60.0) -> dict:
        r = GhtPoolResult()
        rc = lib().ght_pool_wait(self._p, int(ticket), float(timeout), C.byref(r))
        self._keep.pop(ticket, None)
        if rc != 0:
            raise GhtError(rc, ght_last_error())
        return r.as_dict()

    def drop(self, table: int) -> None:
        _check(lib().ght_pool_drop_table(self._p, int(table)))

    def stats(self) -> dict:
        s = GhtPoolStats()
        rc = lib().ght_pool_stats(self._p, C.byref(s))
        if rc != 0:
            raise GhtError(rc, ght_last_error())
        return s.as_dict()

    def replay(self, trace, serial: bool = False):
        """trace: list of dicts with kind ('find'|'build'), table, queries/keys,
        values, out, capacity, load_factor, seed, arrival_s. Returns
        (latencies [s] as numpy, statuses, makespan [s])."""
        import numpy as np
        n = len(trace)
        arr = (GhtPoolRequest * max(n, 1))()
        for i, t in enumerate(trace):
            r = arr[i]
            build = t["kind"] == "build"
            r.kind = 1 if build else 0
            r.table = int(t.get("table", 0))
            r.d_in = _ptr(t["keys"] if build else t["queries"])
            r.d_values = _ptr(t["values"]) if build else None
            r.d_out = None if build else _ptr(t["out"])
            r.n = (t["keys"] if build else t["queries"]).numel()
            r.capacity = int(t.get("capacity", 0))
            r.load_factor = float(t.get("load_factor", 0.0))
            r.seed = int(t.get("seed", 0))
            r.arrival_s = float(t["arrival_s"])
        lat = np.zeros(n, dtype=np.float64)
        st = np.zeros(n, dtype=np.int32)
        mk = C.c_double(0.0)
        rc = lib().ght_pool_replay(self._p, C.addressof(arr), n, 1 if serial else 0, lat.ctypes.data, st.ctypes.data,
                                   C.byref(mk))
        if rc != 0:
            raise GhtError(rc, ght_last_error())
        return lat, st, mk.value
