"""GB300-native static bucketed GPU hash tables (Awad et al., "Better GPU Hash
Tables", arXiv 2108.07232), as a C-ABI CUDA library with a thin Python binding.

The binding only marshals arguments: every step of building and querying a
table runs in the sm_103a kernels of ``libght.so``. There is no CPU fallback;
if the library has not been built, loading it raises.

Low-level names mirror the C ABI (``ght_create``, ``ght_build``, ``ght_find``,
``ght_stats``, ``ght_export``, ``ght_destroy``...); :class:`HashTable` wraps
them over torch tensors (int32 tensors carry the uint32 bit patterns).
"""

from __future__ import annotations

from ._binding import (  # noqa: F401
    BCHT, BCHT_LB, BCHT_SET, CUCKOO1, EMPTY, IHT, P2BHT, SCHEMES, Batch, GhtBatchStats, GhtConfig, GhtError, GhtStats,
    HashTable, Pool,
    ght_build, ght_build_host, ght_create, ght_create_ex, ght_default_config, ght_destroy,
    ght_export, ght_find, ght_find_host, ght_find_host_noalloc, ght_hash_device, ght_hash_host, ght_last_error, ght_probe_lines,
    ght_reset_counters, ght_set_stream, ght_stats, ght_table_bytes, ght_version, lib, lib_path,
    NOALLOC_MAX_QUERIES, ght_build_scratch_bytes, ght_find_scratch_bytes, ght_set_build_scratch,
)

__all__ = [
    "BCHT", "P2BHT", "IHT", "CUCKOO1", "BCHT_LB", "BCHT_SET", "EMPTY", "SCHEMES", "HashTable", "Batch", "Pool", "GhtError",
    "GhtConfig", "GhtStats", "lib", "lib_path",
]
