/*
 * ght.h -- C ABI of the GB300 (sm_103a) static bucketed GPU hash tables.
 *
 * The method is that of Awad, Ashkiani, Porumbescu, Farach-Colton and Owens,
 * "Better GPU Hash Tables" (arXiv 2108.07232): a static table built once on one
 * GPU from an unordered array of 32-bit key/value pairs, then queried in bulk
 * (Section I). Schemes:
 *   GHT_BCHT     bucketed cuckoo, b = 16, three hash functions (Sec. III-A, V-B)
 *   GHT_P2BHT    bucketed power of two choices, b = 16 (Sec. III-B, V-C)
 *   GHT_IHT      iceberg, b = 16, primary + two secondaries, t = 13 (Sec. III-C, V-D)
 *   GHT_CUCKOO1  bucket size one cuckoo ("1CHT"), three hash functions (Sec. VII)
 *   GHT_BCHT_LB  load-balanced bucketed cuckoo (Sec. III-A, last paragraph)
 *   GHT_BCHT_SET keys-only bucketed cuckoo, a membership set: 32 four-byte keys
 *                per 128-byte bucket, three hash functions (the tables "storing
 *                keys" of Sec. I and Sec. III-A); values are not stored, a find
 *                writes 1 for a present key and 0 for an absent one
 *
 * Conventions used by every entry point:
 *   - Keys and values are uint32. 0xFFFFFFFF (GHT_EMPTY) is the empty key and
 *     the empty value (Sec. V): it may not be inserted as a key; a find that
 *     misses, or that queries GHT_EMPTY, returns GHT_EMPTY. A stored value equal
 *     to GHT_EMPTY cannot be told apart from a miss.
 *   - Keys passed to one build must be unique (the paper's inputs are unique,
 *     Sec. VII); duplicates are a precondition violation, detected only when
 *     the config's check_duplicates is set.
 *   - Pointers named d_* are device memory owned by the caller (for example
 *     torch tensors, int32 reinterpreted as uint32); the library never frees
 *     them. Pointers named h_* are host memory owned by the caller.
 *   - Work is issued on the table's stream (ght_set_stream; default: the legacy
 *     default stream). ght_find is asynchronous; ght_build synchronises the
 *     stream once per attempt to read the build status.
 *   - Functions return a ght_status; on error ght_last_error() gives a
 *     thread-local message. No C++ exception crosses this ABI.
 *   - Every host wait for the device polls an event with a deadline: the
 *     environment variable GHT_WAIT_TIMEOUT_S in seconds (default 300); when
 *     it runs out the call returns GHT_ERR_DEVICE_TIMEOUT.
 *   - The hash family is h_i(k) = ((a_i k + c_i) mod p) mod m, p = 4294967291
 *     (Sec. VII setup; the paper writes b for c_i). a_i, c_i come from SplitMix64
 *     seeded with seed XOR (attempt * 0x9E3779B97F4A7C15), drawn a_0, c_0, a_1, ...
 *     with a_i = 1 + x mod (p-1) and c_i = x mod p.
 *   - Sizing (Sec. III): m = ceil(capacity / (load_factor * b)) buckets of b
 *     64-bit slots, slot = (value << 32) | key, empty slot = all ones.
 */
#ifndef GHT_H
#define GHT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GHT_EMPTY 0xFFFFFFFFu
#define GHT_ABI_VERSION 1

typedef enum {
  GHT_BCHT = 0,
  GHT_P2BHT = 1,
  GHT_IHT = 2,
  GHT_CUCKOO1 = 3,
  GHT_BCHT_LB = 4,
  GHT_BCHT_SET = 5
} ght_scheme;

typedef enum {
  GHT_OK = 0,
  GHT_ERR_INVALID_ARG = 1,     /* bad scheme, size, load factor or pointer */
  GHT_ERR_OOM = 2,             /* device allocation failed */
  GHT_ERR_BUILD_FAILED = 3,    /* every attempt hit the chain bound or full buckets */
  GHT_ERR_SENTINEL_KEY = 4,    /* an input key was 0xFFFFFFFF */
  GHT_ERR_NOT_BUILT = 5,       /* find on a table without a successful build */
  GHT_ERR_CUDA = 6,            /* a CUDA runtime call failed */
  GHT_ERR_DEVICE_TIMEOUT = 7,  /* a bounded device or host wait ran out */
  GHT_ERR_CAPACITY = 8,        /* n larger than the table's capacity */
  GHT_ERR_DUPLICATE_KEY = 9    /* check_duplicates found a key stored more than once */
} ght_status;

typedef struct ght_table ght_table; /* opaque, library-owned */

/* Optional knobs; zero means "scheme default". */
typedef struct {
  int32_t bucket_size;   /* slots per bucket: 16 or 32 for bucketed schemes, 1 for CUCKOO1 */
  int32_t num_hashes;    /* BCHT/BCHT_LB: 2..4; CUCKOO1: 2..4; P2BHT: 2; IHT: 3 */
  int32_t threshold;     /* IHT t: the primary takes a key while it would hold
                            fewer than t keys afterwards (default ceil(0.8 b)) */
  uint32_t max_chain;    /* cuckoo exchanges per insert before failing (default 1000) */
  uint32_t max_attempts; /* builds with fresh constants before GHT_ERR_BUILD_FAILED (default 50, Sec. VII) */
  int32_t count_probes;  /* 1: kernels accumulate probe counters (slower; off for timing) */
  /* Launch shapes (0 = tuned default). Find: lanes that read one bucket
   * together (4, 8 or 16; 8 or 16 for 32-pair buckets; 8 for schemes other
   * than BCHT; 4 for the staged find, see find_async), queries each lane
   * keeps in flight (1 or 2; 2..8 for the staged find), blocks per SM.
   * Build: the same three for the insert kernel. */
  int32_t tile_lanes;
  int32_t blocks_per_sm;
  int32_t keys_per_lane;
  int32_t build_tile_lanes;
  int32_t build_keys_per_lane;
  int32_t build_blocks_per_sm;
  /* Grouped build: the pairs are first regrouped by first-choice bucket
   * range (H_0(k) >> s), so the build's concurrent stores and atomics stay in
   * a few MB of the table at a time. 1 = on, -1 = off, 0 = default: on for
   * BCHT and BCHT_SET tables of at least 4x the device's L2 size. Needs
   * scratch (ght_build_scratch_bytes) and 16-byte aligned key and value
   * arrays, else the build runs in input order. */
  int32_t group_build;
  /* Two-phase build of BCHT and BCHT_SET: every key that arrives at its
   * first-choice bucket while it has room is stored at its arrival rank
   * without reading the bucket, the rest are inserted by the cuckoo insert
   * (the same BCHT, Sec. III-A, with those keys inserted first). 1 = on,
   * -1 = off, 0 = default: on when the build is grouped. Needs scratch
   * (ght_build_scratch_bytes), else the build runs the cuckoo insert for
   * every key. */
  int32_t ranked_build;
  /* Finds of 128-byte buckets (16 pairs: BCHT with 4-lane tiles, P2BHT, IHT
   * and the load-balanced BCHT, whose find tiles then have 4 lanes; the
   * keys-only set, likewise): 1 = stage the bucket parts in shared memory
   * with asynchronous copies, keys_per_lane (2..8, default 6, of which two
   * stay in registers) query sets in flight per lane, each scheme's own
   * probe order and stop rule; -1 = off
   * (bucket parts in registers, keys_per_lane 1..2); 0 = default: on where
   * it applies, the table's slots take at least the device's L2 size and
   * neither keys_per_lane 1 nor (except for BCHT's 4) tile_lanes is given.
   * Other shapes (32-pair buckets, CUCKOO1) reject 1. */
  int32_t find_async;
  /* 1: after a successful ght_build / ght_build_host, check that no input key
   * is stored more than once (every candidate bucket of every input key is
   * read: a debug aid, off by default). A duplicate fails the call with
   * GHT_ERR_DUPLICATE_KEY and leaves the table unbuilt. */
  int32_t check_duplicates;
  /* Per-key step bound of the bucketed insert kernels: a key that has made
   * this many bucket visits (reads, CAS retries and exchanges together) stops,
   * sets the table's timeout status and the build returns
   * GHT_ERR_DEVICE_TIMEOUT with the table unbuilt (no retry with new
   * constants). 0 = derived: (max_chain + 2) * h * (b + 2) + 64, which a
   * correct insert never reaches (every visit stores the key, exchanges, or
   * loses a CAS to a slot that stays filled). A smaller value only serves to
   * test that the device loop ends and the error reaches the caller. */
  uint32_t max_steps;
  /* Grouped find of device queries (16-pair buckets: BCHT, P2BHT, IHT, the
   * load-balanced BCHT): the same probes with the same stop rule as every
   * other find (Sec. V), made round by round -- round r reads bucket H_r of
   * every query still open, the queries grouped by 64 KB range of the table
   * so each range is read once per round from shared memory -- and the
   * answers returned to query order by position. 1 = on; 0 or -1 = off
   * (the default: on GB300 the grouped find is faster for batches of mostly
   * missing keys -- 2^28 misses against a 2^28-key BCHT at LF 0.99: 16.6 ms
   * against 19.9 ms -- and slower for mostly present ones, 10.4 against 9.8
   * ms). Needs scratch (the library pool for tables on library storage, else
   * ght_set_build_scratch's buffer when large enough; ght_find_scratch_bytes),
   * 16-byte aligned queries, tables of up to 2^25 buckets and batches of at
   * least ~5500 queries per group of 2^shift buckets (shift = bits of the
   * bucket count - 9); where these do not hold, the find runs per query.
   * Other shapes (32-pair buckets, CUCKOO1, the set) reject 1. */
  int32_t find_grouped;
} ght_config;

typedef struct {
  int32_t scheme, bucket_size, num_hashes, threshold;
  uint64_t num_buckets, num_slots, capacity, n_stored;
  double load_factor;          /* n_stored / num_slots of the last successful build */
  uint32_t attempts;           /* attempts used by the last build */
  uint32_t max_chain;
  uint32_t hash_a[4], hash_c[4];
  uint64_t insert_probes;      /* bucket reads by inserts, CAS retries excluded (needs count_probes) */
  uint64_t insert_retries;     /* bucket re-reads after a failed CAS */
  uint64_t insert_evictions;   /* cuckoo exchanges */
  uint64_t longest_chain;      /* most exchanges one insert made (needs count_probes) */
  uint64_t find_probes;        /* bucket reads by finds since the last reset */
  uint64_t find_queries;       /* queries answered since the last reset */
  uint64_t table_bytes;        /* device bytes of the table (control block + slots) */
  int32_t built;
  int32_t tile_lanes, keys_per_lane, build_tile_lanes, build_keys_per_lane;
  /* device time of the last build's fill, grouping (-1 if not grouped) and
   * cuckoo insert (in a two-phase build: of the placement's overflow), and of
   * the last find, from events on the table's stream (-1 if not yet
   * complete) */
  double last_fill_ms, last_insert_ms, last_find_ms, last_group_ms;
  int32_t last_build_grouped;
  int32_t slot_bytes;          /* 8 for key/value pairs, 4 for GHT_BCHT_SET */
  int32_t last_build_ranked;   /* 1 if the last build was two-phase (ranked placement first) */
  double last_place_ms;        /* device time of its ranked placement (-1 if not two-phase) */
  uint64_t place_overflow;     /* keys the ranked placement left to the cuckoo insert */
  int32_t find_staged;         /* 1 if finds stage bucket parts in shared memory (find_async) */
  int32_t last_build_split;    /* 1 if the last build split its groups into 64 KB sub-groups and placed
                                  each whole in shared memory (block placement, no table fill) */
  /* host-to-device copies of the last ght_build_host / ght_find_host call:
   * device time from its first copy's start to its last copy's end (-1 if
   * none, as for a build read in place, or not complete) and the bytes copied */
  double last_h2d_ms;
  uint64_t last_h2d_bytes;
  int32_t find_grouped;        /* the table's grouped-find setting (1 on, else off) */
  int32_t last_find_grouped;   /* 1 if the last ght_find ran grouped */
  /* device time of the last build's second grouping level (the split into
   * 64 KB sub-groups of a block placement; -1 if none); last_group_ms is
   * then the first level alone */
  double last_split_ms;
} ght_stats_t;

/* Library version string; never NULL. */
const char *ght_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char *ght_last_error(void);

/* Fill *out with the defaults of `scheme`. */
int ght_default_config(int scheme, ght_config *out);

/* Device bytes a table of this shape needs (control block + slots), or 0 if
 * the arguments are invalid. Lets callers supply their own storage. */
uint64_t ght_table_bytes(int scheme, uint64_t capacity, double load_factor, const ght_config *cfg);

/* Create an empty table sized for `capacity` keys at `load_factor` in (0, 1]
 * (Sec. III sizing), with hash constants derived from `seed`. Storage is
 * allocated on the current device. Returns NULL on error (see ght_last_error). */
ght_table *ght_create(int scheme, uint64_t capacity, double load_factor, uint64_t seed);

/* As ght_create, with optional knobs (cfg may be NULL) and optional caller
 * storage: if d_storage is non-NULL it must be device memory of at least
 * ght_table_bytes(...) bytes, 256-byte aligned, owned by the caller and kept
 * alive until ght_destroy; the library then allocates no device memory. */
ght_table *ght_create_ex(int scheme, uint64_t capacity, double load_factor, uint64_t seed,
                         const ght_config *cfg, void *d_storage, uint64_t storage_bytes);

/* Issue all later work on `cuda_stream` (a cudaStream_t; NULL = legacy default). */
int ght_set_stream(ght_table *t, void *cuda_stream);

/* Bulk build (Sec. III insertion of every key, Sec. V-B..D kernels); for
 * GHT_BCHT_SET d_values is ignored and may be NULL. Fill the
 * table with empty pairs, insert the n pairs (d_keys[i], d_values[i]), read
 * the device status; on failure retry with the next attempt's constants, up
 * to max_attempts. n <= capacity (else GHT_ERR_CAPACITY). n = 0 builds an
 * empty table. A second build replaces the contents. */
int ght_build(ght_table *t, const uint32_t *d_keys, const uint32_t *d_values, uint64_t n);

/* Bulk find (Sec. V-B find and its P2BHT/IHT variants): d_out[i] = value of
 * d_queries[i], or GHT_EMPTY. Asynchronous on the table's stream; d_out may
 * not alias d_queries. n = 0 is a no-op. GHT_ERR_NOT_BUILT before a
 * successful build. */
int ght_find(const ght_table *t, const uint32_t *d_queries, uint32_t *d_out, uint64_t n);

/* As ght_build / ght_find with HOST arrays: the library stages them in
 * device memory from its own stream-ordered pool (find pipelines chunked
 * host<->device copies with the kernel) and returns when the table is built
 * or the results are in h_out. Pinned host memory copies fastest. A build
 * from page-locked keys and values (allocated or registered with the CUDA
 * runtime) that requests neither grouping nor the two-phase build
 * (group_build and ranked_build <= 0, the host-buffer defaults) copies
 * nothing: its input-order insert reads them in place (last_h2d_ms -1); they
 * must stay unchanged until the call returns. If the bounded wait for the
 * device runs out (GHT_ERR_DEVICE_TIMEOUT, see GHT_WAIT_TIMEOUT_S), copies
 * or kernels already queued may still read h_keys/h_values or write h_out
 * afterwards. */
int ght_build_host(ght_table *t, const uint32_t *h_keys, const uint32_t *h_values, uint64_t n);
int ght_find_host(const ght_table *t, const uint32_t *h_queries, uint32_t *h_out, uint64_t n);

/* Host-buffer find that allocates nothing. This paper has no counterpart to
 * it: it exists for callers that must not call the CUDA allocator once they
 * run -- for example an inference-server plugin whose execute step may not
 * allocate, or code that runs while another memory pool owns the device
 * memory -- and that would otherwise need ght_find_host, whose device
 * staging buffers are allocated per call.
 *
 * The queries are copied into a staging array that is part of the library
 * image (a static device array of 2 x GHT_NOALLOC_MAX_QUERIES uint32, 32 MiB),
 * found there by the ordinary per-query find kernel (also on a table set for
 * the grouped find, whose scratch would need an allocator), and the results
 * are copied back into h_out before the call returns. n must not exceed
 * GHT_NOALLOC_MAX_QUERIES (else GHT_ERR_CAPACITY, nothing is done); n = 0 is
 * a no-op. The table must have been built, and the device current at its
 * creation must be current (else GHT_ERR_INVALID_ARG, nothing is done).
 *
 * The array is reserved on a device when the first table is created there:
 * ght_create / ght_create_ex look up its device address once per device
 * (cudaGetSymbolAddress, which has the driver load it), so this call itself
 * neither allocates nor loads anything. The array then stays reserved on that
 * device until the process exits. Every call on a device shares it, and its
 * contents are whatever the last call left there: calls that overlap on the
 * GPU (from several host threads or streams at once) race on it and must be
 * serialised by the caller. If the wait for the device runs out
 * (GHT_ERR_DEVICE_TIMEOUT), the copies may still be running and may still
 * write h_out; later calls on that device return GHT_ERR_DEVICE_TIMEOUT until
 * they have finished. */
#define GHT_NOALLOC_MAX_QUERIES (1u << 22)
int ght_find_host_noalloc(const ght_table *t, const uint32_t *h_queries, uint32_t *h_out, uint64_t n);

/* ---------------------------------------------------------------------------
 * Sharding one table over G GPUs (one rank each). The paper's tables live on
 * one GPU; they shard by key: a partition hash g(k) = ((a_g k + c_g) mod p)
 * mod G (the same family as the tables' hash functions, p = 4294967291, with
 * constants of its own, so g is independent of every h_i) sends each key to
 * one shard, and each shard is an ordinary table of the keys it received. A
 * build partitions each rank's pairs by g, exchanges them (one all-to-all),
 * and builds the shard; a find partitions the queries by g remembering their
 * positions, exchanges them, finds them in the shard, exchanges the answers
 * back and returns them to query order (ght_unpermute). The exchanges are
 * the caller's collectives (torch.distributed in the Python binding).
 * ------------------------------------------------------------------------- */
#define GHT_PARTITION_SEED_SALT 0x5348415244ull /* a_g, c_g derive from seed XOR this */

/* a_g and c_g of the partition hash for `seed`: the tables' derivation
 * (SplitMix64, a = 1 + x mod (p-1), c = y mod p) from seed XOR
 * GHT_PARTITION_SEED_SALT, attempt 0. Host only. */
int ght_partition_constants(uint64_t seed, uint32_t *a, uint32_t *c);

/* Reorder n keys by shard g(k) (shards in [1, 4096]) into d_out_keys, shard
 * 0's keys first, with d_values carried alongside into d_out_values; if
 * d_values is NULL, d_out_values receives each key's input position (for
 * ght_unpermute). h_counts[s] receives the number of keys of shard s. The
 * key 0xFFFFFFFF goes to shard 0. Order within a shard is unspecified.
 * d_keys and d_values must be 16-byte aligned; n < 2^32. Runs on cuda_stream
 * (NULL = legacy default) with scratch from the library's pool and waits for
 * the counts. */
int ght_partition(const uint32_t *d_keys, const uint32_t *d_values, uint64_t n, uint64_t seed, uint32_t shards,
                  uint32_t *d_out_keys, uint32_t *d_out_values, uint64_t *h_counts, void *cuda_stream);

/* d_dst[d_pos[j]] = d_src[j] for j < n (d_pos a permutation of [0, n));
 * asynchronous on cuda_stream. */
int ght_unpermute(const uint32_t *d_src, const uint32_t *d_pos, uint64_t n, uint32_t *d_dst, void *cuda_stream);

/* Device scratch a build of n keys uses for grouping (0 if this table
 * builds without grouping). */
uint64_t ght_build_scratch_bytes(const ght_table *t, uint64_t n);

/* Device scratch a ght_find of n device queries uses when it runs grouped
 * (config find_grouped): about 45 bytes per query; 0 if such a find runs per
 * query and needs none. */
uint64_t ght_find_scratch_bytes(const ght_table *t, uint64_t n);

/* Caller-owned device scratch (256-byte aligned, `bytes` long, kept alive
 * by the caller) for later builds and grouped finds; NULL clears it. Without
 * it (or where it is smaller than the call needs), a table whose storage the
 * library owns takes scratch from the library's stream-ordered pool, and a
 * table on caller storage builds ungrouped and finds per query. Calls that
 * use this buffer must not overlap on the device (they share it). */
int ght_set_build_scratch(ght_table *t, void *d_scratch, uint64_t bytes);

/* Fill *out (synchronises the stream when probe counters are on). */
int ght_stats(const ght_table *t, ght_stats_t *out);

/* Zero the find counters. */
int ght_reset_counters(ght_table *t);

/* Copy the raw slot array (num_slots slots of slot_bytes each, bucket-major)
 * to host memory h_slots, which holds n_slots 8-byte words (enough for
 * num_slots * slot_bytes bytes); synchronous. For validation. */
int ght_export(const ght_table *t, uint64_t *h_slots, uint64_t n_slots);

/* Bucket indices of each key under each of the table's hash functions,
 * computed by a device kernel: d_buckets[i * h + j] = h_j(d_keys[i]). */
int ght_hash_device(const ght_table *t, const uint32_t *d_keys, uint32_t *d_buckets, uint64_t n);

/* The same bucket computation on the host, with explicit constants:
 * h_out[i] = ((a * h_keys[i] + c) mod p) mod m, for 1 <= m < 2^32. */
int ght_hash_host(uint32_t a, uint32_t c, uint32_t m, const uint32_t *h_keys, uint32_t *h_out,
                  uint64_t n);

/* Memory-system ceiling probe (a measurement aid; the paper has no
 * counterpart). Runs `ops` operations on random 128-byte lines of d_lines
 * (num_lines lines, caller-owned device memory, 128-byte aligned, contents
 * are modified in modes 1-3), asynchronously on `cuda_stream` (NULL = legacy
 * default stream). The line of operation i is a mixer of (seed, i) mod
 * num_lines. Modes, after the access patterns of Sec. V:
 *   0  read the line (one 8-byte word of each 32-byte sector, so DRAM
 *      delivers all of it: a find's bucket probe, Sec. V-A/V-B);
 *   1  read the line, then one 64-bit CAS into its first slot that depends on
 *      the data read (an insert's probe and CAS, Sec. V-B), results unused;
 *   2  as 1, and each step's CAS results are consumed before the next
 *      step's reads (one atomic round trip per read);
 *   3  one 64-bit atomic add into a random line, no read;
 *   4  read the first half of the line (two 32-byte sectors);
 *   5  as 4, then one sector of the second half chosen by the data read.
 * Time it with events on the same stream. num_lines must be in [1, 2^32-1]. */
int ght_probe_lines(int mode, void *d_lines, uint64_t num_lines, uint64_t ops, uint32_t seed, void *cuda_stream);

/* Release the table (and its storage, if library-owned). NULL is a no-op. */
void ght_destroy(ght_table *t);

/* ---------------------------------------------------------------------------
 * Batched tables: many independent BCHT tables (b = 16, h = 3; Sec. III-A,
 * V-B) built and queried by single launches instead of one build and one find
 * per table. Not in the paper: it is the same per-table method, with the
 * tables' work merged into shared launches, for workloads of many small or
 * uneven tables.
 *
 * Inputs are concatenated over the tables: table t owns keys/values
 * [key_offsets[t], key_offsets[t+1]) and queries/results
 * [query_offsets[t], query_offsets[t+1]). Table t's hash constants come from
 * seed + t * 0x9E3779B97F4A7C15 (mod 2^64) with the same derivation as a
 * single table, per attempt.
 * ------------------------------------------------------------------------- */
typedef struct ght_batch ght_batch; /* opaque, library-owned */

typedef struct {
  uint32_t num_tables;
  uint32_t tables_failed;      /* tables without a successful build after repair */
  uint64_t total_keys, total_queries, total_slots, table_bytes;
  uint32_t rebuilds;           /* per-table rebuilds with fresh constants in the last build or run */
  int32_t tuned;               /* 1 after ght_batch_autotune */
  int32_t tile_lanes, keys_per_lane;              /* find shape */
  int32_t build_tile_lanes, build_keys_per_lane;  /* insert shape */
  double last_run_ms;          /* device time of the last ght_batch_run graph launch */
  uint64_t graph_launches;
  int32_t blocks_per_sm;       /* find grid: resident blocks per SM (0 = as many as fit) */
  int32_t build_blocks_per_sm; /* insert grid, likewise */
} ght_batch_stats_t;

/* Create num_tables empty tables, table t sized for h_capacities[t] keys at
 * h_load_factors[t] (Sec. III sizing), in one device allocation. cfg may be
 * NULL (max_chain, max_attempts and the launch shapes apply). NULL on error. */
ght_batch *ght_batch_create(uint32_t num_tables, const uint64_t *h_capacities, const double *h_load_factors,
                            uint64_t seed, const ght_config *cfg);

/* Issue later work on `cuda_stream` (NULL = legacy default stream). */
int ght_batch_set_stream(ght_batch *b, void *cuda_stream);

/* Set the input layout: num_tables + 1 non-decreasing offsets each, starting
 * at 0; table t's key count may not exceed its capacity. Synchronous upload. */
int ght_batch_set_layout(ght_batch *b, const uint64_t *h_key_offsets, const uint64_t *h_query_offsets);

/* Build every table from the concatenated device arrays with one fill and
 * one insert launch for the whole batch; reads the tables' status words
 * once, then rebuilds each failed table alone with its next constants (up to
 * max_attempts). GHT_ERR_BUILD_FAILED if any table stays unbuilt. */
int ght_batch_build(ght_batch *b, const uint32_t *d_keys, const uint32_t *d_values);

/* Find every table's queries with one launch (asynchronous). */
int ght_batch_find(const ght_batch *b, const uint32_t *d_queries, uint32_t *d_out);

/* Build and find in one CUDA-graph launch (fill, insert, find, status read
 * back), captured on the first call and re-captured when the arrays or the
 * launch shapes change; waits once. Tables whose build failed are rebuilt
 * alone and their queries answered again before returning. The graph is
 * launched on the batch's stream, which must not be capturing. */
int ght_batch_run(ght_batch *b, const uint32_t *d_keys, const uint32_t *d_values, const uint32_t *d_queries,
                  uint32_t *d_out);

/* Choose the insert and find launch shapes by timing each candidate on
 * these arrays: first the tile shape (lanes per bucket tile, keys per lane;
 * for finds also 4-lane tiles with 6 query sets per lane, the staged find
 * whose bucket parts wait in shared memory), then the grid (1-4 resident
 * blocks per SM, or as many as fit) of the best shape; keeps the fastest.
 * The tables are rebuilt as a side effect. */
int ght_batch_autotune(ght_batch *b, const uint32_t *d_keys, const uint32_t *d_values,
                       const uint32_t *d_queries, uint32_t *d_out);

int ght_batch_stats(const ght_batch *b, ght_batch_stats_t *out);

/* Per-table view in the single-table stats format (shape, constants, n). */
int ght_batch_table_stats(const ght_batch *b, uint32_t table, ght_stats_t *out);

/* Copy table `table`'s slots to host memory (synchronous). */
int ght_batch_export(const ght_batch *b, uint32_t table, uint64_t *h_slots, uint64_t n_slots);

void ght_batch_destroy(ght_batch *b);

/* ---------------------------------------------------------------------------
 * Served pool: device-resident BCHT tables answering a stream of find
 * requests and admitting build requests under an HBM budget. Not in the
 * paper: it serves the paper's tables to many clients.
 *
 * Continuous batching: a scheduler thread keeps up to two batched find
 * launches in flight; each new launch takes every pending find whose table is
 * built (oldest first, at most 2^22 queries and 4096 requests), gathers their
 * queries, finds them in one launch and scatters the answers, so requests that
 * arrive while others run join the next launch. A build worker admits build
 * requests in arrival order once the table fits in the budget (storage from
 * the library's stream-ordered pool) and builds on its own stream, overlapping
 * the finds. Each answer is exactly what a single-table find returns.
 * Device arrays passed to submit calls must stay valid until the request
 * completes.
 * ------------------------------------------------------------------------- */
typedef struct ght_pool ght_pool; /* opaque, library-owned */

typedef struct {
  int32_t status;           /* ght_status of the request */
  int32_t kind;             /* 0 find, 1 build */
  uint32_t table;
  int32_t launch_requests;  /* find requests packed into the same launch */
  uint64_t n;
  double queue_s;           /* submit -> start of its launch (or build) */
  double latency_s;         /* submit (or scheduled arrival) -> completion */
} ght_pool_result_t;

typedef struct {
  uint64_t budget_bytes, used_bytes;
  uint32_t tables, tables_ready;
  uint64_t find_launches, finds_done, queries_done, builds_done, builds_refused;
  uint64_t pending_finds, pending_builds;
  double mean_requests_per_launch;
} ght_pool_stats_t;

/* One request of a replayed trace. */
typedef struct {
  int32_t kind;             /* 0 find, 1 build */
  uint32_t table;           /* find: table id */
  const uint32_t *d_in;     /* find: queries; build: keys */
  const uint32_t *d_values; /* build: values */
  uint32_t *d_out;          /* find: answers */
  uint64_t n;               /* queries or pairs */
  uint64_t capacity;        /* build */
  double load_factor;       /* build */
  uint64_t seed;            /* build */
  double arrival_s;         /* arrival time from the start of the replay */
} ght_pool_request_t;

/* Create a pool on the current device with `hbm_budget_bytes` for table
 * storage; cfg (may be NULL) supplies max_chain, max_attempts and shapes. */
ght_pool *ght_pool_create(uint64_t hbm_budget_bytes, const ght_config *cfg);

/* Queue a build of a new table (capacity, load factor, seed) from n pairs;
 * *table_id receives the new table's id at once (finds on it wait for the
 * build). Returns a ticket, 0 on invalid arguments. A table larger than the
 * whole budget completes with GHT_ERR_OOM. */
uint64_t ght_pool_submit_build(ght_pool *p, uint64_t capacity, double load_factor, uint64_t seed,
                               const uint32_t *d_keys, const uint32_t *d_values, uint64_t n, uint32_t *table_id);

/* Queue a find of n queries on a table; returns a ticket (0 on error). */
uint64_t ght_pool_submit_find(ght_pool *p, uint32_t table_id, const uint32_t *d_queries, uint32_t *d_out, uint64_t n);

/* Wait (at most timeout_s) for a request; fills *out (may be NULL) and
 * forgets the ticket. Returns the request's status. */
int ght_pool_wait(ght_pool *p, uint64_t ticket, double timeout_s, ght_pool_result_t *out);

/* Drop a built table; its storage returns to the budget once no launch reads it. */
int ght_pool_drop_table(ght_pool *p, uint32_t table_id);

int ght_pool_stats(ght_pool *p, ght_pool_stats_t *out);

/* Replay `count` requests at their arrival times: through the pool
 * (serial = 0) or as plain single-table calls one at a time in arrival order
 * (serial = 1). latency_s[i] = completion - scheduled arrival; status[i];
 * *makespan_s = last completion - start. Arrays may be NULL. */
int ght_pool_replay(ght_pool *p, const ght_pool_request_t *trace, uint64_t count, int serial, double *latency_s,
                    int32_t *status, double *makespan_s);

/* Stop the scheduler threads (after the queued requests finish) and free
 * everything. */
void ght_pool_destroy(ght_pool *p);

#ifdef __cplusplus
}
#endif
#endif
