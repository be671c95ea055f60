// ght_api.cu -- host side of the C ABI declared in include/ght.h.
//
// Sizing, constant derivation, the build retry loop and the host<->device
// pipelines live here; all table arithmetic on keys runs in the kernels of
// kern_bcht.cu / kern_other.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>
#include <thread>

#include "ght.h"
#include "ght_device.cuh"
#include "ght_batch.h"
#include "ght_host.h"
#include "ght_internal.h"

namespace {

using ght::host::cuda_fail;
using ght::host::fail;
using ght::host::pool_alloc;

using ght::host::wait_event;

constexpr uint64_t kCtrlBytes = sizeof(ght::Ctrl);

struct Shape {
  int scheme, b, h, t;
  uint32_t max_chain, max_attempts;
  int count_probes;
  int tile_lanes, blocks_per_sm, keys_per_lane;                    // find
  int build_tile_lanes, build_blocks_per_sm, build_keys_per_lane;  // build
  int group_build;  // 1: group the input by first-choice bucket range before inserting
  int ranked_build;  // 1: two-phase build (ranked first-choice placement, then cuckoo insert)
  int find_async;    // 1: finds stage bucket parts in shared memory (BCHT b = 16, the set)
  int check_dups;    // 1: a successful build checks that no key is stored twice
  int slot_bytes;   // 8 (key/value pair) or 4 (keys-only set)
  uint32_t max_steps;  // per-key step bound of the insert kernels (0: derived)
  int find_grouped;    // 1: grouped find (rounds by bucket range), else per query
  uint64_t m;
};

// Launch shapes measured fastest on GB300 at 2^27-2^28 keys (insert with
// dynamic chunk claims; load factors near each scheme's working range).
// Finds read 16-pair buckets fastest with two queries in flight per lane
// and 32-pair buckets with one; builds the other way round, except the
// keys-only set, fastest with one key per lane for both. BCHT reads a
// 16-pair bucket with 4 lanes in its finds and 16 in its inserts; every
// other bucketed kernel uses 8.
void default_shape(int scheme, int b, ght_config *c) {
  if (scheme == GHT_CUCKOO1) {
    c->tile_lanes = c->build_tile_lanes = 1;
    c->keys_per_lane = c->build_keys_per_lane = 1;
    return;
  }
  c->tile_lanes = scheme == GHT_BCHT && b == 16 ? 4 : 8;
  c->build_tile_lanes = scheme == GHT_BCHT && b == 16 ? 16 : 8;
  if (scheme == GHT_BCHT_SET) {
    c->keys_per_lane = c->build_keys_per_lane = 1;
  } else {
    c->keys_per_lane = b == 16 ? 2 : 1;
    c->build_keys_per_lane = b == 16 ? 1 : 2;
  }
}

int default_config(int scheme, ght_config *c) {
  memset(c, 0, sizeof *c);
  switch (scheme) {
    case GHT_BCHT: c->bucket_size = 16; c->num_hashes = 3; c->max_chain = 1000; break;
    case GHT_P2BHT: c->bucket_size = 16; c->num_hashes = 2; break;
    case GHT_IHT: c->bucket_size = 16; c->num_hashes = 3; c->threshold = 13; break;
    case GHT_CUCKOO1: c->bucket_size = 1; c->num_hashes = 3; c->max_chain = 1000; break;
    case GHT_BCHT_LB: c->bucket_size = 16; c->num_hashes = 3; c->max_chain = 1000; break;
    case GHT_BCHT_SET: c->bucket_size = 32; c->num_hashes = 3; c->max_chain = 1000; break;
    default: return fail(GHT_ERR_INVALID_ARG, "unknown scheme %d", scheme);
  }
  c->max_attempts = 50;
  default_shape(scheme, c->bucket_size, c);
  return GHT_OK;
}

uint64_t device_l2_bytes();

// Resolve a config against the scheme's defaults and validate the shape.
int resolve(int scheme, uint64_t capacity, double lf, const ght_config *user, Shape *s) {
  ght_config d;
  int rc = default_config(scheme, &d);
  if (rc) return rc;
  if (user) {
    if (user->bucket_size) d.bucket_size = user->bucket_size;
    if (user->num_hashes) d.num_hashes = user->num_hashes;
    if (user->max_chain) d.max_chain = user->max_chain;
    if (user->max_attempts) d.max_attempts = user->max_attempts;
    default_shape(scheme, d.bucket_size, &d);
    if (user->tile_lanes) d.tile_lanes = user->tile_lanes;
    if (user->build_tile_lanes) d.build_tile_lanes = user->build_tile_lanes;
    d.count_probes = user->count_probes;
    d.blocks_per_sm = user->blocks_per_sm;
    d.build_blocks_per_sm = user->build_blocks_per_sm;
    if (user->keys_per_lane) d.keys_per_lane = user->keys_per_lane;
    if (user->build_keys_per_lane) d.build_keys_per_lane = user->build_keys_per_lane;
    d.group_build = user->group_build;
    d.ranked_build = user->ranked_build;
    d.find_async = user->find_async;
    d.check_duplicates = user->check_duplicates;
    d.max_steps = user->max_steps;
    d.find_grouped = user->find_grouped;
    if (user->threshold) d.threshold = user->threshold;
    else if (scheme == GHT_IHT) d.threshold = (4 * d.bucket_size + 4) / 5;  // ceil(0.8 b)
  }
  if (!(lf > 0.0) || !(lf <= 1.0)) return fail(GHT_ERR_INVALID_ARG, "load factor %g is not in (0, 1]", lf);
  const int b = d.bucket_size, h = d.num_hashes;
  if (scheme == GHT_BCHT_SET) {
    if (b != 32) return fail(GHT_ERR_INVALID_ARG, "the keys-only set has 32 keys per bucket");
    if (h < 2 || h > 4) return fail(GHT_ERR_INVALID_ARG, "the keys-only set needs 2..4 hash functions");
    if (!ght::set_shape_supported(b, d.build_tile_lanes))
      return fail(GHT_ERR_INVALID_ARG, "tile of %d lanes unsupported for the set", d.build_tile_lanes);
    // find tiles: 8 lanes, or 4 for the staged find (checked below)
    if (!ght::set_shape_supported(b, d.tile_lanes) && d.tile_lanes != 4)
      return fail(GHT_ERR_INVALID_ARG, "tile of %d lanes unsupported for the set", d.tile_lanes);
  } else if (scheme == GHT_CUCKOO1) {
    if (b != 1) return fail(GHT_ERR_INVALID_ARG, "CUCKOO1 has bucket size 1");
    if (h < 2 || h > 4) return fail(GHT_ERR_INVALID_ARG, "CUCKOO1 needs 2..4 hash functions");
  } else {
    if (b != 16 && b != 32) return fail(GHT_ERR_INVALID_ARG, "bucket size %d (16 or 32)", b);
    if (scheme == GHT_P2BHT && h != 2) return fail(GHT_ERR_INVALID_ARG, "P2BHT uses 2 hash functions");
    if (scheme == GHT_IHT && h != 3) return fail(GHT_ERR_INVALID_ARG, "IHT uses 3 hash functions");
    if ((scheme == GHT_BCHT || scheme == GHT_BCHT_LB) && (h < 2 || h > 4))
      return fail(GHT_ERR_INVALID_ARG, "BCHT needs 2..4 hash functions");
    for (int g : {d.tile_lanes, d.build_tile_lanes}) {
      const bool ok = scheme == GHT_BCHT ? ght::bcht_shape_supported(b, g) : ght::other_shape_supported(scheme, b, g);
      if (!ok) return fail(GHT_ERR_INVALID_ARG, "tile of %d lanes unsupported for bucket size %d", g, b);
    }
  }
  // the staged find reads buckets of 16 or 32 pairs (BCHT, P2BHT, IHT, the
  // load-balanced BCHT) or 32 keys (the set) with 4-lane tiles; a default
  // find tile of another width gives way to it unless tile_lanes is given
  const bool user_tile = user && user->tile_lanes;
  const bool staged_bucket = scheme != GHT_CUCKOO1;
  const bool staged_shape = staged_bucket && (d.tile_lanes == 4 || !user_tile);
  if (d.find_async > 0 && !staged_shape)
    return fail(GHT_ERR_INVALID_ARG, "the staged find is for bucketed tables with 4-lane tiles");
  const bool two_lines = scheme != GHT_BCHT_SET && b == 32;  // 256-byte buckets
  const int max_sets = two_lines ? 6 : 8;
  if (d.build_keys_per_lane != 1 && d.build_keys_per_lane != 2)
    return fail(GHT_ERR_INVALID_ARG, "keys per lane must be 1 or 2");
  if (scheme == GHT_IHT && (d.threshold < 1 || d.threshold > b + 1))
    return fail(GHT_ERR_INVALID_ARG, "IHT threshold %d outside [1, b+1]", d.threshold);
  // Sec. III: C = m b, load factor n / C  =>  m = ceil(capacity / (lf b))
  double want = std::ceil((double)capacity / (lf * (double)b));
  if (want < 1.0) want = 1.0;
  if (want > 4294967295.0) return fail(GHT_ERR_INVALID_ARG, "table needs more than 2^32-1 buckets");
  // The staged find by default where it applies and the slots do not fit in
  // the L2: there its deeper pipeline hides DRAM latency; on an L2-resident
  // table the register find's higher occupancy wins. A given keys_per_lane of
  // 1 keeps the register find. 6 query sets in flight (3 for 256-byte
  // buckets) unless keys_per_lane is given.
  const uint64_t slot_bytes = scheme == GHT_BCHT_SET ? 4 : 8;
  const bool kpl_given = user && user->keys_per_lane;
  const bool async_find =
      d.find_async > 0 || (d.find_async == 0 && staged_shape && !(kpl_given && d.keys_per_lane < 2) &&
                           (uint64_t)want * b * slot_bytes >= device_l2_bytes());
  if (async_find && !kpl_given) d.keys_per_lane = two_lines ? 3 : 6;
  if (async_find) d.tile_lanes = 4;
  if (!async_find && scheme == GHT_BCHT_SET && d.tile_lanes == 4)
    return fail(GHT_ERR_INVALID_ARG, "4-lane find tiles of the set need the staged find");
  if (async_find ? (d.keys_per_lane < 2 || d.keys_per_lane > max_sets) : (d.keys_per_lane != 1 && d.keys_per_lane != 2))
    return fail(GHT_ERR_INVALID_ARG, "keys per lane must be 1 or 2 (2 to %d for the staged find)", max_sets);
  // the grouped find reads 16-pair buckets (BCHT, P2BHT, IHT, the load-balanced BCHT)
  const bool grouped_shape = scheme != GHT_CUCKOO1 && scheme != GHT_BCHT_SET && b == 16;
  if (d.find_grouped > 0 && !grouped_shape)
    return fail(GHT_ERR_INVALID_ARG, "the grouped find is for tables of 16-pair buckets");
  s->scheme = scheme;
  s->b = b;
  s->h = h;
  s->t = d.threshold;
  s->max_chain = d.max_chain;
  s->max_attempts = d.max_attempts ? d.max_attempts : 1;
  s->count_probes = d.count_probes;
  s->tile_lanes = d.tile_lanes;
  s->blocks_per_sm = d.blocks_per_sm;
  s->keys_per_lane = d.keys_per_lane;
  s->build_tile_lanes = d.build_tile_lanes;
  s->build_blocks_per_sm = d.build_blocks_per_sm;
  s->build_keys_per_lane = d.build_keys_per_lane;
  s->group_build = d.group_build;
  // ranked placement applies to the cuckoo tables with buckets (BCHT and the set)
  s->ranked_build = (scheme == GHT_BCHT || scheme == GHT_BCHT_SET) ? d.ranked_build : -1;
  s->slot_bytes = (int)slot_bytes;
  s->find_async = async_find ? 1 : 0;
  s->check_dups = d.check_duplicates > 0 ? 1 : 0;
  s->max_steps = d.max_steps;
  s->find_grouped = grouped_shape ? d.find_grouped : -1;
  s->m = (uint64_t)want;
  return GHT_OK;
}

uint64_t bytes_of(const Shape &s) {
  const uint64_t slots = s.m * (uint64_t)s.b * (uint64_t)s.slot_bytes;
  return kCtrlBytes + ((slots + 255ull) & ~255ull);
}

// Grouping shape: at most 512 groups of 2^shift consecutive buckets.
void group_shape(uint64_t m, int *shift, uint32_t *groups) {
  int bits = 0;
  while ((1ull << bits) < m) ++bits;
  *shift = bits > 9 ? bits - 9 : 0;
  *groups = (uint32_t)(((m - 1) >> *shift) + 1);
}

// Region of each group in a two-phase grouped build: the grouping writes
// group g's pairs from g * region on, which needs no count pass; the region
// holds the mean group size plus eight standard deviations of a uniform
// hash's group sizes and 64, so only inputs whose first-choice buckets
// crowd far beyond a random hash's overflow it (the build then regroups with
// exact offsets). 0: exact offsets (a region layout would not fit 32-bit
// indices).
uint32_t group_region(uint64_t n, uint32_t groups) {
  if (n == 0 || groups == 0) return 0;
  const double mean = (double)n / groups;
  const uint64_t region = ((uint64_t)std::ceil(mean + 8.0 * std::sqrt(mean) + 64.0) + 7ull) & ~7ull;
  return region * groups <= 0xFFFFFFFFull ? (uint32_t)region : 0u;
}

// Scratch of a grouped build: counts and cursors, then the regrouped keys and
// values (`len` entries each).
uint64_t group_scratch_bytes(uint64_t len) {
  const uint64_t head = 2ull * ght::kMaxGroups * sizeof(uint32_t);
  const uint64_t arr = (len * sizeof(uint32_t) + 255ull) & ~255ull;
  return head + 2 * arr;
}

// Overflow list capacity of a two-phase build of n keys: far above the ~10 %
// of keys that overflow their first-choice bucket at load factor 1 with
// 16-slot buckets; a larger overflow (many keys sharing a bucket) falls back
// to the cuckoo insert of every key.
uint64_t place_cap(uint64_t n) { return std::min<uint64_t>(n, n / 4 + 1024); }

uint64_t align256(uint64_t x) { return (x + 255ull) & ~255ull; }

uint64_t place_scratch_bytes(uint64_t m, uint64_t n) {
  return align256(m * sizeof(uint32_t)) + 2 * align256(place_cap(n) * sizeof(uint32_t));
}

ght::PlaceBuffers place_buffers(char *scr, uint64_t m, uint64_t n) {
  ght::PlaceBuffers pb;
  pb.counters = reinterpret_cast<uint32_t *>(scr);
  pb.cap = place_cap(n);
  pb.ovf_k = reinterpret_cast<uint32_t *>(scr + align256(m * sizeof(uint32_t)));
  pb.ovf_v = pb.ovf_k + align256(pb.cap * sizeof(uint32_t)) / sizeof(uint32_t);
  return pb;
}

}  // namespace

// Static staging array of the allocation-free host find
// (ght_find_host_noalloc). It is a file-scope device variable, so no
// allocator is involved once it exists; but with lazy module loading the
// driver creates it (32 MiB) only when the host first asks for its address.
// That first lookup therefore happens when a table is created on a device --
// a call that allocates anyway -- never inside the allocation-free call.
// In host code the name g_noalloc_staging is only a host-side stand-in: the
// device address is looked up once per device, with that device current,
// and passed to the copies and the kernel.
namespace {

constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) uint32_t g_noalloc_staging[2ull * GHT_NOALLOC_MAX_QUERIES];

struct NoAllocDevice {
  uint32_t *base = nullptr;     // device address of g_noalloc_staging on this device
  cudaEvent_t pending = nullptr;  // completion of a call that timed out
  bool busy = false;            // a timed-out call may still use the array
  bool failed = false;          // set-up failed on this device
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc[kNoAllocMaxDevices];

// Once per device, with that device current: resolve the staging array's
// device address and create the event that tracks a timed-out call.
void noalloc_setup(int dev) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocDevice &d = g_noalloc[dev];
  if (d.base || d.failed) return;
  void *p = nullptr;
  cudaEvent_t ev = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_staging) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    d.failed = true;
    return;
  }
  d.base = static_cast<uint32_t *>(p);
  d.pending = ev;
}

}  // namespace

struct ght_table {
  Shape shape;
  int device = 0;  // the device current at creation, where the storage lives
  uint64_t capacity = 0;
  double lf = 0;
  uint64_t seed = 0;
  cudaStream_t stream = nullptr;
  void *storage = nullptr;
  uint64_t storage_bytes = 0;
  bool owns_storage = false;
  uint64_t *slots = nullptr;
  ght::Ctrl *ctrl = nullptr;
  uint32_t a[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
  uint32_t rng_seed = 1;
  bool built = false;
  uint64_t n_stored = 0;
  uint32_t attempts = 0;
  ght::Ctrl *h_ctrl = nullptr;  // pinned mirror of the control block
  cudaEvent_t done = nullptr;
  // timing events: fill start, fill end, pre-insert work end (grouping and/or ranked placement),
  // insert end, find start, find end, grouping end (when a grouped build also places by rank),
  // first and last host-to-device copy of the last host-buffer call
  // first grouping level end (when a second level splits the groups)
  cudaEvent_t tev[10] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  mutable bool timed_h2d = false;
  mutable uint64_t h2d_bytes = 0;
  bool timed_build = false;
  bool last_grouped = false;
  bool last_split = false;
  bool last_ranked = false;
  mutable bool last_find_grouped = false;
  uint64_t place_overflow = 0;
  void *scratch = nullptr;  // caller-owned build scratch (ght_set_build_scratch)
  uint64_t scratch_bytes = 0;
  mutable bool timed_find = false;
  mutable uint64_t insert_probes = 0, insert_retries = 0, insert_evictions = 0, longest_chain = 0;

  void derive(uint32_t attempt) {
    ght::host::derive_constants(seed, attempt, shape.h, a, c);
    rng_seed = ght::host::derive_rng_seed(seed, attempt);
  }

  // table size in 8-byte words (what the fill kernel writes)
  uint64_t words() const { return shape.m * (uint64_t)shape.b * (uint64_t)shape.slot_bytes / 8ull; }

  ght::TableView view() const {
    ght::TableView v;
    v.slots = slots;
    v.ctrl = ctrl;
    for (int i = 0; i < 4; ++i) {
      v.hf.a[i] = a[i];
      v.hf.c[i] = c[i];
    }
    v.hf.mod = ght::make_fastmod((uint32_t)shape.m);
    v.m = (uint32_t)shape.m;
    v.h = shape.h;
    v.t = shape.t;
    v.max_chain = shape.max_chain;
    v.rng_seed = rng_seed;
    // Every bucket visit ends in a stored key, an exchange, or a failed CAS
    // that fills one more slot for good, so a key needs at most
    // (max_chain + 1) visits of at most h * (b + 1) reads each. A configured
    // bound replaces the derived one.
    const uint64_t steps = ((uint64_t)shape.max_chain + 2ull) * (uint64_t)shape.h * ((uint64_t)shape.b + 2ull) + 64ull;
    v.max_steps = shape.max_steps ? shape.max_steps : (uint32_t)std::min<uint64_t>(steps, 0xFFFFFFF0ull);
    v.first = 0;
    return v;
  }

  ght::LaunchOpts find_opts() const {
    ght::LaunchOpts o;
    o.tile_lanes = shape.tile_lanes;
    o.blocks_per_sm = shape.blocks_per_sm;
    o.keys_per_lane = shape.keys_per_lane;
    o.count = shape.count_probes != 0;
    o.async_find = shape.find_async != 0;
    return o;
  }

  ght::LaunchOpts build_opts() const {
    ght::LaunchOpts o;
    o.tile_lanes = shape.build_tile_lanes;
    o.blocks_per_sm = shape.build_blocks_per_sm;
    o.keys_per_lane = shape.build_keys_per_lane;
    o.count = shape.count_probes != 0;
    return o;
  }
};

namespace {

// Insert n pairs. The warps claim runs of 32-pair chunks from the control
// block's work cursor, which must be zero at launch (the fill clears it), so
// that the warps finish together however long the eviction chains of their
// keys are; a static slice per warp left a slow tail of 15-30 % at 2^28 keys.
// past_first: the keys are the overflow of a first-choice placement, whose
// H_0 buckets are full (the placement counted that visit), so a BCHT insert
// starts them at H_1 instead of reading H_0 again and exchanging there.
cudaError_t launch_insert(const ght_table *t, const uint32_t *k, const uint32_t *v, uint64_t n,
                          bool past_first = false) {
  ght::TableView tv = t->view();
  if (past_first && tv.h > 1 && (t->shape.scheme == GHT_BCHT || t->shape.scheme == GHT_BCHT_SET)) tv.first = 1;
  ght::LaunchOpts o = t->build_opts();
  o.dynamic = true;
  if (t->shape.scheme == GHT_BCHT) return ght::launch_insert_bcht(t->shape.b, tv, k, v, n, o, t->stream);
  if (t->shape.scheme == GHT_BCHT_SET) return ght::launch_insert_set(tv, k, v ? v : k, n, o, t->stream);
  return ght::launch_insert_other(t->shape.scheme, t->shape.b, tv, k, v, n, o, t->stream);
}

// L2 size of the current device (bytes; cached per device).
uint64_t device_l2_bytes() {
  static std::mutex mu;
  static uint64_t cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 128ull << 20;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!cache[dev]) {
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || l2 <= 0) {
      cudaGetLastError();
      l2 = 128 << 20;
    }
    cache[dev] = (uint64_t)l2;
  }
  return cache[dev];
}

// Whether a build of n keys groups its input first by first-choice bucket
// range (config group_build: 1 on, -1 off, 0 by table size); it also needs
// scratch (caller-set, or the library pool when the library owns the table
// storage), else the build runs in input order.
bool wants_grouping(const ght_table *t, uint64_t n) {
  if (t->shape.scheme == GHT_CUCKOO1 || n == 0 || n > 0xFFFFFFFFull) return false;
  if (t->shape.group_build != 0) return t->shape.group_build > 0;
  // default: cuckoo tables with buckets far larger than the L2, where the
  // grouped two-phase build measured 1.3-1.4x faster than the insert of
  // every key in input order (2^28 keys); at 2^20-2^24 keys it was slower
  if (t->shape.scheme != GHT_BCHT && t->shape.scheme != GHT_BCHT_SET) return false;
  return t->storage_bytes >= 4ull * device_l2_bytes();
}

// Whether a build of n keys runs in two phases (ranked first-choice
// placement, then the cuckoo insert of the overflow).
bool wants_ranked(const ght_table *t, uint64_t n) {
  if (t->shape.ranked_build < 0 || n == 0 || n > 0xFFFFFFFFull) return false;
  // default: with the grouping, whose order keeps the placement's stores in L2
  return t->shape.ranked_build > 0 || wants_grouping(t, n);
}

// Second-level split of a two-phase grouped build (the block placement):
// sub-groups of 2^fine_shift buckets (64 KB of table each), 2^subs_log2 <=
// 128 per group, `bins` in all, each in a region of region2 pairs. False
// where the first level's regions are too small or the split too fine.
struct SubShape {
  int fine_shift = 0, subs_log2 = 0;
  uint32_t bins = 0, region2 = 0;
};

bool sub_shape(const Shape &s, uint64_t n, int shift, uint32_t region1, SubShape *out) {
  if (region1 < ght::kSubgroupMinRegion) return false;
  const uint64_t m = s.m;
  const int fine = ght::block_place_fine_shift(s.b, s.scheme == GHT_BCHT_SET);
  SubShape sh;
  sh.fine_shift = shift < fine ? shift : fine;
  sh.subs_log2 = shift - sh.fine_shift;
  if (sh.subs_log2 > 7) return false;
  sh.bins = (uint32_t)(((m - 1) >> sh.fine_shift) + 1);
  sh.region2 = group_region(n, sh.bins);
  if (!sh.region2) return false;
  *out = sh;
  return true;
}

// Entries of the regrouped arrays of a build of n pairs (the groups' regions
// when the build places by rank, else n).
uint64_t grouped_len(const ght_table *t, uint64_t n) {
  int shift = 0;
  uint32_t groups = 1;
  group_shape(t->shape.m, &shift, &groups);
  const uint32_t region = wants_ranked(t, n) ? group_region(n, groups) : 0u;
  return region ? (uint64_t)groups * region : n;
}

// Scratch of the second-level split: the split pairs and one cursor per
// sub-group (0 where the build does not use it).
uint64_t sub_scratch_bytes(const ght_table *t, uint64_t n) {
  if (!wants_grouping(t, n) || !wants_ranked(t, n)) return 0;
  int shift = 0;
  uint32_t groups = 1;
  group_shape(t->shape.m, &shift, &groups);
  SubShape sh;
  if (!sub_shape(t->shape, n, shift, group_region(n, groups), &sh)) return 0;
  return 2 * align256((uint64_t)sh.bins * sh.region2 * sizeof(uint32_t)) + align256(sh.bins * sizeof(uint32_t));
}

uint64_t build_scratch_need(const ght_table *t, uint64_t n) {
  return (wants_grouping(t, n) ? group_scratch_bytes(grouped_len(t, n)) : 0) +
         (wants_ranked(t, n) ? place_scratch_bytes(t->shape.m, n) : 0) + sub_scratch_bytes(t, n);
}

// Scratch of a two- or grouped-phase build: the caller's, else (for tables on
// library storage) the library pool; NULL if neither is available.
char *build_scratch(ght_table *t, uint64_t need, void **pool_buf) {
  *pool_buf = nullptr;
  if (t->scratch && t->scratch_bytes >= need) return static_cast<char *>(t->scratch);
  if (t->owns_storage && pool_alloc(pool_buf, need, t->stream) == cudaSuccess) return static_cast<char *>(*pool_buf);
  cudaGetLastError();
  *pool_buf = nullptr;
  return nullptr;
}

cudaError_t launch_place(const ght_table *t, const uint32_t *k, const uint32_t *v, uint64_t n,
                         const ght::PlaceBuffers &pb) {
  const bool count = t->shape.count_probes != 0;
  if (t->shape.scheme == GHT_BCHT_SET) return ght::launch_place_set(t->view(), k, n, pb, count, t->stream);
  return ght::launch_place_bcht(t->shape.b, t->view(), k, v, n, pb, count, t->stream);
}

// Grouped find (kern_gfind.cu): shape of the two grouping levels of each
// round (by H_r bucket range: 2^shift-bucket groups, then 256-bucket (32 KB)
// sub-groups) and of the return to query order (by position: 2^20-position
// groups, then 2^13-position windows). Regions are sized for the whole
// batch, which bounds every round's list.
struct GFindShape {
  int shift = 0;
  uint32_t groups = 0, region1 = 0;
  SubShape sub;
  uint32_t rgroups = 0, rbins = 0;
  uint64_t l1_len = 0, l2_len = 0;
};

constexpr int kRetShift1 = 20;

bool gfind_shape(const ght_table *t, uint64_t n, GFindShape *g) {
  if (n == 0 || n > 0xFFFFFFFFull - (1ull << kRetShift1)) return false;
  group_shape(t->shape.m, &g->shift, &g->groups);
  g->region1 = group_region(n, g->groups);
  if (!g->region1 || g->region1 < ght::kSubgroupMinRegion) return false;
  // second level: sub-groups of 2^kGFindFineShift buckets, at most 256 per group
  g->sub.fine_shift = std::min(g->shift, ght::kGFindFineShift);
  g->sub.subs_log2 = g->shift - g->sub.fine_shift;
  if (g->sub.subs_log2 > 8) return false;
  g->sub.bins = (uint32_t)(((t->shape.m - 1) >> g->sub.fine_shift) + 1);
  g->sub.region2 = group_region(n, g->sub.bins);
  if (!g->sub.region2) return false;
  g->rgroups = (uint32_t)((n + (1ull << kRetShift1) - 1) >> kRetShift1);
  g->rbins = (uint32_t)((n + (1ull << ght::kGFindWindowLog2) - 1) >> ght::kGFindWindowLog2);
  g->l1_len = std::max<uint64_t>((uint64_t)g->groups * g->region1, (uint64_t)g->rgroups << kRetShift1);
  g->l2_len = std::max<uint64_t>((uint64_t)g->sub.bins * g->sub.region2, (uint64_t)g->rbins << ght::kGFindWindowLog2);
  return g->l2_len <= 0xFFFFFFFFull;
}

// scratch: [counters][cursors: level 1, level 2, return 1, return 2][level-1
// keys, positions][level-2 keys, positions, buckets][next-round keys,
// positions][answers: positions, values][spill: keys, positions, rounds]
constexpr uint64_t kGFindCounters = 64;  // 8-byte counters
uint64_t gfind_scratch_bytes(const GFindShape &g, uint64_t n) {
  const uint64_t cur = 2 * align256(ght::kMaxGroups * 4ull) + 2 * align256(std::max<uint64_t>(g.sub.bins, g.rbins) * 4ull);
  return kGFindCounters * 8 + cur + 2 * align256(g.l1_len * 4) + 2 * align256(g.l2_len * 4) + align256(g.l2_len) +
         7 * align256(n * 4);
}

// Whether a find of n device queries runs grouped: only where config
// find_grouped is 1. Measured on GB300 with 2^28 queries against a 2^28-key
// BCHT (2.2 GB of slots): grouped 16.6 / 12.0 ms against 19.9 / 12.8 ms per
// query for all-missing keys at LF 0.99 / 0.9, but 10.4 / 9.1 against 9.8 /
// 7.8 ms for all-present keys -- the answers' return to query order (2.6 ms)
// costs more than the rounds save when most queries end at their first
// bucket -- so the per-query find stays the default.
bool wants_grouped_find(const ght_table *t, uint64_t n) { return t->shape.find_grouped > 0 && n > 0; }

// The grouped find's launches on the table's stream. Returns cudaErrorNotSupported
// (nothing launched) where the batch's shape or scratch does not allow it.
cudaError_t launch_find_grouped(const ght_table *t, const uint32_t *q, uint32_t *out, uint64_t n) {
  GFindShape g;
  if ((reinterpret_cast<uintptr_t>(q) & 15u) || !gfind_shape(t, n, &g)) return cudaErrorNotSupported;
  const uint64_t need = gfind_scratch_bytes(g, n);
  void *pool_buf = nullptr;
  char *scr = nullptr;
  if (t->scratch && t->scratch_bytes >= need) scr = static_cast<char *>(t->scratch);
  else if (t->owns_storage && pool_alloc(&pool_buf, need, t->stream) == cudaSuccess) scr = static_cast<char *>(pool_buf);
  if (!scr) {
    cudaGetLastError();
    return cudaErrorNotSupported;
  }
  const cudaStream_t s = t->stream;
  const bool early = t->shape.scheme == GHT_BCHT;
  const bool count = t->shape.count_probes != 0;
  char *p = scr;
  unsigned long long *ctr = reinterpret_cast<unsigned long long *>(p);  // [0..4): claims, [4..8): next-round counts,
  p += kGFindCounters * 8;                                              // [8]: answers, [9]: spill
  auto take = [&](uint64_t bytes) {
    char *r = p;
    p += align256(bytes);
    return reinterpret_cast<uint32_t *>(r);
  };
  const uint64_t bins_max = std::max<uint64_t>(g.sub.bins, g.rbins);
  uint32_t *cur1 = take(ght::kMaxGroups * 4ull), *cur_r1 = take(ght::kMaxGroups * 4ull);
  uint32_t *cur2 = take(bins_max * 4), *cur_r2 = take(bins_max * 4);
  uint32_t *l1k = take(g.l1_len * 4), *l1p = take(g.l1_len * 4);
  uint32_t *l2k = take(g.l2_len * 4), *l2p = take(g.l2_len * 4);
  uint8_t *l2b = reinterpret_cast<uint8_t *>(take(g.l2_len));  // each item's bucket within its sub-group
  uint32_t *ck = take(n * 4), *cp = take(n * 4);
  uint32_t *rp = take(n * 4), *rv = take(n * 4);
  ght::SpillList spill;
  spill.k = take(n * 4);
  spill.v = take(n * 4);
  spill.round = take(n * 4);
  spill.count = ctr + 9;
  spill.cap = n;
  ght::GroupedFindLists fl;
  fl.res_p = rp;
  fl.res_v = rv;
  fl.res_count = ctr + 8;
  fl.cont_k = ck;
  fl.cont_p = cp;
  fl.cap = n;
  cudaError_t e = cudaMemsetAsync(ctr, 0, kGFindCounters * 8, s);
  ght::SubSplit ss;
  ss.ends1 = cur1;
  ss.region1 = g.region1;
  ss.region1_M = ght::make_fastmod(g.region1).M;
  ss.fine_shift = g.sub.fine_shift;
  ss.subs_log2 = g.sub.subs_log2;
  ss.groups = g.groups;
  for (int r = 0; r < t->shape.h && e == cudaSuccess; ++r) {
    ght::TableView tv = t->view();
    tv.first = r;  // the groupings of round r go by H_r
    ght::GroupExtras x;
    x.spill = spill;
    if (r == 0) {  // the queries themselves, with their positions
      e = ght::launch_group(tv, q, nullptr, n, g.shift, g.groups, nullptr, cur1, l1k, l1p, s, g.region1, x);
    } else {  // the items left by round r - 1
      x.d_n = ctr + 4 + (r - 1);
      e = ght::launch_group(tv, ck, cp, n, g.shift, g.groups, nullptr, cur1, l1k, l1p, s, g.region1, x);
    }
    if (e == cudaSuccess) {
      ght::GroupExtras x2;
      x2.spill = spill;
      x2.out_b = l2b;
      e = ght::launch_subgroup(tv, l1k, l1p, (uint64_t)g.groups * g.region1, ss, g.sub.bins, cur2, g.sub.region2, l2k,
                               l2p, s, x2);
    }
    if (e == cudaSuccess) {
      ght::GroupedFindLists fr = fl;
      fr.claim = ctr + r;
      fr.cont_count = ctr + 4 + r;
      e = ght::launch_grouped_lookup(tv, r, early, count, l2k, l2p, l2b, cur2, g.sub.region2, g.sub.bins,
                                     g.sub.fine_shift, fr, s);
    }
  }
  if (e == cudaSuccess) e = ght::launch_grouped_spill(t->view(), early, count, spill, fl, n, s);
  // every query has exactly one answer: back to query order by position
  if (e == cudaSuccess) {
    ght::GroupExtras xr;
    xr.ident = true;
    xr.d_n = fl.res_count;  // n, unless a grouping fault dropped items (kStatusCorrupt)
    e = ght::launch_group(t->view(), rp, rv, n, kRetShift1, g.rgroups, nullptr, cur_r1, l1k, l1p, s,
                          1u << kRetShift1, xr);
  }
  if (e == cudaSuccess) {
    ght::SubSplit sr;
    sr.ends1 = cur_r1;
    sr.region1 = 1u << kRetShift1;
    sr.region1_M = ght::make_fastmod(sr.region1).M;
    sr.fine_shift = ght::kGFindWindowLog2;
    sr.subs_log2 = kRetShift1 - ght::kGFindWindowLog2;
    sr.groups = g.rgroups;
    ght::GroupExtras xr;
    xr.ident = true;
    e = ght::launch_subgroup(t->view(), l1k, l1p, (uint64_t)g.rgroups << kRetShift1, sr, g.rbins, cur_r2,
                             1u << ght::kGFindWindowLog2, l2k, l2p, s, xr);
  }
  if (e == cudaSuccess) e = ght::launch_window_write(l2k, l2p, cur_r2, n, out, s);
  if (pool_buf) cudaFreeAsync(pool_buf, s);
  return e;
}

// allow_grouped = false: the per-query find even where the table asks for
// the grouped one (whose scratch comes from an allocator).
cudaError_t launch_find(const ght_table *t, const uint32_t *q, uint32_t *out, uint64_t n,
                        bool allow_grouped = true) {
  t->last_find_grouped = false;
  if (allow_grouped && wants_grouped_find(t, n)) {
    const cudaError_t eg = launch_find_grouped(t, q, out, n);
    if (eg != cudaErrorNotSupported) {
      t->last_find_grouped = eg == cudaSuccess;
      return eg;
    }
  }
  const ght::TableView tv = t->view();
  if (t->shape.scheme == GHT_BCHT) {
    const ght::LaunchOpts o = t->find_opts();
    return o.async_find ? ght::launch_find_bcht_async(t->shape.b, tv, q, out, n, o, t->stream)
                        : ght::launch_find_bcht(t->shape.b, tv, q, out, n, o, t->stream);
  }
  if (t->shape.scheme == GHT_BCHT_SET) {
    const ght::LaunchOpts o = t->find_opts();
    return o.async_find ? ght::launch_find_set_async(tv, q, out, n, o, t->stream)
                        : ght::launch_find_set(tv, q, out, n, o, t->stream);
  }
  const ght::LaunchOpts o = t->find_opts();
  if (o.async_find) return ght::launch_find_bcht_async(t->shape.b, tv, q, out, n, o, t->stream, false);
  return ght::launch_find_other(t->shape.scheme, t->shape.b, tv, q, out, n, o, t->stream);
}

// Read the control block after the stream's work; bounded wait.
int read_ctrl(const ght_table *t) {
  cudaError_t e = cudaMemcpyAsync(t->h_ctrl, t->ctrl, kCtrlBytes, cudaMemcpyDeviceToHost, t->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading the control block");
  e = cudaEventRecord(t->done, t->stream);
  if (e != cudaSuccess) return cuda_fail(e, "recording an event");
  return wait_event(t->done);
}

// The device address of page-locked host memory (allocated or registered
// with the CUDA runtime), or false for memory the device cannot address.
bool device_view(const void *h, const void **d) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
  *d = a.devicePointer;
  return true;
}

// One build from device-resident keys: fill, (group,) insert, status; retry
// with the next attempt's constants on failure.
int build_device(ght_table *t, const uint32_t *k, const uint32_t *v, uint64_t n, uint32_t first_attempt,
                 bool input_order = false) {
  t->built = false;
  t->n_stored = 0;
  bool ranked = !input_order && wants_ranked(t, n);
  bool grouped = !input_order && wants_grouping(t, n);
  if (grouped && ((reinterpret_cast<uintptr_t>(k) | reinterpret_cast<uintptr_t>(v ? v : k)) & 15u)) {
    // the grouping copies 16-byte pieces of the input: unaligned arrays build ungrouped
    grouped = false;
    ranked = t->shape.ranked_build > 0;
  }
  void *pool_buf = nullptr;
  char *scr = nullptr;
  if (ranked || grouped) {
    scr = build_scratch(t, build_scratch_need(t, n), &pool_buf);
    if (!scr) ranked = grouped = false;  // no scratch: the cuckoo insert of every key in input order
  }
  int shift = 0;
  uint32_t groups = 1;
  group_shape(t->shape.m, &shift, &groups);
  // grouped pairs in per-group regions when placed by rank (no count pass)
  const uint64_t glen = grouped ? grouped_len(t, n) : n;
  uint32_t region = grouped && ranked && glen != n ? group_region(n, groups) : 0u;
  uint32_t *counts = reinterpret_cast<uint32_t *>(scr);
  uint32_t *cursors = counts + ght::kMaxGroups;
  uint32_t *gk = reinterpret_cast<uint32_t *>(scr + 2ull * ght::kMaxGroups * sizeof(uint32_t));
  uint32_t *gv = gk + align256(glen * sizeof(uint32_t)) / sizeof(uint32_t);
  // scratch layout: [grouping: counts, cursors, keys, values][ranked placement]
  const ght::PlaceBuffers pb =
      ranked ? place_buffers(scr + (grouped ? group_scratch_bytes(glen) : 0), t->shape.m, n) : ght::PlaceBuffers();
  // second-level split and block placement: [sub-group keys, values, cursors] after the placement scratch
  SubShape sub;
  bool two_level = region && sub_shape(t->shape, n, shift, region, &sub) && sub_scratch_bytes(t, n) > 0;
  uint32_t *sk = nullptr, *sv = nullptr, *scur = nullptr;
  if (two_level) {
    char *p = scr + group_scratch_bytes(glen) + place_scratch_bytes(t->shape.m, n);
    const uint64_t arr = align256((uint64_t)sub.bins * sub.region2 * sizeof(uint32_t));
    sk = reinterpret_cast<uint32_t *>(p);
    sv = reinterpret_cast<uint32_t *>(p + arr);
    scur = reinterpret_cast<uint32_t *>(p + 2 * arr);
  }
  int rc = fail(GHT_ERR_BUILD_FAILED, "build failed in %u attempts (chain bound or full buckets)",
                t->shape.max_attempts);
  for (uint32_t attempt = first_attempt; attempt < t->shape.max_attempts; ++attempt) {
    t->derive(attempt);
    const ght::TableView tv = t->view();
    cudaEventRecord(t->tev[0], t->stream);
    // the block placement writes every table line: only the control block is reset
    cudaError_t e = two_level ? cudaMemsetAsync(t->ctrl, 0, kCtrlBytes, t->stream) : ght::launch_fill(tv, t->words(), t->stream);
    if (e != cudaSuccess) { rc = cuda_fail(e, "launching fill"); break; }
    cudaEventRecord(t->tev[1], t->stream);
    const uint32_t *ik = k, *iv = v;  // what the cuckoo insert takes
    uint64_t in = n;
    bool this_ranked = false;
    t->place_overflow = 0;
    if (grouped) {
      e = ght::launch_group(tv, k, v ? v : k, n, shift, groups, counts, cursors, gk, gv, t->stream, region);
      if (e == cudaSuccess && two_level) {
        cudaEventRecord(t->tev[9], t->stream);
        ght::SubSplit ss;
        ss.ends1 = cursors;
        ss.region1 = region;
        ss.region1_M = ght::make_fastmod(region).M;
        ss.fine_shift = sub.fine_shift;
        ss.subs_log2 = sub.subs_log2;
        ss.groups = groups;
        e = ght::launch_subgroup(tv, gk, gv, (uint64_t)groups * region, ss, sub.bins, scur, sub.region2, sk, sv,
                                 t->stream);
      }
      if (e != cudaSuccess) { rc = cuda_fail(e, "launching grouping"); break; }
      ik = gk;
      iv = gv;
      cudaEventRecord(t->tev[6], t->stream);
    }
    if (ranked) {
      // phase 1: ranked first-choice placement (of the grouped pairs, when
      // grouped: the stores then stay in a few MB of the table, whose lines
      // fill up in L2); its overflow goes to phase 2
      ght::PlaceBuffers pa = pb;
      if (region) {  // the pairs of group g are [g * region, cursors[g])
        pa.ends = cursors;
        pa.region = region;
        pa.region_M = ght::make_fastmod(region).M;
      }
      if (two_level) {
        e = ght::launch_block_place(t->shape.b, t->shape.scheme == GHT_BCHT_SET, tv, sk, sv, scur, sub.region2,
                                    sub.bins, sub.fine_shift, pb, t->shape.count_probes != 0, t->stream);
      } else if ((e = cudaMemsetAsync(pb.counters, 0, t->shape.m * sizeof(uint32_t), t->stream)) == cudaSuccess) {
        e = launch_place(t, ik, iv, region ? (uint64_t)groups * region : n, pa);
      }
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "launching the ranked placement");
        break;
      }
      cudaEventRecord(t->tev[2], t->stream);
      if ((rc = read_ctrl(t)) != GHT_OK) break;
      if (region && ((t->h_ctrl->status & ght::kStatusGroupRegion) || t->h_ctrl->reserved[0] > pb.cap)) {
        // a group outgrew its region, or the overflow outgrew its list: this
        // attempt again with exact group offsets and the filled table of the
        // global-counter placement (its fallback reads dense arrays)
        region = 0;
        two_level = false;
        --attempt;
        continue;
      }
      if (t->h_ctrl->status & ght::kStatusSentinel) { rc = fail(GHT_ERR_SENTINEL_KEY, "an input key is the sentinel 0xFFFFFFFF"); break; }
      const uint64_t ovf = t->h_ctrl->reserved[0];
      t->place_overflow = ovf;
      if (ovf <= pb.cap) {
        this_ranked = true;
        ik = pb.ovf_k;
        iv = pb.ovf_v;
        in = ovf;
      } else {
        // too many keys share first-choice buckets for the overflow list:
        // start over and insert every key (grouped, if it was) with the cuckoo insert
        cudaEventRecord(t->tev[0], t->stream);
        if ((e = ght::launch_fill(tv, t->words(), t->stream)) != cudaSuccess) { rc = cuda_fail(e, "launching fill"); break; }
        cudaEventRecord(t->tev[1], t->stream);
        cudaEventRecord(t->tev[2], t->stream);
      }
    } else {
      cudaEventRecord(t->tev[2], t->stream);
    }
    if (in > 0) {
      e = launch_insert(t, ik, iv, in, this_ranked);
      if (e != cudaSuccess) { rc = cuda_fail(e, "launching insert"); break; }
    }
    cudaEventRecord(t->tev[3], t->stream);
    t->timed_build = true;
    t->last_grouped = grouped;
    t->last_split = this_ranked && two_level;
    t->last_ranked = this_ranked;
    rc = read_ctrl(t);
    if (rc) break;
    const uint32_t st = t->h_ctrl->status;
    t->attempts = attempt + 1;
    t->insert_probes = t->h_ctrl->insert_probes;
    t->insert_retries = t->h_ctrl->insert_retries;
    t->insert_evictions = t->h_ctrl->insert_evictions;
    t->longest_chain = t->h_ctrl->longest_chain;
    if (st == 0u) {
      t->built = true;
      t->n_stored = n;
      rc = GHT_OK;
      break;
    }
    if (st & ght::kStatusSentinel) { rc = fail(GHT_ERR_SENTINEL_KEY, "an input key is the sentinel 0xFFFFFFFF"); break; }
    if (st & ght::kStatusTimeout) { rc = fail(GHT_ERR_DEVICE_TIMEOUT, "a key exceeded the per-key step bound"); break; }
    if (st & ght::kStatusCorrupt) { rc = fail(GHT_ERR_CUDA, "table corrupt: an evicted key did not hash to its bucket"); break; }
    rc = fail(GHT_ERR_BUILD_FAILED, "build failed in %u attempts (chain bound or full buckets)", t->shape.max_attempts);
  }
  if (pool_buf) cudaFreeAsync(pool_buf, t->stream);
  return rc;
}

// Chunks of a find's host<->device pipeline: from 2^20 queries doubling up
// to 2^25 at the front and halving back down to 2^20 at the end, so the
// copy-in before the first find and the copy-out after the last are short
// and the middle runs few, long launches.
constexpr uint64_t kChunkFirst = 1ull << 20, kChunkCap = 1ull << 25;

std::vector<uint64_t> find_chunks(uint64_t n) {
  std::vector<uint64_t> head, mid;
  uint64_t left = n;
  for (uint64_t c = kChunkFirst; c < kChunkCap && left >= 2 * c; c *= 2) {
    head.push_back(c);
    left -= 2 * c;
  }
  while (left > 0) {
    const uint64_t c = std::min(left, kChunkCap);
    mid.push_back(c);
    left -= c;
  }
  std::vector<uint64_t> plan(head);
  plan.insert(plan.end(), mid.begin(), mid.end());
  plan.insert(plan.end(), head.rbegin(), head.rend());
  return plan;
}
constexpr uint64_t kBuildChunk = 1ull << 25;  // pairs per chunk of a host-buffer build (fewer insert launch tails)

// check_duplicates: after a successful build from device keys, no key may be
// stored twice; a duplicate leaves the table unbuilt.
int check_duplicates(ght_table *t, const uint32_t *d_keys, uint64_t n) {
  if (!t->shape.check_dups || !t->built || n == 0) return GHT_OK;
  const cudaError_t e = ght::launch_dup_check(t->view(), t->shape.b, t->shape.scheme == GHT_BCHT_SET, d_keys, n,
                                              t->stream);
  if (e != cudaSuccess) return cuda_fail(e, "launching the duplicate check");
  const int rc = read_ctrl(t);
  if (rc) return rc;
  if (t->h_ctrl->status & ght::kStatusDuplicate) {
    t->built = false;
    t->n_stored = 0;
    return fail(GHT_ERR_DUPLICATE_KEY, "an input key is stored more than once (duplicate keys)");
  }
  return GHT_OK;
}

}  // namespace

bool ght::table_descriptor(const ght_table *t, ght::BatchTable *out) {
  if (!t || !t->built || t->shape.scheme != GHT_BCHT || t->shape.b != 16 || t->shape.h != 3) return false;
  memset(out, 0, sizeof *out);
  out->slots = t->slots;
  out->m = (uint32_t)t->shape.m;
  out->mod = ght::make_fastmod(out->m);
  for (int i = 0; i < 4; ++i) {
    out->a[i] = t->a[i];
    out->c[i] = t->c[i];
  }
  return true;
}

extern "C" {

const char *ght_version(void) { return "ght 0.1 (sm_103a)"; }

const char *ght_last_error(void) { return ght::host::last_error(); }

int ght_default_config(int scheme, ght_config *out) {
  if (!out) return fail(GHT_ERR_INVALID_ARG, "out is NULL");
  return default_config(scheme, out);
}

uint64_t ght_table_bytes(int scheme, uint64_t capacity, double load_factor, const ght_config *cfg) {
  Shape s;
  if (resolve(scheme, capacity, load_factor, cfg, &s)) return 0;
  return bytes_of(s);
}

ght_table *ght_create_ex(int scheme, uint64_t capacity, double load_factor, uint64_t seed,
                         const ght_config *cfg, void *d_storage, uint64_t storage_bytes) {
  Shape s;
  if (resolve(scheme, capacity, load_factor, cfg, &s)) return nullptr;
  const uint64_t need = bytes_of(s);
  if (d_storage) {
    if (storage_bytes < need) {
      fail(GHT_ERR_INVALID_ARG, "storage of %llu bytes, need %llu", (unsigned long long)storage_bytes,
           (unsigned long long)need);
      return nullptr;
    }
    if (((uintptr_t)d_storage & 255u) != 0u) {
      fail(GHT_ERR_INVALID_ARG, "storage must be 256-byte aligned");
      return nullptr;
    }
  }
  int dev = 0;
  if (const cudaError_t e = cudaGetDevice(&dev); e != cudaSuccess) {
    cuda_fail(e, "querying the current device");
    return nullptr;
  }
  ght_table *t = new (std::nothrow) ght_table();
  if (!t) {
    fail(GHT_ERR_OOM, "host allocation failed");
    return nullptr;
  }
  t->shape = s;
  t->device = dev;
  t->capacity = capacity;
  t->lf = load_factor;
  t->seed = seed;
  t->storage_bytes = need;
  if (d_storage) {
    t->storage = d_storage;
  } else {
    const cudaError_t e = cudaMalloc(&t->storage, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete t;
      fail(GHT_ERR_OOM, "cudaMalloc of %llu bytes: %s", (unsigned long long)need, cudaGetErrorString(e));
      return nullptr;
    }
    t->owns_storage = true;
  }
  t->ctrl = reinterpret_cast<ght::Ctrl *>(t->storage);
  t->slots = reinterpret_cast<uint64_t *>(reinterpret_cast<char *>(t->storage) + kCtrlBytes);
  cudaError_t e = cudaMallocHost(reinterpret_cast<void **>(&t->h_ctrl), kCtrlBytes);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->done, cudaEventDisableTiming);
  for (int i = 0; i < 10 && e == cudaSuccess; ++i) e = cudaEventCreate(&t->tev[i]);
  if (e != cudaSuccess) {
    cuda_fail(e, "creating table resources");
    ght_destroy(t);
    return nullptr;
  }
  memset(t->h_ctrl, 0, kCtrlBytes);
  t->derive(0);
  noalloc_setup(dev);  // reserves the allocation-free find's staging array on this device
  return t;
}

ght_table *ght_create(int scheme, uint64_t capacity, double load_factor, uint64_t seed) {
  return ght_create_ex(scheme, capacity, load_factor, seed, nullptr, nullptr, 0);
}

int ght_set_stream(ght_table *t, void *cuda_stream) {
  if (!t) return fail(GHT_ERR_INVALID_ARG, "table is NULL");
  t->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  return GHT_OK;
}

int ght_build(ght_table *t, const uint32_t *d_keys, const uint32_t *d_values, uint64_t n) {
  if (!t) return fail(GHT_ERR_INVALID_ARG, "table is NULL");
  if (n > t->capacity) return fail(GHT_ERR_CAPACITY, "n = %llu exceeds capacity %llu", (unsigned long long)n,
                                   (unsigned long long)t->capacity);
  if (n > 0 && (!d_keys || (!d_values && t->shape.scheme != GHT_BCHT_SET)))
    return fail(GHT_ERR_INVALID_ARG, "keys or values is NULL");
  const int rc = build_device(t, d_keys, d_values, n, 0);
  return rc == GHT_OK ? check_duplicates(t, d_keys, n) : rc;
}

int ght_find(const ght_table *t, const uint32_t *d_queries, uint32_t *d_out, uint64_t n) {
  if (!t) return fail(GHT_ERR_INVALID_ARG, "table is NULL");
  if (!t->built) return fail(GHT_ERR_NOT_BUILT, "table has no successful build");
  if (n == 0) return GHT_OK;
  if (!d_queries || !d_out) return fail(GHT_ERR_INVALID_ARG, "queries or out is NULL");
  cudaEventRecord(t->tev[4], t->stream);
  const cudaError_t e = launch_find(t, d_queries, d_out, n);
  if (e != cudaSuccess) return cuda_fail(e, "launching find");
  cudaEventRecord(t->tev[5], t->stream);
  t->timed_find = true;
  return GHT_OK;
}

int ght_build_host(ght_table *t, const uint32_t *h_keys, const uint32_t *h_values, uint64_t n) {
  if (!t) return fail(GHT_ERR_INVALID_ARG, "table is NULL");
  if (n > t->capacity) return fail(GHT_ERR_CAPACITY, "n = %llu exceeds capacity %llu", (unsigned long long)n,
                                   (unsigned long long)t->capacity);
  if (n > 0 && (!h_keys || (!h_values && t->shape.scheme != GHT_BCHT_SET)))
    return fail(GHT_ERR_INVALID_ARG, "keys or values is NULL");
  if (n == 0) return build_device(t, nullptr, nullptr, 0, 0);
  if (!h_values) h_values = h_keys;  // a set ignores values
  // Pinned host arrays the device can address: the input-order insert reads
  // them in place, in one launch (the host link's rate is the same for the
  // kernel's reads as for copies, and the copies' chunk pipeline -- its first
  // chunk's wait and one insert launch tail per chunk -- goes away). A
  // requested grouped or two-phase build still stages the pairs.
  const void *dk_in = nullptr, *dv_in = nullptr;
  if (t->shape.group_build <= 0 && t->shape.ranked_build <= 0 && device_view(h_keys, &dk_in) &&
      device_view(h_values, &dv_in)) {
    t->timed_h2d = false;  // no copies: the insert's own loads cross the host link
    int rc = build_device(t, static_cast<const uint32_t *>(dk_in), static_cast<const uint32_t *>(dv_in), n, 0, true);
    if (rc == GHT_OK) rc = check_duplicates(t, static_cast<const uint32_t *>(dk_in), n);
    return rc;
  }
  // Stage the pairs on the device (the library pool keeps the block for the
  // next call). The first attempt works on each chunk as soon as it has
  // landed, overlapping the copies with the ranked placement (two-phase
  // build) or with the inserts (input-order build); later attempts, and
  // grouped builds, run from the staged copy.
  void *buf = nullptr;
  const uint64_t arr = (n * sizeof(uint32_t) + 255ull) & ~255ull;
  cudaError_t e = pool_alloc(&buf, 2 * arr, t->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(GHT_ERR_OOM, "staging allocation: %s", cudaGetErrorString(e));
  }
  uint32_t *d_k = static_cast<uint32_t *>(buf), *d_v = d_k + arr / sizeof(uint32_t);
  int rc = GHT_OK;
  // From host buffers the input-order build overlaps the copies with the
  // inserts chunk by chunk, which a grouped build cannot (the grouping needs
  // every pair); so here grouping and ranked placement run only on request.
  const bool ranked_wanted = t->shape.ranked_build > 0 && wants_ranked(t, n);
  if (t->shape.group_build > 0 && wants_grouping(t, n)) {
    cudaEventRecord(t->tev[7], t->stream);
    if ((e = cudaMemcpyAsync(d_k, h_keys, n * 4, cudaMemcpyHostToDevice, t->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_v, h_values, n * 4, cudaMemcpyHostToDevice, t->stream)) != cudaSuccess)
      rc = cuda_fail(e, "staging keys");
    cudaEventRecord(t->tev[8], t->stream);
    t->timed_h2d = true;
    t->h2d_bytes = 8 * n;
    if (rc == GHT_OK) rc = build_device(t, d_k, d_v, n, 0);
  } else {
    void *place_pool = nullptr;
    char *scr = ranked_wanted ? build_scratch(t, place_scratch_bytes(t->shape.m, n), &place_pool) : nullptr;
    const bool ranked = scr != nullptr;
    const ght::PlaceBuffers pb = ranked ? place_buffers(scr, t->shape.m, n) : ght::PlaceBuffers();
    cudaStream_t copy = nullptr;
    cudaEvent_t landed[2] = {nullptr, nullptr};
    if ((e = cudaStreamCreateWithFlags(&copy, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&landed[0], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&landed[1], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventRecord(landed[0], t->stream)) != cudaSuccess ||  // staging block allocated
        (e = cudaStreamWaitEvent(copy, landed[0], 0)) != cudaSuccess)
      rc = cuda_fail(e, "creating the copy pipeline");
    bool retry_staged = false;   // build again from the staged copy, first attempt
    bool retry_next = false;     // build again from the staged copy, next attempt
    if (rc == GHT_OK) {
      t->built = false;
      t->n_stored = 0;
      t->place_overflow = 0;
      t->derive(0);
      const ght::TableView tv = t->view();
      cudaEventRecord(t->tev[0], t->stream);
      if ((e = ght::launch_fill(tv, t->words(), t->stream)) != cudaSuccess)
        rc = cuda_fail(e, "launching fill");
      if (rc == GHT_OK && ranked &&
          (e = cudaMemsetAsync(pb.counters, 0, t->shape.m * sizeof(uint32_t), t->stream)) != cudaSuccess)
        rc = cuda_fail(e, "clearing the arrival counters");
      cudaEventRecord(t->tev[1], t->stream);
      if (!ranked) cudaEventRecord(t->tev[2], t->stream);
      cudaEventRecord(t->tev[7], copy);
      for (uint64_t off = 0, i = 0; rc == GHT_OK && off < n; off += kBuildChunk, ++i) {
        const uint64_t len = std::min(kBuildChunk, n - off);
        cudaEvent_t ev = landed[i & 1];
        if ((e = cudaMemcpyAsync(d_k + off, h_keys + off, len * 4, cudaMemcpyHostToDevice, copy)) != cudaSuccess ||
            (e = cudaMemcpyAsync(d_v + off, h_values + off, len * 4, cudaMemcpyHostToDevice, copy)) != cudaSuccess ||
            (e = cudaEventRecord(ev, copy)) != cudaSuccess || (e = cudaStreamWaitEvent(t->stream, ev, 0)) != cudaSuccess) {
          rc = cuda_fail(e, "staging keys");
          break;
        }
        if (ranked) {
          // each chunk's placement claims its tiles from zero; the overflow count accumulates
          if ((e = cudaMemsetAsync(&t->ctrl->reserved[1], 0, sizeof t->ctrl->reserved[1], t->stream)) != cudaSuccess ||
              (e = launch_place(t, d_k + off, d_v + off, len, pb)) != cudaSuccess)
            rc = cuda_fail(e, "launching the ranked placement");
        } else if ((e = cudaMemsetAsync(&t->ctrl->work_cursor, 0, sizeof t->ctrl->work_cursor, t->stream)) != cudaSuccess ||
                   (e = launch_insert(t, d_k + off, d_v + off, len)) != cudaSuccess) {
          rc = cuda_fail(e, "launching insert");  // each chunk's insert starts its own claims at zero
        }
      }
      cudaEventRecord(t->tev[8], copy);
      t->timed_h2d = true;
      t->h2d_bytes = 8 * n;
      if (rc == GHT_OK && ranked) {
        // phase 2: the cuckoo insert of the keys whose first-choice bucket was full
        cudaEventRecord(t->tev[2], t->stream);
        rc = read_ctrl(t);
        if (rc == GHT_OK && !(t->h_ctrl->status & ght::kStatusSentinel)) {
          const uint64_t ovf = t->h_ctrl->reserved[0];
          t->place_overflow = ovf;
          if (ovf > pb.cap) retry_staged = true;  // overflow list too small: build_device falls back
          else if (ovf > 0 && (e = launch_insert(t, pb.ovf_k, pb.ovf_v, ovf, true)) != cudaSuccess)
            rc = cuda_fail(e, "launching insert");
        }
      }
      cudaEventRecord(t->tev[3], t->stream);
      t->timed_build = true;
      t->last_grouped = false;
      t->last_split = false;
      t->last_ranked = ranked && !retry_staged;
      if (rc == GHT_OK && !retry_staged) rc = read_ctrl(t);
      if (rc == GHT_OK && !retry_staged) {
        const uint32_t st = t->h_ctrl->status;
        t->attempts = 1;
        t->insert_probes = t->h_ctrl->insert_probes;
        t->insert_retries = t->h_ctrl->insert_retries;
        t->insert_evictions = t->h_ctrl->insert_evictions;
        t->longest_chain = t->h_ctrl->longest_chain;
        if (st == 0u) {
          t->built = true;
          t->n_stored = n;
        } else if (st & ght::kStatusSentinel) {
          rc = fail(GHT_ERR_SENTINEL_KEY, "an input key is the sentinel 0xFFFFFFFF");
        } else if (st & ght::kStatusTimeout) {
          rc = fail(GHT_ERR_DEVICE_TIMEOUT, "a key exceeded the per-key step bound");
        } else if (st & ght::kStatusCorrupt) {
          rc = fail(GHT_ERR_CUDA, "table corrupt: an evicted key did not hash to its bucket");
        } else {
          retry_next = true;
        }
      }
    }
    if (copy) cudaStreamSynchronize(copy);
    if (landed[0]) cudaEventDestroy(landed[0]);
    if (landed[1]) cudaEventDestroy(landed[1]);
    if (copy) cudaStreamDestroy(copy);
    if (place_pool) cudaFreeAsync(place_pool, t->stream);
    // the staged copy is complete: the table stream waited on every chunk
    if (rc == GHT_OK && (retry_staged || retry_next)) rc = build_device(t, d_k, d_v, n, retry_next ? 1 : 0);
  }
  if (rc == GHT_OK) rc = check_duplicates(t, d_k, n);  // on the staged copy, before it is freed
  cudaFreeAsync(buf, t->stream);
  if (rc == GHT_OK) {
    e = cudaEventRecord(t->done, t->stream);
    rc = e == cudaSuccess ? wait_event(t->done) : cuda_fail(e, "recording an event");
  }
  return rc;
}

int ght_find_host(const ght_table *t, const uint32_t *h_queries, uint32_t *h_out, uint64_t n) {
  if (!t) return fail(GHT_ERR_INVALID_ARG, "table is NULL");
  if (!t->built) return fail(GHT_ERR_NOT_BUILT, "table has no successful build");
  if (n == 0) return GHT_OK;
  if (!h_queries || !h_out) return fail(GHT_ERR_INVALID_ARG, "queries or out is NULL");
  // Three-stage pipeline over chunks: H2D on one copy stream, find on the
  // table stream, D2H on a second copy stream (both link directions busy).
  uint32_t *d_buf = nullptr;
  cudaStream_t up = nullptr, down = nullptr;
  const std::vector<uint64_t> chunks = find_chunks(n);
  cudaEvent_t evs[8] = {};
  int rc = GHT_OK;
  bool h2d_started = false;  // the copy-span start event was recorded in this call
  cudaError_t e = pool_alloc(reinterpret_cast<void **>(&d_buf), 2 * n * sizeof(uint32_t), t->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(GHT_ERR_OOM, "staging allocation: %s", cudaGetErrorString(e));
  }
  uint32_t *d_q = d_buf, *d_o = d_buf + n;
  if ((e = cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking)) != cudaSuccess)
    rc = cuda_fail(e, "creating pipeline streams");
  for (int i = 0; rc == GHT_OK && i < 8; ++i)
    if ((e = cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming)) != cudaSuccess) rc = cuda_fail(e, "creating events");
  if (rc == GHT_OK) {
    if ((e = cudaEventRecord(evs[0], t->stream)) != cudaSuccess || (e = cudaStreamWaitEvent(up, evs[0], 0)) != cudaSuccess)
      rc = cuda_fail(e, "ordering the staging copy");
    h2d_started = rc == GHT_OK && cudaEventRecord(t->tev[7], up) == cudaSuccess;
  }
  // events 0..3: "chunk landed" ring; 4..7: "chunk answered" ring. Reusing an
  // event is safe because each stream consumes them in order.
  uint64_t off = 0;
  for (uint64_t i = 0; rc == GHT_OK && i < chunks.size(); off += chunks[i], ++i) {
    const uint64_t len = chunks[i];
    cudaEvent_t in = evs[i & 3], fin = evs[4 + (i & 3)];
    if ((e = cudaMemcpyAsync(d_q + off, h_queries + off, len * 4, cudaMemcpyHostToDevice, up)) != cudaSuccess ||
        (e = cudaEventRecord(in, up)) != cudaSuccess || (e = cudaStreamWaitEvent(t->stream, in, 0)) != cudaSuccess) {
      rc = cuda_fail(e, "staging queries");
      break;
    }
    if ((e = launch_find(t, d_q + off, d_o + off, len)) != cudaSuccess) {
      rc = cuda_fail(e, "launching find");
      break;
    }
    if ((e = cudaEventRecord(fin, t->stream)) != cudaSuccess || (e = cudaStreamWaitEvent(down, fin, 0)) != cudaSuccess ||
        (e = cudaMemcpyAsync(h_out + off, d_o + off, len * 4, cudaMemcpyDeviceToHost, down)) != cudaSuccess) {
      rc = cuda_fail(e, "returning results");
      break;
    }
  }
  if (h2d_started) {
    cudaEventRecord(t->tev[8], up);
    t->timed_h2d = true;
    t->h2d_bytes = 4 * n;
  }
  if (rc == GHT_OK) {
    // the table stream frees the buffer after the last read-back
    if ((e = cudaEventRecord(evs[0], down)) != cudaSuccess || (e = cudaStreamWaitEvent(t->stream, evs[0], 0)) != cudaSuccess)
      rc = cuda_fail(e, "joining the pipeline");
  }
  cudaFreeAsync(d_buf, t->stream);
  if (rc == GHT_OK) {
    e = cudaEventRecord(t->done, t->stream);
    rc = e == cudaSuccess ? wait_event(t->done) : cuda_fail(e, "recording an event");
  } else {
    cudaStreamSynchronize(up);
    cudaStreamSynchronize(down);
  }
  for (auto ev : evs)
    if (ev) cudaEventDestroy(ev);
  if (up) cudaStreamDestroy(up);
  if (down) cudaStreamDestroy(down);
  return rc;
}

uint64_t ght_build_scratch_bytes(const ght_table *t, uint64_t n) {
  if (!t) {
    fail(GHT_ERR_INVALID_ARG, "table is NULL");
    return 0;
  }
  return build_scratch_need(t, n);
}

uint64_t ght_find_scratch_bytes(const ght_table *t, uint64_t n) {
  if (!t) {
    fail(GHT_ERR_INVALID_ARG, "table is NULL");
    return 0;
  }
  GFindShape g;
  return wants_grouped_find(t, n) && gfind_shape(t, n, &g) ? gfind_scratch_bytes(g, n) : 0;
}

int ght_set_build_scratch(ght_table *t, void *d_scratch, uint64_t bytes) {
  if (!t) return fail(GHT_ERR_INVALID_ARG, "table is NULL");
  if (d_scratch && ((uintptr_t)d_scratch & 255u) != 0u) return fail(GHT_ERR_INVALID_ARG, "scratch must be 256-byte aligned");
  t->scratch = d_scratch;
  t->scratch_bytes = d_scratch ? bytes : 0;
  return GHT_OK;
}

int ght_stats(const ght_table *t, ght_stats_t *out) {
  if (!t || !out) return fail(GHT_ERR_INVALID_ARG, "table or out is NULL");
  memset(out, 0, sizeof *out);
  out->scheme = t->shape.scheme;
  out->bucket_size = t->shape.b;
  out->num_hashes = t->shape.h;
  out->threshold = t->shape.t;
  out->num_buckets = t->shape.m;
  out->num_slots = t->shape.m * (uint64_t)t->shape.b;
  out->capacity = t->capacity;
  out->n_stored = t->n_stored;
  out->load_factor = out->num_slots ? (double)t->n_stored / (double)out->num_slots : 0.0;
  out->attempts = t->attempts;
  out->max_chain = t->shape.max_chain;
  for (int i = 0; i < 4; ++i) {
    out->hash_a[i] = t->a[i];
    out->hash_c[i] = t->c[i];
  }
  out->table_bytes = t->storage_bytes;
  out->built = t->built ? 1 : 0;
  out->tile_lanes = t->shape.tile_lanes;
  out->keys_per_lane = t->shape.keys_per_lane;
  out->build_tile_lanes = t->shape.build_tile_lanes;
  out->build_keys_per_lane = t->shape.build_keys_per_lane;
  out->insert_probes = t->insert_probes;
  out->insert_retries = t->insert_retries;
  out->insert_evictions = t->insert_evictions;
  out->longest_chain = t->longest_chain;
  out->last_fill_ms = out->last_insert_ms = out->last_find_ms = -1.0;
  float ms = 0.f;
  out->last_group_ms = -1.0;
  out->last_build_grouped = t->last_grouped ? 1 : 0;
  out->last_build_split = t->last_split ? 1 : 0;
  out->slot_bytes = t->shape.slot_bytes;
  out->last_build_ranked = t->last_ranked ? 1 : 0;
  out->last_place_ms = -1.0;
  out->last_split_ms = -1.0;
  out->place_overflow = t->place_overflow;
  out->find_staged = t->shape.find_async;
  out->find_grouped = t->shape.find_grouped;
  out->last_find_grouped = t->last_find_grouped ? 1 : 0;
  if (t->timed_build && cudaEventQuery(t->tev[3]) == cudaSuccess) {
    if (cudaEventElapsedTime(&ms, t->tev[0], t->tev[1]) == cudaSuccess) out->last_fill_ms = ms;
    // between the fill and the cuckoo insert: the grouping and/or the ranked placement
    if (t->last_grouped && t->last_ranked) {
      if (t->last_split) {  // first level, then the second level's split
        if (cudaEventElapsedTime(&ms, t->tev[1], t->tev[9]) == cudaSuccess) out->last_group_ms = ms;
        if (cudaEventElapsedTime(&ms, t->tev[9], t->tev[6]) == cudaSuccess) out->last_split_ms = ms;
      } else if (cudaEventElapsedTime(&ms, t->tev[1], t->tev[6]) == cudaSuccess) {
        out->last_group_ms = ms;
      }
      if (cudaEventElapsedTime(&ms, t->tev[6], t->tev[2]) == cudaSuccess) out->last_place_ms = ms;
    } else if (cudaEventElapsedTime(&ms, t->tev[1], t->tev[2]) == cudaSuccess) {
      if (t->last_ranked) out->last_place_ms = ms;
      else if (t->last_grouped) out->last_group_ms = ms;
    }
    if (cudaEventElapsedTime(&ms, t->tev[2], t->tev[3]) == cudaSuccess) out->last_insert_ms = ms;
  }
  out->last_h2d_ms = -1.0;
  if (t->timed_h2d && cudaEventQuery(t->tev[8]) == cudaSuccess &&
      cudaEventElapsedTime(&ms, t->tev[7], t->tev[8]) == cudaSuccess) {
    out->last_h2d_ms = ms;
    out->last_h2d_bytes = t->h2d_bytes;
  }
  if (t->timed_find && cudaEventQuery(t->tev[5]) == cudaSuccess &&
      cudaEventElapsedTime(&ms, t->tev[4], t->tev[5]) == cudaSuccess)
    out->last_find_ms = ms;
  cudaGetLastError();
  if (t->shape.count_probes) {
    const int rc = read_ctrl(t);
    if (rc) return rc;
    out->find_probes = t->h_ctrl->find_probes;
    out->find_queries = t->h_ctrl->find_queries;
  }
  return GHT_OK;
}

int ght_reset_counters(ght_table *t) {
  if (!t) return fail(GHT_ERR_INVALID_ARG, "table is NULL");
  const cudaError_t e = cudaMemsetAsync(&t->ctrl->find_probes, 0, 2 * sizeof(unsigned long long), t->stream);
  return e == cudaSuccess ? GHT_OK : cuda_fail(e, "resetting counters");
}

int ght_export(const ght_table *t, uint64_t *h_slots, uint64_t n_slots) {
  if (!t || !h_slots) return fail(GHT_ERR_INVALID_ARG, "table or h_slots is NULL");
  const uint64_t words = t->words();
  if (n_slots < words) return fail(GHT_ERR_INVALID_ARG, "h_slots holds %llu words, need %llu",
                                   (unsigned long long)n_slots, (unsigned long long)words);
  cudaError_t e = cudaMemcpyAsync(h_slots, t->slots, words * 8ull, cudaMemcpyDeviceToHost, t->stream);
  if (e != cudaSuccess) return cuda_fail(e, "exporting slots");
  e = cudaEventRecord(t->done, t->stream);
  if (e != cudaSuccess) return cuda_fail(e, "recording an event");
  return wait_event(t->done);
}

int ght_hash_device(const ght_table *t, const uint32_t *d_keys, uint32_t *d_buckets, uint64_t n) {
  if (!t) return fail(GHT_ERR_INVALID_ARG, "table is NULL");
  if (n == 0) return GHT_OK;
  if (!d_keys || !d_buckets) return fail(GHT_ERR_INVALID_ARG, "keys or buckets is NULL");
  const cudaError_t e = ght::launch_hash(t->view(), d_keys, d_buckets, n, t->stream);
  return e == cudaSuccess ? GHT_OK : cuda_fail(e, "launching hash");
}

int ght_hash_host(uint32_t a, uint32_t c, uint32_t m, const uint32_t *h_keys, uint32_t *h_out, uint64_t n) {
  if (m == 0) return fail(GHT_ERR_INVALID_ARG, "m must be at least 1");
  if (n > 0 && (!h_keys || !h_out)) return fail(GHT_ERR_INVALID_ARG, "keys or out is NULL");
  ght::HashFamily hf;
  memset(&hf, 0, sizeof hf);
  hf.a[0] = a;
  hf.c[0] = c;
  hf.mod = ght::make_fastmod(m);
  for (uint64_t i = 0; i < n; ++i) h_out[i] = ght::bucket_of(hf, 0, h_keys[i]);
  return GHT_OK;
}

int ght_probe_lines(int mode, void *d_lines, uint64_t num_lines, uint64_t ops, uint32_t seed, void *cuda_stream) {
  if (mode < 0 || mode > 5) return fail(GHT_ERR_INVALID_ARG, "probe mode %d (0..5)", mode);
  if (!d_lines || (reinterpret_cast<uintptr_t>(d_lines) & 127u))
    return fail(GHT_ERR_INVALID_ARG, "lines must be a 128-byte aligned device pointer");
  if (num_lines == 0 || num_lines > 0xFFFFFFFFull) return fail(GHT_ERR_INVALID_ARG, "num_lines outside [1, 2^32-1]");
  if (ops == 0) return GHT_OK;
  const cudaError_t e =
      ght::launch_line_probe(mode, d_lines, num_lines, ops, seed, static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? GHT_OK : cuda_fail(e, "launching the line probe");
}

void ght_destroy(ght_table *t) {
  if (!t) return;
  if (t->owns_storage && t->storage) {
    cudaStreamSynchronize(t->stream);
    cudaFree(t->storage);
  }
  if (t->h_ctrl) cudaFreeHost(t->h_ctrl);
  if (t->done) cudaEventDestroy(t->done);
  for (auto ev : t->tev)
    if (ev) cudaEventDestroy(ev);
  delete t;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Host-buffer find without allocation (declared in ght.h), on the static
// staging array set up when the table was created.
extern "C" int ght_find_host_noalloc(const ght_table *t, const uint32_t *h_queries, uint32_t *h_out,
                                     uint64_t n) {
  if (!t) return fail(GHT_ERR_INVALID_ARG, "table is NULL");
  if (!t->built) return fail(GHT_ERR_NOT_BUILT, "table has no successful build");
  if (n > GHT_NOALLOC_MAX_QUERIES)
    return fail(GHT_ERR_CAPACITY, "n = %llu exceeds the %u queries the static staging array holds",
                (unsigned long long)n, GHT_NOALLOC_MAX_QUERIES);
  if (n == 0) return GHT_OK;
  if (!h_queries || !h_out) return fail(GHT_ERR_INVALID_ARG, "queries or out is NULL");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "querying the current device");
  if (dev != t->device)
    return fail(GHT_ERR_INVALID_ARG, "device %d is current but the table lives on device %d", dev, t->device);
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(GHT_ERR_INVALID_ARG, "device %d out of range", dev);
  uint32_t *base = nullptr;
  cudaEvent_t pending = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocDevice &d = g_noalloc[dev];
    if (!d.base) return fail(GHT_ERR_CUDA, "the static staging array could not be set up on device %d", dev);
    if (d.busy) {
      const cudaError_t q = cudaEventQuery(d.pending);
      if (q == cudaErrorNotReady)
        return fail(GHT_ERR_DEVICE_TIMEOUT, "an earlier call that timed out still uses the staging array");
      if (q != cudaSuccess) return cuda_fail(q, "querying the earlier call");
      d.busy = false;
    }
    base = d.base;
    pending = d.pending;
  }
  uint32_t *d_q = base, *d_o = base + GHT_NOALLOC_MAX_QUERIES;
  e = cudaMemcpyAsync(d_q, h_queries, n * sizeof(uint32_t), cudaMemcpyHostToDevice, t->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copying queries to the staging array");
  e = launch_find(t, d_q, d_o, n, false);  // the per-query find: no scratch
  if (e != cudaSuccess) return cuda_fail(e, "launching find");
  e = cudaMemcpyAsync(h_out, d_o, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, t->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copying results back");
  e = cudaEventRecord(t->done, t->stream);
  if (e != cudaSuccess) return cuda_fail(e, "recording an event");
  const int rc = wait_event(t->done);
  if (rc == GHT_ERR_DEVICE_TIMEOUT) {
    // the copies may still run: later calls on this device wait for them
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (cudaEventRecord(pending, t->stream) == cudaSuccess) g_noalloc[dev].busy = true;
    cudaGetLastError();
    return fail(GHT_ERR_DEVICE_TIMEOUT, "the find did not finish in time; h_out may still be written");
  }
  return rc;
}
