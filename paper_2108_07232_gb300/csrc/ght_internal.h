// ght_internal.h -- launch layer shared by the host API translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <unordered_map>

#include "ght_device.cuh"

namespace ght {

// Launch shape of one kernel: lanes per bucket tile, keys each lane keeps
// in flight, and the grid (0 = as many blocks as are resident at once).
struct LaunchOpts {
  int tile_lanes = 8;
  int keys_per_lane = 2;
  int blocks_per_sm = 0;
  bool count = false;    // probe counters
  bool dynamic = false;  // build: warps claim 32-pair chunks from a global cursor
  bool async_find = false;  // find: bucket parts staged in shared memory (BCHT, b = 16, 4-lane tiles)
};

constexpr uint32_t kMaxGroups = 4096;

constexpr int kThreads = 256;

// Grid for a persistent-style launch: at most as many blocks as are resident
// at once (SMs x blocks per SM), never more than the work needs. SM count and
// occupancy are cached per device.
template <typename K>
inline cudaError_t grid_for(K kernel, uint64_t n, int blocks_per_sm, int *blocks_out) {
  struct PerDevice {
    int sms = 0;
    std::unordered_map<const void *, int> occ;  // per kernel: resident blocks per SM
  };
  static std::mutex mu;
  static std::unordered_map<int, PerDevice> devices;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  PerDevice &d = devices[dev];
  if (d.sms == 0 && (e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  int per_sm = blocks_per_sm;
  if (per_sm <= 0) {
    auto it = d.occ.find((const void *)kernel);
    if (it == d.occ.end()) {
      int nb = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kThreads, 0);
      if (e != cudaSuccess) return e;
      it = d.occ.emplace((const void *)kernel, nb > 0 ? nb : 1).first;
    }
    per_sm = it->second;
  }
  const uint64_t want = (n + kThreads - 1) / kThreads;
  const uint64_t cap = (uint64_t)d.sms * (uint64_t)per_sm;
  *blocks_out = (int)(want < cap ? (want > 0 ? want : 1) : cap);
  return cudaSuccess;
}

// The same for a kernel with `threads` per block and `smem` bytes of dynamic
// shared memory; raises the kernel's dynamic shared-memory limit on the
// current device to `smem` when it is below. Attribute, SM count and
// occupancy are cached per device (the attribute is a per-device setting).
template <typename K>
inline cudaError_t grid_for_smem(K kernel, int threads, size_t smem, uint64_t n, int blocks_per_sm, int *blocks_out) {
  struct PerDevice {
    int sms = 0;
    std::unordered_map<const void *, size_t> limit;                          // per kernel: limit set so far
    std::unordered_map<const void *, std::unordered_map<size_t, int>> occ;  // per kernel and size
  };
  static std::mutex mu;
  static std::unordered_map<int, PerDevice> devices;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  PerDevice &d = devices[dev];
  if (d.sms == 0 && (e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const void *key = (const void *)kernel;
  if (smem > 48 * 1024 && d.limit[key] < smem) {
    if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    d.limit[key] = smem;
  }
  auto &by_size = d.occ[key];
  auto it = by_size.find(smem);
  if (it == by_size.end()) {
    int nb = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem)) != cudaSuccess) return e;
    it = by_size.emplace(smem, nb > 0 ? nb : 1).first;
  }
  const int sms = d.sms;
  int per_sm = it->second;
  if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
  const uint64_t want = (n + threads - 1) / threads;
  const uint64_t cap = (uint64_t)sms * (uint64_t)per_sm;
  *blocks_out = (int)(want < cap ? (want > 0 ? want : 1) : cap);
  return cudaSuccess;
}

// Warps of a grid share the input in contiguous slices of this many items.
inline uint64_t per_warp_of(uint64_t n, int blocks) {
  const uint64_t warps = (uint64_t)blocks * (kThreads / 32);
  return (n + warps - 1) / warps;
}

// Scratch of a two-phase (ranked placement) build: one arrival counter per
// bucket and an overflow list of `cap` pairs (see rank_place_kernel).
struct PlaceBuffers {
  uint32_t *counters = nullptr;
  uint32_t *ovf_k = nullptr;
  uint32_t *ovf_v = nullptr;
  uint64_t cap = 0;
  // Grouped input in regions of `region` items per group (0: a dense input):
  // group g's pairs are [g * region, ends[g]); the rest of its region is unused.
  const uint32_t *ends = nullptr;
  uint32_t region = 0;
  uint64_t region_M = 0;  // Lemire-Kaser-Kurz constant of `region`: i / region = mulhi(region_M, i)
};

// Status bit of a grouping into fixed regions: some group had more pairs than
// its region holds (the pairs beyond it were not written).
constexpr uint32_t kStatusGroupRegion = 32u;

// kern_bcht.cu
cudaError_t launch_place_bcht(int B, const TableView &tv, const uint32_t *k, const uint32_t *v, uint64_t n,
                              const PlaceBuffers &pb, bool count, cudaStream_t s);
cudaError_t launch_insert_bcht(int B, const TableView &tv, const uint32_t *k, const uint32_t *v,
                               uint64_t n, const LaunchOpts &o, cudaStream_t s);
cudaError_t launch_find_bcht(int B, const TableView &tv, const uint32_t *q, uint32_t *out,
                             uint64_t n, const LaunchOpts &o, cudaStream_t s);
// The staged find of 16-pair buckets; early_exit = false gives the stop rule
// of P2BHT, IHT and the load-balanced BCHT (read on until the key is found).
cudaError_t launch_find_bcht_async(int B, const TableView &tv, const uint32_t *q, uint32_t *out, uint64_t n,
                                   const LaunchOpts &o, cudaStream_t s, bool early_exit = true);
cudaError_t launch_find_set_async(const TableView &tv, const uint32_t *q, uint32_t *out, uint64_t n,
                                  const LaunchOpts &o, cudaStream_t s);
bool bcht_shape_supported(int B, int G);

// kern_set.cu (keys-only BCHT, 32 four-byte keys per bucket)
cudaError_t launch_place_set(const TableView &tv, const uint32_t *k, uint64_t n, const PlaceBuffers &pb, bool count,
                             cudaStream_t s);
bool set_shape_supported(int B, int G);
cudaError_t launch_insert_set(const TableView &tv, const uint32_t *k, const uint32_t *v, uint64_t n,
                              const LaunchOpts &o, cudaStream_t s);
cudaError_t launch_find_set(const TableView &tv, const uint32_t *q, uint32_t *out, uint64_t n, const LaunchOpts &o,
                            cudaStream_t s);

// kern_other.cu
cudaError_t launch_insert_other(int scheme, int B, const TableView &tv, const uint32_t *k,
                                const uint32_t *v, uint64_t n, const LaunchOpts &o, cudaStream_t s);
cudaError_t launch_find_other(int scheme, int B, const TableView &tv, const uint32_t *q,
                              uint32_t *out, uint64_t n, const LaunchOpts &o, cudaStream_t s);
bool other_shape_supported(int scheme, int B, int G);
cudaError_t launch_fill(const TableView &tv, uint64_t num_slots, cudaStream_t s);
cudaError_t launch_dup_check(const TableView &tv, int B, bool key_slots, const uint32_t *keys, uint64_t n,
                             cudaStream_t s);
cudaError_t launch_hash(const TableView &tv, const uint32_t *k, uint32_t *out, uint64_t n,
                        cudaStream_t s);

// kern_probe.cu: memory-system ceiling probe (see ght_probe_lines)
cudaError_t launch_line_probe(int mode, void *lines, uint64_t num_lines, uint64_t ops, uint32_t seed,
                              cudaStream_t s);

// kern_group.cu: reorder (keys, values) by H_0(k) >> shift into out_k/out_v
// (values NULL: out_v receives each item's input position); counts[g] = items
// of group g, cursors[g] = end of group g in the output.
// Second-level split of a region-grouped array (launch_subgroup).
struct SubSplit {
  const uint32_t *ends1 = nullptr;  // per group: end of its pairs in the grouped array
  uint32_t region1 = 0;             // the grouped array's region per group
  uint64_t region1_M = 0;           // i / region1 = mulhi(region1_M, i)
  int fine_shift = 0;               // sub-group of a key: H_0(k) >> fine_shift
  int subs_log2 = 0;                // sub-groups per group, log2 (<= 8)
  uint32_t groups = 0;              // groups of the first level
};

// Where a grouping in region mode puts an item that does not fit its
// group's region: with count set (a grouped find), appended to this list as
// (key, value, hash index tv.first); else kStatusGroupRegion is set.
struct SpillList {
  uint32_t *k = nullptr, *v = nullptr, *round = nullptr;
  unsigned long long *count = nullptr;
  unsigned long long cap = 0;
};

// Optional parts of a grouping in region mode. d_n: the input's length is
// min(n, *d_n), read on the device. ident: items are grouped by key >> shift
// (the key is a position), not by a hash of the key.
struct GroupExtras {
  const unsigned long long *d_n = nullptr;
  SpillList spill;
  bool ident = false;
  // second level of a grouped find (sub-groups of at most 256 buckets): each
  // item's bucket within its sub-group, written beside it
  uint8_t *out_b = nullptr;
};

// Reorder the pairs of a region-grouped array (len entries, groups of
// 2^subs_log2 <= 256 sub-groups) by sub-group into regions of `region` entries:
// sub-group f's pairs go to [f * region, cursors[f]); bins = sub-groups in
// all. A sub-group with more pairs than its region sets kStatusGroupRegion.
cudaError_t launch_subgroup(const TableView &tv, const uint32_t *keys, const uint32_t *values, uint64_t len,
                            const SubSplit &sub, uint32_t bins, uint32_t *cursors, uint32_t region, uint32_t *out_k,
                            uint32_t *out_v, cudaStream_t s, const GroupExtras &x = GroupExtras());

// Smallest first-level region a second-level split accepts (smaller regions
// would leave its tiles mostly empty). Regions are multiples of 8 entries, so
// a region's tiles start on 16-byte boundaries.
constexpr uint32_t kSubgroupMinRegion = 6144;

// kern_place.cu: first-choice placement of sub-group-split pairs, one block
// per sub-group of 2^fine_shift buckets (see block_place_kernel); writes every
// table line, so the table needs no fill. Sub-group f's pairs are
// [f * region, ends[f]) of pk/pv; bins sub-groups in all. fine_shift may not
// exceed block_place_fine_shift (the sub-groups whose buckets fill 64 KB).
int block_place_fine_shift(int B, bool key_slots);
cudaError_t launch_block_place(int B, bool key_slots, const TableView &tv, const uint32_t *pk, const uint32_t *pv,
                               const uint32_t *ends, uint32_t region, uint32_t bins, int fine_shift,
                               const PlaceBuffers &pb, bool count, cudaStream_t s);

// region > 0: no count pass; group g's pairs go to [g * region, ...) and
// cursors[g] ends as the end of its pairs (counts is not written); a group
// with more than `region` pairs sets kStatusGroupRegion in tv.ctrl.
cudaError_t launch_group(const TableView &tv, const uint32_t *keys, const uint32_t *values, uint64_t n,
                         int shift, uint32_t groups, uint32_t *counts, uint32_t *cursors, uint32_t *out_k,
                         uint32_t *out_v, cudaStream_t s, uint32_t region = 0,
                         const GroupExtras &x = GroupExtras());
// kern_gfind.cu: grouped bulk find of 16-pair buckets (see grouped_lookup_kernel).
// Lists of one round: items answered (query position, value) and items left
// for the next round (key, query position); `cap` entries each.
struct GroupedFindLists {
  uint32_t *res_p = nullptr, *res_v = nullptr;
  unsigned long long *res_count = nullptr;
  uint32_t *cont_k = nullptr, *cont_p = nullptr;
  unsigned long long *cont_count = nullptr;
  unsigned long long *claim = nullptr;  // sub-group claim cursor of the round, zero at launch
  unsigned long long cap = 0;
};
// Sub-groups of a grouped find: 2^8 buckets (32 KB of 16-pair buckets).
constexpr int kGFindFineShift = 8;
// Answers return to query order in windows of 2^13 positions (32 KB).
constexpr int kGFindWindowLog2 = 13;
cudaError_t launch_grouped_lookup(const TableView &tv, int round, bool early_exit, bool count, const uint32_t *gk,
                                  const uint32_t *gp, const uint8_t *gb, const uint32_t *ends, uint32_t region,
                                  uint32_t bins, int fine_shift, const GroupedFindLists &fl, cudaStream_t s);
cudaError_t launch_grouped_spill(const TableView &tv, bool early_exit, bool count, const SpillList &spill,
                                 const GroupedFindLists &fl, uint64_t n_queries, cudaStream_t s);
cudaError_t launch_window_write(const uint32_t *rp, const uint32_t *rv, const uint32_t *ends, uint64_t n,
                                uint32_t *out, cudaStream_t s);

// dst[pos[j]] = src[j] for j < n.
cudaError_t launch_unpermute(const uint32_t *src, const uint32_t *pos, uint64_t n, uint32_t *dst, cudaStream_t s);

}  // namespace ght
