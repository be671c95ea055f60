// kern_group.cu -- grouping of the input pairs by first-choice bucket range
// before a build (a GB300 locality measure, not part of the paper's method,
// which may insert keys in any order).
//
// A random insert touches a 128-byte bucket line that has usually left the
// L2 since the previous insert into it, so every insert pays a DRAM line read
// plus a partial-line write-back. Grouping the pairs by H_0(k) >> shift and
// inserting the groups in order keeps the in-flight inserts inside a window
// of a few MB of the table, whose lines then stay in L2 while they fill up.
#include "ght_bulk.cuh"
#include "ght_internal.h"
#include "ght_kernels.cuh"

namespace ght {

// The hash a grouping goes by, h_{tv.first} (0 for builds; a grouped find's
// round r groups by H_r), as hash index 0 of a family, so the per-item hash
// takes its constants from registers.
__device__ __forceinline__ HashFamily grouping_hash(const TableView &tv) {
  HashFamily hf = tv.hf;
  hf.a[0] = select4(tv.hf.a, tv.first);
  hf.c[0] = select4(tv.hf.c, tv.first);
  return hf;
}

// Group of key k: its bucket under hf's hash 0, shifted down; sentinels go to group 0.
__device__ __forceinline__ uint32_t group_of(const HashFamily &hf, uint32_t k, int shift) {
  return k == kEmptyKey ? 0u : (bucket_of(hf, 0, k) >> shift);  // sentinels are flagged by the insert
}

// Pass 1: per-group counts (block-local histogram in shared memory). With
// 16-byte aligned keys each thread takes four keys per 16-byte load, two
// loads in flight per turn.
__global__ void __launch_bounds__(256)
group_count_kernel(TableView tv, const uint32_t *__restrict__ keys, uint64_t n, int shift, uint32_t groups,
                   uint32_t *__restrict__ counts) {
  extern __shared__ uint32_t sh[];
  const HashFamily hf = grouping_hash(tv);
  for (uint32_t i = threadIdx.x; i < groups; i += blockDim.x) sh[i] = 0u;
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t head = 0;
  if ((reinterpret_cast<uintptr_t>(keys) & 15u) == 0u) {
    const uint4 *k4 = reinterpret_cast<const uint4 *>(keys);
    const uint64_t n4 = n / 4;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += 2 * stride) {
      const bool second = i + stride < n4;
      const uint4 ka = __ldg(k4 + i);
      const uint4 kb = second ? __ldg(k4 + i + stride) : ka;
      const uint32_t a[4] = {ka.x, ka.y, ka.z, ka.w}, b[4] = {kb.x, kb.y, kb.z, kb.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) atomicAdd(&sh[group_of(hf, a[j], shift)], 1u);
      if (second) {
#pragma unroll
        for (int j = 0; j < 4; ++j) atomicAdd(&sh[group_of(hf, b[j], shift)], 1u);
      }
    }
    head = n4 * 4;
  }
  for (uint64_t i = head + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    atomicAdd(&sh[group_of(hf, __ldg(keys + i), shift)], 1u);
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < groups; i += blockDim.x)
    if (sh[i]) atomicAdd(&counts[i], sh[i]);
}

// Exclusive prefix sum of the counts into the cursors (one block).
__global__ void __launch_bounds__(1024)
group_scan_kernel(const uint32_t *__restrict__ counts, uint32_t groups, uint32_t *__restrict__ cursors) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (uint32_t base = 0; base < groups; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t x = i < groups ? counts[i] : 0u;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      uint32_t t = warp_tot[lane];
      uint32_t ti = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, ti, o);
        if (lane >= o) ti += y;
      }
      warp_tot[lane] = ti - t;  // exclusive warp offsets
    }
    __syncthreads();
    if (i < groups) cursors[i] = carry + warp_tot[wid] + incl - x;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += warp_tot[wid] + incl;
    __syncthreads();
  }
}

// Pass 2: scatter pairs to their group. Each block takes tiles of
// kGroupTile pairs; a tile's keys and values arrive in shared memory by bulk
// asynchronous copies issued one tile ahead (two buffers, each completed on
// its own mbarrier), so the copies of tile i + 1 run while tile i is ranked
// per group, reordered by group in place, and written out. One output range
// per non-empty group is reserved with a single global atomic, and
// consecutive threads store consecutive items, so a group's items leave as
// one contiguous run instead of scattered 4-byte stores. Keys and values
// must be 16-byte aligned (the host checks); a tile's last n mod 4 items are
// read directly.
constexpr int kGroupThreads = 384;
// 6144-pair tiles: 111 KB of shared memory, two blocks (24 warps) per SM.
// The tile's fixed cost (a prefix over every group, one reservation per
// group) is what large tiles amortise: at 2^28 pairs the grouping took 2.98
// / 2.25 / 1.73 / 1.67 ms with 2560 / 3840 / 6144 (512 threads) / 6144 (384
// threads) pairs per tile.
constexpr int kGroupPerThread = 16;
constexpr int kGroupTile = kGroupThreads * kGroupPerThread;
constexpr uint32_t kGroupWaitPolls = 1u << 26;  // bounded wait for a tile's copies

// shared memory of the scatter: two tile buffers (keys, values), the group
// of each reordered item, and per-group count, prefix and reserved position
size_t group_scatter_smem(uint32_t groups) {
  return 4ull * kGroupTile * sizeof(uint32_t) + kGroupTile * sizeof(uint16_t) + 3ull * groups * sizeof(uint32_t);
}

// POS: the values are the items' input positions (values is not read).
// IDENT: the grouping key is the key itself (k >> shift), not a hash of it:
// a grouped find returns its answers to query order by grouping (position,
// answer) items by position.
// d_n: when set, the number of items is min(n, *d_n), read on the device (a
// list whose length an earlier kernel wrote).
// spill.count: when set, an item beyond its group's region is appended to the
// spill list (key, value, tv.first) instead of setting kStatusGroupRegion.
// SUB: the input is itself grouped into regions (sub.ends1, sub.region1), and
// each group is split further into 2^sub.subs_log2 sub-groups of
// H_0 >> sub.fine_shift. Tiles then follow the regions (tile t of group g
// starts at g * region1 + t * kGroupTile and ends at most at ends1[g]), so
// `groups` (= 1 << subs_log2) local bins cover a tile, and bin j of a tile of
// group g is sub-group (g << subs_log2) + j.
// LB (with SUB, a grouped find's second level): each item's bucket within
// its sub-group (< 256) is written to out_b beside it.
template <bool POS, bool SUB, bool IDENT = false, bool LB = false>
__global__ void __launch_bounds__(kGroupThreads, 2)
group_scatter_kernel(TableView tv, const uint32_t *__restrict__ keys, const uint32_t *__restrict__ values,
                     uint64_t n, int shift, uint32_t groups, uint32_t *__restrict__ cursors,
                     uint32_t *__restrict__ out_k, uint32_t *__restrict__ out_v, uint32_t region, SubSplit sub,
                     const unsigned long long *__restrict__ d_n, SpillList spill, uint8_t *__restrict__ out_b) {
  static_assert(!LB || (SUB && !IDENT && !POS), "bucket indexes come with a second level by hash");
  if (d_n) {
    const unsigned long long dn = *d_n;
    if (dn < n) n = dn;
  }
  extern __shared__ uint4 gs_smem[];
  uint32_t *bufs = reinterpret_cast<uint32_t *>(gs_smem);  // [2][keys kGroupTile | values kGroupTile]
  uint16_t *gid = reinterpret_cast<uint16_t *>(bufs + 4 * kGroupTile);  // [kGroupTile] group of each reordered item
  uint32_t *cnt = reinterpret_cast<uint32_t *>(gid + kGroupTile);      // [groups] items of each group in the tile
  uint32_t *pre = cnt + groups;                                           // [groups] exclusive prefix of cnt
  uint32_t *base = pre + groups;                                          // [groups] reserved output position
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t warp_sums[kGroupThreads / 32];
  __shared__ int s_abort;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const HashFamily hf = grouping_hash(tv);
  // SUB: tiles per region; a tile's start and length follow its group's pairs
  const uint32_t tpg = SUB ? (sub.region1 + kGroupTile - 1) / kGroupTile : 0u;
  const uint64_t ntiles = SUB ? (uint64_t)sub.groups * tpg : (n + kGroupTile - 1) / kGroupTile;
  auto tile_span = [&](uint64_t tile, uint64_t *t0, uint32_t *tn) {
    if (SUB) {
      const uint32_t g = (uint32_t)(tile / tpg), t = (uint32_t)(tile % tpg);
      // a group's cursor passes its region's end when the group overflowed
      // (the items beyond were not written): read the region at most
      const uint64_t start = (uint64_t)g * sub.region1 + (uint64_t)t * kGroupTile;
      const uint64_t end = min((uint64_t)__ldg(sub.ends1 + g), (uint64_t)(g + 1u) * sub.region1);
      *t0 = start;
      *tn = end > start ? (uint32_t)(end - start < (uint64_t)kGroupTile ? end - start : (uint64_t)kGroupTile) : 0u;
    } else {
      *t0 = tile * kGroupTile;
      *tn = (uint32_t)(n - *t0 < (uint64_t)kGroupTile ? n - *t0 : (uint64_t)kGroupTile);
    }
  };
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init_fence();
    s_abort = 0;
  }
  __syncthreads();
  // thread 0: copy the whole 16-byte pieces of tile `tile` into buffer b
  auto issue = [&](uint64_t tile, int b) {
    uint64_t t0;
    uint32_t tn;
    tile_span(tile, &t0, &tn);
    const uint32_t bytes = (tn / 4u) * 16u;
    uint32_t *dk = bufs + 2 * b * kGroupTile;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bars[b], (POS ? 1u : 2u) * bytes);
    if (bytes) {
      bulk_g2s(dk, keys + t0, bytes, &bars[b]);
      if (!POS) bulk_g2s(dk + kGroupTile, values + t0, bytes, &bars[b]);
    }
  };
  uint32_t j = 0;  // this block's tile count so far
  uint64_t tile = blockIdx.x;
  if (tid == 0 && tile < ntiles) issue(tile, 0);
  for (; tile < ntiles; tile += gridDim.x, ++j) {
    const int b = (int)(j & 1u);
    const uint64_t next = tile + gridDim.x;
    if (tid == 0 && next < ntiles) issue(next, b ^ 1);  // buffer b ^ 1 was released at the end of the last tile
    for (uint32_t i = tid; i < groups; i += kGroupThreads) cnt[i] = 0u;
    if (!mbar_wait_bounded(&bars[b], (j >> 1) & 1u, kGroupWaitPolls)) s_abort = 1;
    __syncthreads();
    if (s_abort) {
      if (tid == 0) {
        atomicOr(&tv.ctrl->status, kStatusTimeout);
        if (next < ntiles) mbar_wait_bounded(&bars[b ^ 1], ((j + 1) >> 1) & 1u, kGroupWaitPolls);
      }
      return;
    }
    uint64_t t0;
    uint32_t tn;
    tile_span(tile, &t0, &tn);
    // an empty tile (a region's tail): nothing read or written; the next
    // iteration's copy goes to the other buffer, and the barrier above
    // ordered this tile's counter reset before the next one's
    if (tn == 0u) continue;
    const uint32_t tbulk = tn & ~3u;  // items that came by the bulk copies
    uint32_t *sk = bufs + 2 * b * kGroupTile, *sv = sk + kGroupTile;
    // SUB: the first sub-group of the tile's group
    const uint32_t bin0 = SUB ? (uint32_t)(tile / tpg) << sub.subs_log2 : 0u;
    uint32_t k[kGroupPerThread], v[kGroupPerThread], gr[kGroupPerThread];
#pragma unroll
    for (int u = 0; u < kGroupPerThread; ++u) {
      const uint32_t i = (uint32_t)u * kGroupThreads + tid;
      if (i < tn) {
        k[u] = i < tbulk ? sk[i] : __ldg(keys + t0 + i);
        v[u] = POS ? (uint32_t)(t0 + i) : (i < tbulk ? sv[i] : __ldg(values + t0 + i));
        // (IDENT: positions below the batch size give groups in range; the
        // clamp keeps any other key inside the tile's counters)
        uint32_t g, lb = 0u;
        if constexpr (IDENT) {
          g = min(SUB ? (k[u] >> sub.fine_shift) - bin0 : k[u] >> shift, groups - 1u);
        } else if constexpr (SUB) {
          const uint32_t bk = k[u] == kEmptyKey ? 0u : bucket_of(hf, 0, k[u]);
          g = (bk >> sub.fine_shift) - bin0;
          if (LB) lb = bk & ((1u << sub.fine_shift) - 1u);
        } else {
          g = group_of(hf, k[u], shift);
        }
        // group < 4096 (LB: < 256, bucket in bits 24..31), rank < kGroupTile
        gr[u] = (lb << 24) | (g << 16) | atomicAdd(&cnt[g], 1u);
      }
    }
    __syncthreads();
    // exclusive prefix over the groups (each thread a contiguous run of them)
    // and one output reservation per non-empty group
    const uint32_t per = (groups + kGroupThreads - 1) / kGroupThreads;
    const uint32_t g0 = tid * per, g1 = g0 + per < groups ? g0 + per : groups;
    uint32_t run = 0;
    for (uint32_t i = g0; i < g1; ++i) run += cnt[i];
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < wid; ++w) before += warp_sums[w];
    uint32_t acc = before + incl - run;
    uint32_t *cur = cursors + bin0;  // this tile's cursors
    // reservations: with at most two groups per thread the atomics' results
    // stay in registers until after the reorder, so their round trip overlaps it
    uint32_t r0 = 0u, r1 = 0u;
    if (per <= 2) {
      const uint32_t c0 = g0 < g1 ? cnt[g0] : 0u, c1 = g0 + 1 < g1 ? cnt[g0 + 1] : 0u;
      if (c0) r0 = atomicAdd(&cur[g0], c0);
      if (c1) r1 = atomicAdd(&cur[g0 + 1], c1);
      if (g0 < g1) pre[g0] = acc;
      if (g0 + 1 < g1) pre[g0 + 1] = acc + c0;
    } else {
      for (uint32_t i = g0; i < g1; ++i) {
        pre[i] = acc;
        acc += cnt[i];
        if (cnt[i]) base[i] = atomicAdd(&cur[i], cnt[i]);
      }
    }
    __syncthreads();
    // reorder by group in place (every item of the buffer was read above)
#pragma unroll
    for (int u = 0; u < kGroupPerThread; ++u) {
      if ((uint32_t)u * kGroupThreads + tid < tn) {
        const uint32_t g = LB ? (gr[u] >> 16) & 0xFFu : gr[u] >> 16;
        const uint32_t at = pre[g] + (gr[u] & 0xFFFFu);
        sk[at] = k[u];
        sv[at] = v[u];
        gid[at] = (uint16_t)(LB ? g | ((gr[u] >> 24) << 8) : g);
      }
    }
    if (per <= 2) {
      if (g0 < g1) base[g0] = r0;
      if (g0 + 1 < g1) base[g0 + 1] = r1;
    }
    __syncthreads();
    for (uint32_t i = tid; i < tn; i += kGroupThreads) {
      const uint32_t gl = gid[i];
      const uint32_t g = LB ? gl & 0xFFu : gl;
      const uint32_t at = base[g] + (i - pre[g]);
      if (region && at >= (bin0 + g + 1u) * region) {  // beyond the group's region
        if (spill.count) {  // a grouped find answers it separately
          const unsigned long long at_s = atomicAdd(spill.count, 1ull);
          if (at_s < spill.cap) {
            spill.k[at_s] = sk[i];
            spill.v[at_s] = sv[i];
            spill.round[at_s] = (uint32_t)tv.first;
          }
        } else {  // a build regroups exactly
          atomicOr(&tv.ctrl->status, kStatusGroupRegion);
        }
        continue;
      }
      out_k[at] = sk[i];
      out_v[at] = sv[i];
      if (LB) out_b[at] = (uint8_t)(gl >> 8);
    }
    __syncthreads();
  }
}

// Region mode: each group's cursor starts at the group's region.
__global__ void region_cursors_kernel(uint32_t *__restrict__ cursors, uint32_t groups, uint32_t region) {
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += gridDim.x * blockDim.x)
    cursors[g] = g * region;
}

// dst[pos[j]] = src[j]: answers of position-carrying items back to input order.
__global__ void __launch_bounds__(256)
unpermute_kernel(const uint32_t *__restrict__ src, const uint32_t *__restrict__ pos, uint64_t n,
                 uint32_t *__restrict__ dst) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride)
    dst[__ldg(pos + j)] = __ldg(src + j);
}

cudaError_t launch_unpermute(const uint32_t *src, const uint32_t *pos, uint64_t n, uint32_t *dst, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int blocks = 0;
  const cudaError_t e = grid_for(unpermute_kernel, n, 0, &blocks);
  if (e != cudaSuccess) return e;
  unpermute_kernel<<<blocks, 256, 0, s>>>(src, pos, n, dst);
  return cudaGetLastError();
}

cudaError_t launch_group(const TableView &tv, const uint32_t *keys, const uint32_t *values, uint64_t n,
                         int shift, uint32_t groups, uint32_t *counts, uint32_t *cursors, uint32_t *out_k,
                         uint32_t *out_v, cudaStream_t s, uint32_t region, const GroupExtras &x) {
  if (groups == 0 || groups > kMaxGroups) return cudaErrorInvalidValue;
  if (region) {
    if ((uint64_t)groups * region > 0xFFFFFFFFull) return cudaErrorInvalidValue;
    region_cursors_kernel<<<(groups + 255) / 256, 256, 0, s>>>(cursors, groups, region);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || n == 0) return e;
  } else if (n == 0) {
    return cudaMemsetAsync(counts, 0, groups * sizeof(uint32_t), s);
  }
  if (n > 0xFFFFFFFFull) return cudaErrorInvalidValue;
  if ((x.d_n || x.spill.count || x.ident) && !region) return cudaErrorInvalidValue;  // region mode only
  const bool pos = values == nullptr;  // carry input positions instead of values
  if (pos && x.ident) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(values)) & 15u) return cudaErrorInvalidValue;
  cudaError_t e;
  int blocks = 0;
  if (!region) {  // exact offsets: count pass and prefix
    if ((e = cudaMemsetAsync(counts, 0, groups * sizeof(uint32_t), s)) != cudaSuccess) return e;
    e = grid_for(group_count_kernel, n, 0, &blocks);
    if (e != cudaSuccess) return e;
    group_count_kernel<<<blocks, 256, groups * sizeof(uint32_t), s>>>(tv, keys, n, shift, groups, counts);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    group_scan_kernel<<<1, 1024, 0, s>>>(counts, groups, cursors);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const uint64_t tiles = (n + kGroupTile - 1) / kGroupTile;
  const size_t smem = group_scatter_smem(groups);
  auto kern = pos ? group_scatter_kernel<true, false>
                  : (x.ident ? group_scatter_kernel<false, false, true> : group_scatter_kernel<false, false>);
  e = grid_for_smem(kern, kGroupThreads, smem, tiles * kGroupThreads, 0, &blocks);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kGroupThreads, smem, s>>>(tv, keys, values, n, shift, groups, cursors, out_k, out_v, region,
                                           SubSplit(), x.d_n, x.spill, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_subgroup(const TableView &tv, const uint32_t *keys, const uint32_t *values, uint64_t len,
                            const SubSplit &sub, uint32_t bins, uint32_t *cursors, uint32_t region, uint32_t *out_k,
                            uint32_t *out_v, cudaStream_t s, const GroupExtras &x) {
  if (len > 0xFFFFFFFFull || (uint64_t)bins * region > 0xFFFFFFFFull || sub.subs_log2 > 8 || region == 0 ||
      sub.region1 < kSubgroupMinRegion || (sub.region1 & 7u) || sub.groups == 0)
    return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(values)) & 15u) return cudaErrorInvalidValue;
  region_cursors_kernel<<<(bins + 255) / 256, 256, 0, s>>>(cursors, bins, region);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || len == 0) return e;
  const uint32_t local = 1u << sub.subs_log2;  // a tile lies in one group
  const uint64_t tiles = (uint64_t)sub.groups * ((sub.region1 + kGroupTile - 1) / kGroupTile);
  const size_t smem = group_scatter_smem(local);
  int blocks = 0;
  if (x.d_n) return cudaErrorInvalidValue;  // the input's extent comes from sub.ends1
  if (x.out_b && (x.ident || sub.fine_shift > 8 || sub.subs_log2 > 8)) return cudaErrorInvalidValue;
  auto kern = x.ident   ? group_scatter_kernel<false, true, true>
              : x.out_b ? group_scatter_kernel<false, true, false, true>
                        : group_scatter_kernel<false, true>;
  e = grid_for_smem(kern, kGroupThreads, smem, tiles * kGroupThreads, 0, &blocks);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kGroupThreads, smem, s>>>(tv, keys, values, len, 0, local, cursors, out_k, out_v, region, sub,
                                           nullptr, x.spill, x.out_b);
  return cudaGetLastError();
}

}  // namespace ght
