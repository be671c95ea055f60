// kern_group.cu -- grouping of the input pairs by first-choice bucket range
// before a build (a GB300 locality measure, not part of the paper's method,
// which may insert keys in any order).
//
// A random insert touches a 128-byte bucket line that has usually left the
// L2 since the previous insert into it, so every insert pays a DRAM line read
// plus a partial-line write-back. Grouping the pairs by H_0(k) >> shift and
// inserting the groups in order keeps the in-flight inserts inside a window
// of a few MB of the table, whose lines then stay in L2 while they fill up.
#include "ght_internal.h"
#include "ght_kernels.cuh"

namespace ght {

__device__ __forceinline__ uint32_t group_of(const TableView &tv, uint32_t k, int shift) {
  return k == kEmptyKey ? 0u : (bucket_of(tv.hf, 0, k) >> shift);  // sentinels are flagged by the insert
}

// Pass 1: per-group counts (block-local histogram in shared memory). With
// 16-byte aligned keys each thread takes four keys per 16-byte load.
__global__ void __launch_bounds__(256)
group_count_kernel(TableView tv, const uint32_t *__restrict__ keys, uint64_t n, int shift, uint32_t groups,
                   uint32_t *__restrict__ counts) {
  extern __shared__ uint32_t sh[];
  for (uint32_t i = threadIdx.x; i < groups; i += blockDim.x) sh[i] = 0u;
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t head = 0;
  if ((reinterpret_cast<uintptr_t>(keys) & 15u) == 0u) {
    const uint4 *k4 = reinterpret_cast<const uint4 *>(keys);
    const uint64_t n4 = n / 4;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
      const uint4 k = __ldg(k4 + i);
      const uint32_t g0 = group_of(tv, k.x, shift), g1 = group_of(tv, k.y, shift);
      const uint32_t g2 = group_of(tv, k.z, shift), g3 = group_of(tv, k.w, shift);
      atomicAdd(&sh[g0], 1u);
      atomicAdd(&sh[g1], 1u);
      atomicAdd(&sh[g2], 1u);
      atomicAdd(&sh[g3], 1u);
    }
    head = n4 * 4;
  }
  for (uint64_t i = head + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    atomicAdd(&sh[group_of(tv, __ldg(keys + i), shift)], 1u);
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

// Pass 2: scatter pairs to their group. Each block takes a tile of
// kGroupTile pairs, ranks them per group in shared memory, reserves one
// output range per non-empty group with a single global atomic, orders the
// tile by group in shared memory, and then writes it with consecutive
// threads storing consecutive items, so a group's items leave as one
// contiguous run instead of scattered 4-byte stores.
constexpr int kGroupPerThread = 16;
constexpr int kGroupTile = 256 * kGroupPerThread;

// Compiled for 4 resident blocks per SM (64 registers, a few spilled; the
// shared memory, 46 KB per block at 512 groups, allows 4): the pass is
// latency-bound between its barriers, so resident blocks are what count
// (2.65 ms at 2^28 pairs against 3.43 ms at the compiler's 2 blocks).
__global__ void __launch_bounds__(256, 4)
group_scatter_kernel(TableView tv, const uint32_t *__restrict__ keys, const uint32_t *__restrict__ values,
                     uint64_t n, int shift, uint32_t groups, uint32_t *__restrict__ cursors,
                     uint32_t *__restrict__ out_k, uint32_t *__restrict__ out_v) {
  extern __shared__ uint32_t sh[];
  uint32_t *cnt = sh;                    // [groups] items of each group in the tile
  uint32_t *pre = cnt + groups;          // [groups] exclusive prefix of cnt
  uint32_t *base = pre + groups;         // [groups] reserved output position
  uint32_t *sk = base + groups;          // [kGroupTile] tile keys ordered by group
  uint32_t *sv = sk + kGroupTile;        // [kGroupTile] tile values
  uint16_t *sg = reinterpret_cast<uint16_t *>(sv + kGroupTile);  // [kGroupTile] group of each ordered item
  __shared__ uint32_t warp_sums[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (uint64_t t0 = (uint64_t)blockIdx.x * kGroupTile; t0 < n; t0 += (uint64_t)gridDim.x * kGroupTile) {
    const uint32_t tile_n = (uint32_t)(n - t0 < (uint64_t)kGroupTile ? n - t0 : (uint64_t)kGroupTile);
    for (uint32_t i = threadIdx.x; i < groups; i += blockDim.x) cnt[i] = 0u;
    __syncthreads();
    uint32_t k[kGroupPerThread], v[kGroupPerThread], g[kGroupPerThread], rank[kGroupPerThread];
#pragma unroll
    for (int u = 0; u < kGroupPerThread; ++u) {
      const uint32_t i = (uint32_t)u * blockDim.x + threadIdx.x;  // coalesced reads
      if (i < tile_n) {
        k[u] = __ldg(keys + t0 + i);
        v[u] = __ldg(values + t0 + i);
        g[u] = group_of(tv, k[u], shift);
        rank[u] = atomicAdd(&cnt[g[u]], 1u);
      }
    }
    __syncthreads();
    // exclusive prefix over the groups (each thread a contiguous run of them)
    // and one output reservation per non-empty group
    const uint32_t per = (groups + blockDim.x - 1) / blockDim.x;
    const uint32_t g0 = threadIdx.x * per, g1 = g0 + per < groups ? g0 + per : groups;
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
    for (uint32_t i = g0; i < g1; ++i) {
      pre[i] = acc;
      acc += cnt[i];
      if (cnt[i]) base[i] = atomicAdd(&cursors[i], cnt[i]);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kGroupPerThread; ++u) {
      const uint32_t i = (uint32_t)u * blockDim.x + threadIdx.x;
      if (i < tile_n) {
        const uint32_t at = pre[g[u]] + rank[u];
        sk[at] = k[u];
        sv[at] = v[u];
        sg[at] = (uint16_t)g[u];
      }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < tile_n; i += blockDim.x) {
      const uint32_t gi = sg[i];
      const uint32_t at = base[gi] + (i - pre[gi]);
      out_k[at] = sk[i];
      out_v[at] = sv[i];
    }
    __syncthreads();
  }
}

cudaError_t launch_group(const TableView &tv, const uint32_t *keys, const uint32_t *values, uint64_t n,
                         int shift, uint32_t groups, uint32_t *counts, uint32_t *cursors, uint32_t *out_k,
                         uint32_t *out_v, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (n > 0xFFFFFFFFull || groups == 0 || groups > kMaxGroups) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(counts, 0, groups * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  int blocks = 0;
  e = grid_for(group_count_kernel, n, 0, &blocks);
  if (e != cudaSuccess) return e;
  group_count_kernel<<<blocks, 256, groups * sizeof(uint32_t), s>>>(tv, keys, n, shift, groups, counts);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  group_scan_kernel<<<1, 1024, 0, s>>>(counts, groups, cursors);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const uint64_t tiles = (n + kGroupTile - 1) / kGroupTile;
  const size_t smem = 3ull * groups * sizeof(uint32_t) + 2ull * kGroupTile * sizeof(uint32_t) +
                      kGroupTile * sizeof(uint16_t);
  e = grid_for_smem(group_scatter_kernel, 256, smem, tiles * 256, 0, &blocks);
  if (e != cudaSuccess) return e;
  group_scatter_kernel<<<blocks, 256, smem, s>>>(tv, keys, values, n, shift, groups, cursors, out_k, out_v);
  return cudaGetLastError();
}

}  // namespace ght
