// ght_find_async.cuh -- bulk find of the bucketed tables with bucket parts
// staged in shared memory by asynchronous copies (cp.async), for 128-byte
// buckets (16 pairs, or 32 keys of the keys-only set) read by 4-lane tiles.
//
// The probe order, stop rules and tile evaluation are those of
// bucketed_find_kernel: every scheme probes H_0, H_1, ... and stops at the
// bucket holding the key; BCHT (and the set) also stops at a bucket with an
// empty slot (Sec. V-B find), P2BHT, IHT and the load-balanced BCHT read on
// until the last candidate (Sec. V-C, V-D: no early exit), which the
// early_exit argument selects. The difference is where a bucket in
// flight lives: there, in registers (32 per query set and lane), which caps
// a lane at two sets, evaluated one step after their reads are issued; here,
// mostly in the warp's shared memory, so a lane keeps KPL sets in flight and
// a set is evaluated KPL - 1 steps after its copies were issued, with the
// copies of the newer sets still outstanding (cp.async.wait_group). With the
// default six sets, two of them stay in registers: the same depth in 16 KB
// of shared memory per warp instead of 24, so 12 warps fit on an SM instead
// of 8 (2^28 keys: 3 % faster finds).
#pragma once

#include "ght_find.cuh"
#include "ght_internal.h"

namespace ght {

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Shared memory per warp: KPL sets x 32 buckets (one per lane of the warp as
// owner) x 8 LINES chunks of 16 bytes (LINES = 128-byte lines per bucket).
// One line: lane r of a tile holds chunks 2r and 2r + 1 of each of its
// tile's buckets, and chunk c of the bucket of owner lane o is stored at
// chunk position c ^ (o >> 2 & 7), so the eight tiles of a warp read
// different bank groups. Two lines (32 pairs): lane r holds chunks r + 4i,
// i < 4, at position c ^ 4 (o >> 2 & 1): the two tiles that share a quarter
// of the warp's 16-byte accesses then cover the eight bank groups once.
template <int KPL, int LINES = 1>
constexpr size_t find_async_smem_per_warp() {
  return (size_t)KPL * 32 * 8 * LINES * 16;
}

template <int LINES>
__device__ __forceinline__ unsigned staged_chunk(int r, int i) {
  return LINES == 1 ? (unsigned)(2 * r + i) : (unsigned)(r + 4 * i);
}

// KR > 0: the last KR of the KPL sets hold their bucket parts in registers
// (plain 16-byte loads, 8 registers per tile member and lane) instead of
// shared memory, so a warp keeps the same depth in (KPL - KR) x 4 KB.
template <int KPL, int WARPS, bool COUNT, typename S = PairSlot, int LINES = 1, int KR = 0>
__global__ void __launch_bounds__(32 * WARPS)
bcht_find_async_kernel(TableView tv, const uint32_t *__restrict__ queries, uint32_t *__restrict__ out, uint64_t n,
                       uint64_t per_warp, bool early_exit) {
  constexpr int G = 4;
  constexpr bool kPairs = sizeof(typename S::T) == 8;  // else 32-bit keys (a set)
  constexpr int kChunks = 8 * LINES;                   // 16-byte chunks per bucket
  constexpr int kPerLane = kChunks / G;                // chunks a tile lane copies and evaluates
  constexpr int KS = KPL - KR;                         // sets staged in shared memory
  static_assert(KPL >= 2 && KPL <= 8, "query sets in flight");
  static_assert(LINES == 1 || (LINES == 2 && kPairs), "one-line buckets, or 32-pair buckets");
  static_assert(KR >= 0 && KS >= 1 && (KR == 0 || LINES == 1), "register sets hold one-line buckets");
  uint4 rbuf[KR > 0 ? KR : 1][G][kPerLane];  // register sets: [set - KS][tile member][chunk]
  extern __shared__ uint4 fa_smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int r = lane & (G - 1);
  const int tbase = lane - r;
  // this tile's chunk swizzle
  const unsigned swz = LINES == 1 ? ((unsigned)(lane >> 2) & 7u) : (((unsigned)(lane >> 2) & 1u) << 2);
  const unsigned tmask = ((1u << G) - 1u) << tbase;
  uint4 *wbuf = fa_smem + (size_t)wib * KS * 32 * kChunks;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t beg = warp * per_warp;
  if (beg >= n) return;  // whole warp
  const uint64_t end = beg + per_warp < n ? beg + per_warp : n;
  const unsigned below = lanemask_lt();

  StreamQueue sq;
  stream_init(sq, queries, beg, end, lane);
  bool active[KPL];
  uint32_t key[KPL], act[KPL];
  uint64_t idx[KPL];
  int probe[KPL];
#pragma unroll
  for (int s = 0; s < KPL; ++s) {
    active[s] = false;
    key[s] = kEmptyKey;
    act[s] = 0u;
    idx[s] = 0;
    probe[s] = 0;
  }
  unsigned long long probes = 0, answered = 0;

  for (;;) {
#pragma unroll
    for (int s = 0; s < KPL; ++s) {
      // -- refill set s from the stream, then issue the copies of its buckets
      const unsigned need = __ballot_sync(kFull, !active[s]);
      if (need != 0u && sq.base + sq.head < end) {
        uint32_t k;
        const uint64_t at = stream_take(sq, queries, end, need, below, lane, k);
        if (at < end) {
          if (COUNT) answered++;
          if (k == kEmptyKey) {
            out[at] = S::missing();  // the sentinel is never a key
          } else {
            active[s] = true;
            key[s] = k;
            idx[s] = at;
            probe[s] = 0;
          }
        }
      }
      act[s] = __ballot_sync(kFull, active[s]);
      if (act[s] != 0u) {
        const uint32_t myb = active[s] ? bucket_of(tv.hf, probe[s], key[s]) : 0u;
        uint4 *sbuf = wbuf + (size_t)(s < KS ? s : 0) * 32 * kChunks;
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const int owner = tbase + j;
          const uint32_t bj = __shfl_sync(kFull, myb, owner);
          if ((act[s] >> owner) & 1u) {
            // this lane's quarter of the bucket (one line: pairs [4r, 4r + 4) or keys [8r, 8r + 8))
            const uint4 *src = reinterpret_cast<const uint4 *>(tv.slots) + (uint64_t)bj * kChunks;
            uint4 *row = sbuf + owner * kChunks;
#pragma unroll
            for (int i = 0; i < kPerLane; ++i) {
              const unsigned c = staged_chunk<LINES>(r, i);
              if (s < KS) cp_async16(row + (c ^ swz), src + c);
              else rbuf[s >= KS ? s - KS : 0][j][i] = __ldg(src + c);
            }
          }
        }
      }
      cp_async_commit();  // one group per set step, empty or not
      // -- evaluate the set issued KPL - 1 steps ago: its copies are the
      // oldest outstanding group of this lane
      const int e = (s + 1) % KPL;
      cp_async_wait<KPL - 1>();
      __syncwarp();  // the other lanes' copies of set e are visible
      if (act[e] != 0u) {
        const uint4 *ebuf = wbuf + (size_t)(e < KS ? e : 0) * 32 * kChunks;
        bool my_hit = false, my_emp = false;
        uint32_t my_val = S::missing();
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const int owner = tbase + j;
          const uint32_t kj = __shfl_sync(kFull, key[e], owner);
          const bool aj = (act[e] >> owner) & 1u;
          bool hit = false, emp = false;
          uint32_t hv = 0u;
          if (aj) {
            const uint4 *row = ebuf + owner * kChunks;
            if constexpr (kPairs) {
#pragma unroll
              for (int i = 0; i < kPerLane; ++i) {
                // pairs (c.x, c.y), (c.z, c.w)
                const uint4 c = e < KS ? row[staged_chunk<LINES>(r, i) ^ swz] : rbuf[e >= KS ? e - KS : 0][j][i];
                if (c.x == kj) {
                  hit = true;
                  hv = c.y;
                }
                if (c.z == kj) {
                  hit = true;
                  hv = c.w;
                }
                emp |= c.x == kEmptyKey || c.z == kEmptyKey;
              }
            } else {
              const uint4 c0 = e < KS ? row[(2u * r) ^ swz] : rbuf[e >= KS ? e - KS : 0][j][0];
              const uint4 c1 = e < KS ? row[(2u * r + 1u) ^ swz] : rbuf[e >= KS ? e - KS : 0][j][1];
              const uint32_t ks[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
              for (int p = 0; p < 8; ++p) {
                hit |= ks[p] == kj;
                emp |= ks[p] == kEmptyKey;
              }
              hv = 1u;
            }
          }
          const unsigned hb = __ballot_sync(kFull, hit) & tmask;
          const unsigned eb = __ballot_sync(kFull, emp) & tmask;
          const uint32_t val = __shfl_sync(kFull, hv, hb ? __ffs(hb) - 1 : lane);
          if (lane == owner) {
            my_hit = hb != 0u;
            my_emp = eb != 0u;
            my_val = val;
          }
        }
        if ((act[e] >> lane) & 1u) {
          if (COUNT) probes++;
          bool finish = false;
          uint32_t result = S::missing();
          if (my_hit) {
            result = my_val;
            finish = true;
          } else if (early_exit && my_emp) {
            finish = true;
          } else if (++probe[e] >= tv.h) {
            finish = true;
          }
          if (finish) {
            out[idx[e]] = result;
            active[e] = false;
          }
        }
        act[e] = 0u;  // evaluated; the set's next copies are issued on its next refill
      }
      __syncwarp();  // set e's buffer is read before the next step reuses it
    }
    bool any = false;
#pragma unroll
    for (int s = 0; s < KPL; ++s) any |= active[s];
    if (__ballot_sync(kFull, any) == 0u && sq.base + sq.head >= end) break;
  }
  cp_async_wait<0>();
  if (COUNT) {
    probes = warp_sum(probes);
    answered = warp_sum(answered);
    if (lane == 0) {
      atomicAdd(&tv.ctrl->find_probes, probes);
      atomicAdd(&tv.ctrl->find_queries, answered);
    }
  }
}


// Launch with KPL sets in flight (KR of them in registers) and WARPS warps
// per block, as many blocks as are resident at once (shared memory sets the
// residency, (KPL - KR) x 4 KB per warp and bucket line, or registers);
// 2-warp blocks for the deep pipelines keep the resident warps a multiple of
// the SM's four schedulers (6 sets of one-line buckets, 2 in registers: 6
// blocks, 12 warps per SM).
template <int KPL, int WARPS, typename S, int LINES = 1, int KR = 0>
inline cudaError_t launch_staged_find(const TableView &tv, const uint32_t *q, uint32_t *out, uint64_t n, bool count,
                                      int blocks_per_sm, bool early_exit, cudaStream_t s) {
  auto kern = count ? bcht_find_async_kernel<KPL, WARPS, true, S, LINES, KR>
                    : bcht_find_async_kernel<KPL, WARPS, false, S, LINES, KR>;
  constexpr int kBlock = 32 * WARPS;
  const size_t smem = WARPS * find_async_smem_per_warp<KPL - KR, LINES>();
  int blocks = 0;
  cudaError_t e = grid_for_smem(kern, kBlock, smem, n, blocks_per_sm, &blocks);
  if (e != cudaSuccess) return e;
  const uint64_t warps = (uint64_t)blocks * WARPS;
  kern<<<blocks, kBlock, smem, s>>>(tv, q, out, n, (n + warps - 1) / warps, early_exit);
  return cudaGetLastError();
}

// keys_per_lane = sets in flight: 2..8 for one-line buckets, 2..6 for
// two-line buckets (8 KB per set and warp)
template <typename S, int LINES = 1>
inline cudaError_t launch_staged_find_kpl(const TableView &tv, const uint32_t *q, uint32_t *out, uint64_t n,
                                          int keys_per_lane, bool count, int blocks_per_sm, bool early_exit,
                                          cudaStream_t s) {
  if constexpr (LINES == 2) {
    switch (keys_per_lane) {
      case 2: return launch_staged_find<2, 4, S, LINES>(tv, q, out, n, count, blocks_per_sm, early_exit, s);
      case 3: return launch_staged_find<3, 4, S, LINES>(tv, q, out, n, count, blocks_per_sm, early_exit, s);
      case 4: return launch_staged_find<4, 2, S, LINES>(tv, q, out, n, count, blocks_per_sm, early_exit, s);
      case 5: return launch_staged_find<5, 2, S, LINES>(tv, q, out, n, count, blocks_per_sm, early_exit, s);
      case 6: return launch_staged_find<6, 2, S, LINES>(tv, q, out, n, count, blocks_per_sm, early_exit, s);
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (keys_per_lane) {
      case 2: return launch_staged_find<2, 4, S, LINES>(tv, q, out, n, count, blocks_per_sm, early_exit, s);
      case 3: return launch_staged_find<3, 4, S, LINES>(tv, q, out, n, count, blocks_per_sm, early_exit, s);
      case 4: return launch_staged_find<4, 4, S, LINES>(tv, q, out, n, count, blocks_per_sm, early_exit, s);
      case 5: return launch_staged_find<5, 2, S, LINES>(tv, q, out, n, count, blocks_per_sm, early_exit, s);
      // six sets, two of them in registers: 16 KB per warp, six 2-warp
      // blocks (168 registers a thread), 12 warps per SM
      case 6: return launch_staged_find<6, 2, S, LINES, 2>(tv, q, out, n, count, blocks_per_sm, early_exit, s);
      case 7: return launch_staged_find<7, 2, S, LINES>(tv, q, out, n, count, blocks_per_sm, early_exit, s);
      case 8: return launch_staged_find<8, 2, S, LINES>(tv, q, out, n, count, blocks_per_sm, early_exit, s);
      default: return cudaErrorInvalidValue;
    }
  }
}

}  // namespace ght
