// ght_find_async.cuh -- BCHT bulk find with bucket parts staged in shared
// memory by asynchronous copies (cp.async), for 16-pair buckets read by
// 4-lane tiles.
//
// The probe order, early exit and tile evaluation are those of
// bucketed_find_kernel (Sec. V-B find). The difference is where a bucket in
// flight lives: there, in registers (32 per query set and lane), which caps
// a lane at two sets, evaluated one step after their reads are issued; here,
// in the warp's shared memory, so a lane keeps KPL sets in flight and a set
// is evaluated KPL - 1 steps after its copies were issued, with the copies of
// the newer sets still outstanding (cp.async.wait_group).
#pragma once

#include "ght_find.cuh"

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
// owner) x 8 chunks of 16 bytes. Lane r of a tile holds chunks 2r and 2r + 1
// of each of its tile's buckets; chunk c of the bucket of owner lane o is
// stored at chunk position c ^ (o >> 2 & 7), so the eight tiles of a warp
// read different bank groups.
template <int KPL>
constexpr size_t find_async_smem_per_warp() {
  return (size_t)KPL * 32 * 8 * 16;
}

template <int KPL, int WARPS, bool COUNT>
__global__ void __launch_bounds__(32 * WARPS)
bcht_find_async_kernel(TableView tv, const uint32_t *__restrict__ queries, uint32_t *__restrict__ out, uint64_t n,
                       uint64_t per_warp) {
  constexpr int B = 16, G = 4;
  static_assert(KPL >= 2 && KPL <= 8, "query sets in flight");
  extern __shared__ uint4 fa_smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int r = lane & (G - 1);
  const int tbase = lane - r;
  const unsigned swz = (unsigned)(lane >> 2) & 7u;  // this tile's chunk swizzle
  const unsigned tmask = ((1u << G) - 1u) << tbase;
  uint4 *wbuf = fa_smem + (size_t)wib * KPL * 32 * 8;
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
            out[at] = kEmptyKey;  // the sentinel is never a key
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
        uint4 *sbuf = wbuf + (size_t)s * 32 * 8;
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const int owner = tbase + j;
          const uint32_t bj = __shfl_sync(kFull, myb, owner);
          if ((act[s] >> owner) & 1u) {
            const uint64_t *src = tv.slots + (uint64_t)bj * B + 4 * r;  // 32 bytes: slots [4r, 4r + 4)
            uint4 *row = sbuf + owner * 8;
            cp_async16(row + ((2u * r) ^ swz), src);
            cp_async16(row + ((2u * r + 1u) ^ swz), src + 2);
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
        const uint4 *ebuf = wbuf + (size_t)e * 32 * 8;
        bool my_hit = false, my_emp = false;
        uint32_t my_val = kEmptyKey;
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const int owner = tbase + j;
          const uint32_t kj = __shfl_sync(kFull, key[e], owner);
          const bool aj = (act[e] >> owner) & 1u;
          bool hit = false, emp = false;
          uint32_t hv = 0u;
          if (aj) {
            const uint4 *row = ebuf + owner * 8;
            const uint4 c0 = row[(2u * r) ^ swz], c1 = row[(2u * r + 1u) ^ swz];
            const uint32_t ks[4] = {c0.x, c0.z, c1.x, c1.z}, vs[4] = {c0.y, c0.w, c1.y, c1.w};
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              if (ks[p] == kj) {
                hit = true;
                hv = vs[p];
              }
              emp |= ks[p] == kEmptyKey;
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
          uint32_t result = kEmptyKey;
          if (my_hit) {
            result = my_val;
            finish = true;
          } else if (my_emp) {
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


}  // namespace ght
