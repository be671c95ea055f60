// ght_find.cuh -- the bulk find kernel for sm_103a and the input stream it
// reads queries with.
//
// Work distribution (a GB300 design, not the paper's): every lane owns one
// query at a time, drawn from its warp's contiguous slice of the input. A
// "tile" of G lanes reads one 128-byte bucket together, each lane B/G pairs
// with 16-byte vector loads, and every tile member's bucket is gathered in one
// round, so a warp keeps up to 32 independent bucket reads in flight per
// query set. The paper instead serialises a tile over its lanes' queries, one
// bucket read in flight per tile (Sec. V-A).
#pragma once

#include "ght_device.cuh"

namespace ght {

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ----------------------------------------------------------------------------
// Input stream of a warp's slice, read 32 items at a time with one coalesced
// load and kept two chunks ahead of use, so refilling a lane never waits on
// memory. Chunk x lives in register x of lane i (entry i).
struct StreamQueue {
  uint64_t base;  // slice index of entry 0 of chunk a (warp-uniform)
  int head;       // next unused entry of chunk a (warp-uniform)
  uint32_t a, b, c;
};

__device__ __forceinline__ uint32_t stream_load(const uint32_t *__restrict__ p, uint64_t i, uint64_t end) {
  return i < end ? __ldg(p + i) : kEmptyKey;
}

__device__ __forceinline__ void stream_init(StreamQueue &q, const uint32_t *__restrict__ p, uint64_t beg,
                                            uint64_t end, int lane) {
  q.base = beg;
  q.head = 0;
  q.a = stream_load(p, beg + lane, end);
  q.b = stream_load(p, beg + 32 + lane, end);
  q.c = stream_load(p, beg + 64 + lane, end);
}

// Hand the next popc(need) entries to the lanes set in `need` (in lane
// order); returns the entry's slice index (>= end when the slice is spent).
__device__ __forceinline__ uint64_t stream_take(StreamQueue &q, const uint32_t *__restrict__ p, uint64_t end,
                                                unsigned need, unsigned below, int lane, uint32_t &item) {
  const int pos = q.head + __popc(need & below);
  const uint32_t from_a = __shfl_sync(kFull, q.a, pos & 31);
  const uint32_t from_b = __shfl_sync(kFull, q.b, pos & 31);
  item = pos < 32 ? from_a : from_b;
  const uint64_t at = q.base + (uint64_t)pos;
  q.head += __popc(need);
  if (q.head >= 32) {
    q.head -= 32;
    q.base += 32;
    q.a = q.b;
    q.b = q.c;
    q.c = stream_load(p, q.base + 64 + lane, end);
  }
  return ((need >> lane) & 1u) ? at : ~0ull;
}

// ----------------------------------------------------------------------------
// Bucketed find. BCHT stops at the first probed bucket with an empty slot
// (Sec. V-B find; valid because keys are placed in hash order and buckets
// never lose keys). P2BHT, IHT and the load-balanced BCHT read their
// candidates in order until the key is found (Sec. V-C, V-D find).
//
// Each lane owns KPL queries (sets). With KPL = 2 the sets are staggered:
// one set's bucket reads are in flight while the other set is evaluated.
// Tile members report a hit (and its value) or an empty slot to the owner
// by ballots over the tile (4-lane tiles) or through per-warp shared memory
// (wider tiles), not by one ballot per slot.
template <int SCHEME, int B, int G, int KPL, bool COUNT, typename S = PairSlot>
__global__ void __launch_bounds__(256)
bucketed_find_kernel(TableView tv, const uint32_t *__restrict__ queries, uint32_t *__restrict__ out,
                     uint64_t n, uint64_t per_warp) {
  using T = typename S::T;
  constexpr int PPL = B / G;
  const T *slots = reinterpret_cast<const T *>(tv.slots);
  constexpr bool kEarlyExit = (SCHEME == kBCHT);
  // Tile evaluation: with 4-lane tiles each owner learns its result from two
  // ballots and a shuffle per tile member (measured 1.4 % faster at 2^28
  // keys, 5-7 % at 2^24 than the shared-memory form); wider tiles report
  // through per-warp shared memory, which measured faster for them.
  constexpr bool kBallotEval = G <= 4;
  static_assert(B % G == 0 && 32 % G == 0 && PPL >= 1 && (KPL == 1 || KPL == 2), "tile shape");
  __shared__ uint32_t s_hit[8][32], s_emp[8][32], s_val[8][32];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int r = lane & (G - 1);
  const int tbase = lane - r;
  const unsigned tmask = (G == 32 ? kFull : ((1u << G) - 1u)) << tbase;
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
  T v[KPL][G][PPL];
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
      // refill set s from the stream, then issue its bucket reads
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
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const uint32_t bj = __shfl_sync(kFull, myb, tbase + j);
          if ((act[s] >> (tbase + j)) & 1u) load_slots_ro<PPL>(slots + (uint64_t)bj * B, r, v[s][j]);
        }
      }
      // evaluate the other set (or this one when KPL = 1)
      const int e = (KPL == 1) ? s : (s + 1) % KPL;
      if (act[e] != 0u) {
        if constexpr (kBallotEval) {
          // each owner learns from two ballots over its tile whether a member
          // holds its key or an empty slot, and the value by one shuffle
          bool my_hit = false, my_emp = false;
          uint32_t my_val = S::missing();
  #pragma unroll
          for (int j = 0; j < G; ++j) {
            const int owner = tbase + j;
            const uint32_t kj = __shfl_sync(kFull, key[e], owner);
            const bool aj = (act[e] >> owner) & 1u;
            bool hit = false, emp = false;
            uint32_t hv = 0u;
  #pragma unroll
            for (int p = 0; p < PPL; ++p) {
              const uint32_t sk = S::key(v[e][j][p]);
              if (sk == kj) {
                hit = true;
                hv = S::found(v[e][j][p]);
              }
              if (kEarlyExit) emp |= sk == kEmptyKey;
            }
            const unsigned hb = __ballot_sync(kFull, aj && hit) & tmask;
            const unsigned eb = kEarlyExit ? (__ballot_sync(kFull, aj && emp) & tmask) : 0u;
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
            } else if (kEarlyExit && my_emp) {
              finish = true;
            } else if (++probe[e] >= tv.h) {
              finish = true;
            }
            if (finish) {
              out[idx[e]] = result;
              active[e] = false;
            }
          }
        } else {
          s_hit[wib][lane] = 0u;
          if (kEarlyExit) s_emp[wib][lane] = 0u;
          __syncwarp();
  #pragma unroll
          for (int j = 0; j < G; ++j) {
            const int owner = tbase + j;
            const uint32_t kj = __shfl_sync(kFull, key[e], owner);
            if ((act[e] >> owner) & 1u) {
  #pragma unroll
              for (int p = 0; p < PPL; ++p) {
                const uint32_t sk = S::key(v[e][j][p]);
                if (sk == kj) {
                  s_hit[wib][owner] = 1u;
                  s_val[wib][owner] = S::found(v[e][j][p]);
                }
                if (kEarlyExit && sk == kEmptyKey) s_emp[wib][owner] = 1u;
              }
            }
          }
          __syncwarp();
          if ((act[e] >> lane) & 1u) {
            if (COUNT) probes++;
            bool finish = false;
            uint32_t result = S::missing();
            if (s_hit[wib][lane]) {
              result = s_val[wib][lane];
              finish = true;
            } else if (kEarlyExit && s_emp[wib][lane]) {
              finish = true;
            } else if (++probe[e] >= tv.h) {
              finish = true;
            }
            if (finish) {
              out[idx[e]] = result;
              active[e] = false;
            }
          }
        }
        act[e] = 0u;  // evaluated; the set's next reads are issued on its next refill
      }
    }
    bool any = false;
#pragma unroll
    for (int s = 0; s < KPL; ++s) any |= active[s];
    if (__ballot_sync(kFull, any) == 0u && sq.base + sq.head >= end) break;
  }
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
