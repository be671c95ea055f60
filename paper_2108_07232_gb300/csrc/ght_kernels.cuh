// ght_kernels.cuh -- bulk build and bulk find kernels for sm_103a.
//
// Work distribution (a GB300 design, not the paper's): every lane owns one
// key (or query) at a time, drawn from its warp's contiguous slice of the
// input. A "tile" of G lanes reads one 128-byte bucket together, each lane
// B/G pairs with 16-byte vector loads. In one round every tile member's
// pending bucket is gathered back to back, so a warp keeps up to 32
// independent bucket reads in flight; the owner then decides from ballots
// over the tile (load = popcount of non-empty slots, key match), issues at
// most one 64-bit CAS or exchange, and a lane whose key is done immediately
// takes the next key of the warp's slice. The paper instead serialises a
// tile over its lanes' keys, one bucket read in flight per tile (Sec. V-A).
#pragma once

#include "ght_device.cuh"

namespace ght {

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ----------------------------------------------------------------------------
// Bucketed find. BCHT stops at the first probed bucket with an empty slot
// (Sec. V-B find; valid because keys are placed in hash order and buckets
// never lose keys). P2BHT, IHT and the load-balanced BCHT read their
// candidates in order until the key is found (Sec. V-C, V-D find).
template <int SCHEME, int B, int G, bool COUNT>
__global__ void __launch_bounds__(256)
bucketed_find_kernel(TableView tv, const uint32_t *__restrict__ queries, uint32_t *__restrict__ out,
                     uint64_t n, uint64_t per_warp) {
  constexpr int PPL = B / G;
  constexpr bool kEarlyExit = (SCHEME == kBCHT);
  static_assert(B % G == 0 && 32 % G == 0 && PPL >= 1, "tile shape");
  const int lane = threadIdx.x & 31;
  const int r = lane & (G - 1);
  const int tbase = lane - r;
  const unsigned tmask = (G == 32 ? kFull : ((1u << G) - 1u)) << tbase;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t beg = warp * per_warp;
  if (beg >= n) return;  // whole warp
  const uint64_t end = beg + per_warp < n ? beg + per_warp : n;
  const unsigned below = lanemask_lt();

  uint64_t cursor = beg, idx = 0;
  bool active = false;
  uint32_t key = 0, result = kEmptyKey;
  int probe = 0;
  unsigned long long probes = 0, answered = 0;

  for (;;) {
    const unsigned need = __ballot_sync(kFull, !active);
    if (need != 0u && cursor < end) {
      const uint64_t mine = cursor + __popc(need & below);
      if (!active && mine < end) {
        idx = mine;
        key = __ldg(queries + mine);
        result = kEmptyKey;
        probe = 0;
        if (COUNT) answered++;
        if (key == kEmptyKey) out[idx] = kEmptyKey;  // the sentinel is never a key
        else active = true;
      }
      cursor += __popc(need);
      if (cursor > end) cursor = end;
    }
    const unsigned act = __ballot_sync(kFull, active);
    if (act == 0u) {
      if (cursor >= end) break;
      continue;
    }

    const uint32_t myb = active ? bucket_of(tv.hf, probe, key) : 0u;
    uint64_t v[G][PPL];
#pragma unroll
    for (int j = 0; j < G; ++j) {
      const uint32_t bj = __shfl_sync(kFull, myb, tbase + j);
      if ((act >> (tbase + j)) & 1u) load_part_ro<PPL>(tv.slots + (uint64_t)bj * B, r, v[j]);
    }
    bool finish = false;
#pragma unroll
    for (int j = 0; j < G; ++j) {
      const uint32_t kj = __shfl_sync(kFull, key, tbase + j);
      const bool aj = (act >> (tbase + j)) & 1u;
      bool hit = false, emp = false;
      uint32_t val = kEmptyKey;
#pragma unroll
      for (int p = 0; p < PPL; ++p) {
        const uint32_t sk = pair_key(v[j][p]);
        if (aj && !hit && sk == kj) {
          hit = true;
          val = pair_value(v[j][p]);
        }
        if (aj && sk == kEmptyKey) emp = true;
      }
      const unsigned hm = __ballot_sync(kFull, hit) & tmask;
      const unsigned em = kEarlyExit ? (__ballot_sync(kFull, emp) & tmask) : 0u;
      const uint32_t fv = __shfl_sync(kFull, val, hm ? (__ffs(hm) - 1) : lane);
      if (lane == tbase + j && aj) {
        if (COUNT) probes++;
        if (hm) {
          result = fv;
          finish = true;
        } else if (kEarlyExit && em) {
          finish = true;
        } else if (++probe >= tv.h) {
          finish = true;
        }
      }
    }
    if (finish) {
      out[idx] = result;
      active = false;
    }
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

// ----------------------------------------------------------------------------
// Bucketed build. Per-lane state machine; every round reads one bucket per
// active key, then issues at most one atomic per lane.
//   BCHT (Sec. III-A, V-B): CAS into an empty slot of the current bucket; if
//     it is full, exchange with a random slot (xorshift) and continue with the
//     evicted pair at H_{(i+1) mod h}, i the lowest index with H_i equal to the
//     current bucket; fail after max_chain exchanges.
//   P2BHT (Sec. III-B, V-C): read H_0 then H_1; fail if both are full, else
//     CAS into the less loaded (ties to H_0).
//   IHT (Sec. III-C, V-D): read H_p = H_0; CAS there if it would still hold
//     fewer than t keys; else read H_s0 = H_1 and H_s1 = H_2 and CAS into the
//     less loaded (ties to H_s0); if both are full, into H_p if it has room;
//     else fail.
//   BCHT_LB (Sec. III-A, last paragraph): read all h candidates, CAS into the
//     least loaded (ties to the lowest index, the bucket it was just evicted
//     from excluded); if all are full, exchange with a random slot of that
//     bucket and continue with the evicted pair.
// A failed CAS means the slot was taken, so the owner re-reads (a "retry";
// each failure removes one empty slot for good, which bounds the retries).
template <int SCHEME, int B, int G, bool COUNT>
__global__ void __launch_bounds__(256)
bucketed_insert_kernel(TableView tv, const uint32_t *__restrict__ keys,
                       const uint32_t *__restrict__ values, uint64_t n, uint64_t per_warp) {
  constexpr int PPL = B / G;
  static_assert(B % G == 0 && 32 % G == 0 && PPL >= 1, "tile shape");
  const int lane = threadIdx.x & 31;
  const int r = lane & (G - 1);
  const int tbase = lane - r;
  const unsigned tmask = (G == 32 ? kFull : ((1u << G) - 1u)) << tbase;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t warp = gtid >> 5;
  const uint64_t beg = warp * per_warp;
  if (beg >= n) return;  // whole warp
  const uint64_t end = beg + per_warp < n ? beg + per_warp : n;
  const unsigned below = lanemask_lt();
  const int h = tv.h;

  uint32_t rng = lane_seed(tv.rng_seed, gtid);
  uint64_t cursor = beg;
  bool active = false, retrying = false;
  uint64_t pair = 0;
  uint32_t cur = 0, chain = 0, steps = 0, round = 0;
  int phase = 0;
  // remembered reads: P2BHT (l_a, s_a, b_a) = H_0; IHT a = primary, b = H_s0;
  // BCHT_LB best candidate so far in (l_a, s_a, b_a) and `from` in b_b
  int l_a = 0, s_a = -1, l_b = 0, s_b = -1;
  uint32_t b_a = 0, b_b = 0xFFFFFFFFu;
  unsigned long long probes = 0, retries = 0, evictions = 0, longest = 0;

  for (;;) {
    if ((++round & 15u) == 0u) {  // leave early once the build has failed anywhere
      uint32_t st = (lane == 0) ? load_status(tv.ctrl) : 0u;
      st = __shfl_sync(kFull, st, 0);
      if (st & (kStatusBuildFailed | kStatusTimeout | kStatusCorrupt)) break;
    }
    const unsigned need = __ballot_sync(kFull, !active);
    if (need != 0u && cursor < end) {
      const uint64_t mine = cursor + __popc(need & below);
      if (!active && mine < end) {
        const uint32_t k = __ldg(keys + mine);
        if (k == kEmptyKey) {
          atomicOr(&tv.ctrl->status, kStatusSentinel);
        } else {
          pair = ((uint64_t)__ldg(values + mine) << 32) | k;
          active = true;
          retrying = false;
          chain = 0;
          steps = 0;
          phase = 0;
          b_b = 0xFFFFFFFFu;
          l_a = B + 1;
          cur = bucket_of(tv.hf, 0, k);
        }
      }
      cursor += __popc(need);
      if (cursor > end) cursor = end;
    }
    const unsigned act = __ballot_sync(kFull, active);
    if (act == 0u) {
      if (cursor >= end) break;
      continue;
    }

    // gather one bucket per active lane of the tile
    uint64_t v[G][PPL];
#pragma unroll
    for (int j = 0; j < G; ++j) {
      const uint32_t bj = __shfl_sync(kFull, cur, tbase + j);
      if ((act >> (tbase + j)) & 1u) load_part_rw<PPL>(tv.slots + (uint64_t)bj * B, r, v[j]);
    }
    // owner learns how many slots are empty and where one of them is
    int my_empty = 0, my_slot = -1;
#pragma unroll
    for (int j = 0; j < G; ++j) {
      const bool aj = (act >> (tbase + j)) & 1u;
      int cnt = 0, slot = -1;
#pragma unroll
      for (int p = 0; p < PPL; ++p) {
        const unsigned em = __ballot_sync(kFull, aj && pair_key(v[j][p]) == kEmptyKey) & tmask;
        cnt += __popc(em);
        if (slot < 0 && em) slot = (__ffs(em) - 1 - tbase) * PPL + p;
      }
      if (lane == tbase + j) {
        my_empty = cnt;
        my_slot = slot;
      }
    }

    int op = 0;  // 1 = CAS, 2 = exchange
    uint64_t *target = nullptr;
    if (active) {
      if (COUNT) {
        if (retrying) retries++;
        else probes++;
      }
      const int load = B - my_empty;
      const uint32_t k = pair_key(pair);
      bool fail = false;
      if (++steps > tv.max_steps) {
        atomicOr(&tv.ctrl->status, kStatusTimeout);
        active = false;
      } else if (SCHEME == kBCHT) {
        if (load < B) {
          op = 1;
          target = tv.slots + (uint64_t)cur * B + my_slot;
        } else if (chain >= tv.max_chain) {
          fail = true;
        } else {
          op = 2;
          target = tv.slots + (uint64_t)cur * B + (xorshift32(rng) % B);
        }
      } else if (SCHEME == kP2BHT) {
        if (phase == 0) {
          l_a = load; s_a = my_slot; b_a = cur;
          phase = 1;
          cur = bucket_of(tv.hf, 1, k);
        } else if (l_a == B && load == B) {
          fail = true;
        } else {
          op = 1;
          target = (l_a <= load) ? tv.slots + (uint64_t)b_a * B + s_a
                                 : tv.slots + (uint64_t)cur * B + my_slot;
        }
      } else if (SCHEME == kIHT) {
        if (phase == 0) {
          l_a = load; s_a = my_slot; b_a = cur;
          if (load + 1 < tv.t) {
            op = 1;
            target = tv.slots + (uint64_t)cur * B + my_slot;
          } else {
            phase = 1;
            cur = bucket_of(tv.hf, 1, k);
          }
        } else if (phase == 1) {
          l_b = load; s_b = my_slot; b_b = cur;
          phase = 2;
          cur = bucket_of(tv.hf, 2, k);
        } else if (l_b < B || load < B) {
          op = 1;
          target = (l_b <= load) ? tv.slots + (uint64_t)b_b * B + s_b
                                 : tv.slots + (uint64_t)cur * B + my_slot;
        } else if (l_a < B) {
          op = 1;
          target = tv.slots + (uint64_t)b_a * B + s_a;
        } else {
          fail = true;
        }
      } else {  // kBCHT_LB
        if (cur != b_b && load < l_a) {
          l_a = load; s_a = my_slot; b_a = cur;
        }
        if (phase + 1 < h) {
          phase++;
          cur = bucket_of(tv.hf, phase, k);
        } else if (l_a < B) {
          op = 1;
          target = tv.slots + (uint64_t)b_a * B + s_a;
        } else if (l_a > B || chain >= tv.max_chain) {
          fail = true;  // no candidate besides the one it came from, or chain bound
        } else {
          op = 2;
          target = tv.slots + (uint64_t)b_a * B + (xorshift32(rng) % B);
        }
      }
      if (fail) {
        atomicOr(&tv.ctrl->status, kStatusBuildFailed);
        active = false;
        if (COUNT && chain > longest) longest = chain;
      }
    }

    // at most one atomic per lane; a warp issues them together
    uint64_t old = 0;
    if (op == 1) old = cas_pair(target, kEmptyPair, pair);
    else if (op == 2) old = exch_pair(target, pair);
    if (op != 0) retrying = false;

    if (op == 1) {
      if (old == kEmptyPair) {
        active = false;  // stored
        if (COUNT && chain > longest) longest = chain;
      } else {
        retrying = true;  // slot taken since the read: read again
        if (SCHEME == kP2BHT || SCHEME == kIHT || SCHEME == kBCHT_LB) {
          phase = 0;
          l_a = B + 1;
          cur = bucket_of(tv.hf, 0, pair_key(pair));
        }
      }
    } else if (op == 2) {
      if (COUNT) evictions++;
      chain++;
      if (pair_key(old) == kEmptyKey) {
        active = false;  // the slot had been emptied -- cannot happen, but storing is complete
      } else if (SCHEME == kBCHT) {
        const uint32_t from = cur;
        pair = old;
        const uint32_t k = pair_key(old);
        int i = -1;
#pragma unroll
        for (int f = 0; f < 4; ++f)
          if (f < h && i < 0 && bucket_of(tv.hf, f, k) == from) i = f;
        if (i < 0) {
          atomicOr(&tv.ctrl->status, kStatusCorrupt);
          active = false;
        } else {
          cur = bucket_of(tv.hf, (i + 1) % h, k);
        }
      } else {  // kBCHT_LB: evicted pair restarts its candidate scan, excluding b_a
        pair = old;
        b_b = b_a;
        phase = 0;
        l_a = B + 1;
        cur = bucket_of(tv.hf, 0, pair_key(old));
      }
    }
  }
  if (COUNT) {
    probes = warp_sum(probes);
    retries = warp_sum(retries);
    evictions = warp_sum(evictions);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(kFull, longest, o);
      longest = other > longest ? other : longest;
    }
    if (lane == 0) {
      atomicAdd(&tv.ctrl->insert_probes, probes);
      atomicAdd(&tv.ctrl->insert_retries, retries);
      atomicAdd(&tv.ctrl->insert_evictions, evictions);
      atomicMax(&tv.ctrl->longest_chain, longest);
    }
  }
}

// ----------------------------------------------------------------------------
// Bucket size one cuckoo ("1CHT", Sec. VII; CUDPP style): one thread per
// key, each step a single 64-bit exchange into H_i(k); a displaced pair moves
// on to H_{(i+1) mod h}. Fails once more than max_chain pairs were displaced.
template <bool COUNT>
__global__ void __launch_bounds__(256)
cuckoo1_insert_kernel(TableView tv, const uint32_t *__restrict__ keys,
                      const uint32_t *__restrict__ values, uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long probes = 0, evictions = 0, longest = 0;
  const int h = tv.h;
  uint32_t seen = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if ((++seen & 63u) == 0u && (load_status(tv.ctrl) & kStatusBuildFailed)) break;
    const uint32_t k0 = __ldg(keys + i);
    if (k0 == kEmptyKey) {
      atomicOr(&tv.ctrl->status, kStatusSentinel);
      continue;
    }
    uint64_t pair = ((uint64_t)__ldg(values + i) << 32) | k0;
    uint32_t cur = bucket_of(tv.hf, 0, k0);
    uint32_t displaced = 0;
    for (;;) {
      const uint64_t old = exch_pair(tv.slots + cur, pair);
      if (COUNT) probes++;
      if (pair_key(old) == kEmptyKey) break;
      if (COUNT) {
        evictions++;
        if (displaced + 1 > longest) longest = displaced + 1;
      }
      if (++displaced > tv.max_chain) {
        atomicOr(&tv.ctrl->status, kStatusBuildFailed);
        break;
      }
      pair = old;
      const uint32_t k = pair_key(old);
      int f0 = -1;
#pragma unroll
      for (int f = 0; f < 4; ++f)
        if (f < h && f0 < 0 && bucket_of(tv.hf, f, k) == cur) f0 = f;
      if (f0 < 0) {
        atomicOr(&tv.ctrl->status, kStatusCorrupt);
        break;
      }
      cur = bucket_of(tv.hf, (f0 + 1) % h, k);
    }
  }
  if (COUNT) {
    probes = warp_sum(probes);
    evictions = warp_sum(evictions);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(kFull, longest, o);
      longest = other > longest ? other : longest;
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&tv.ctrl->insert_probes, probes);
      atomicAdd(&tv.ctrl->insert_evictions, evictions);
      atomicMax(&tv.ctrl->longest_chain, longest);
    }
  }
}

// 1CHT find: one thread per query; H_0, H_1, ... until the key or an empty
// slot is met (an empty slot is the early exit for b = 1).
template <bool COUNT>
__global__ void __launch_bounds__(256)
cuckoo1_find_kernel(TableView tv, const uint32_t *__restrict__ queries, uint32_t *__restrict__ out,
                    uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long probes = 0, answered = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t q = __ldg(queries + i);
    uint32_t result = kEmptyKey;
    if (COUNT) answered++;
    if (q != kEmptyKey) {
      for (int f = 0; f < tv.h; ++f) {
        const uint64_t s = __ldg(reinterpret_cast<const unsigned long long *>(tv.slots) + bucket_of(tv.hf, f, q));
        if (COUNT) probes++;
        if (pair_key(s) == q) {
          result = pair_value(s);
          break;
        }
        if (pair_key(s) == kEmptyKey) break;
      }
    }
    out[i] = result;
  }
  if (COUNT) {
    probes = warp_sum(probes);
    answered = warp_sum(answered);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&tv.ctrl->find_probes, probes);
      atomicAdd(&tv.ctrl->find_queries, answered);
    }
  }
}

}  // namespace ght
