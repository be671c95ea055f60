// ght_kernels.cuh -- bulk build kernels for sm_103a (the find kernel is in
// ght_find.cuh, included here).
//
// Work distribution (a GB300 design, not the paper's): every lane owns one
// key at a time, drawn from input chunks its warp claims. A "tile" of G
// lanes reads one 128-byte bucket together, each lane B/G slots. In one
// round every tile member's pending bucket is gathered back to back, so a
// warp keeps up to 32 independent bucket reads in flight; the owner then
// decides from ballots over the tile (load = popcount of non-empty slots),
// issues at most one 64-bit CAS or exchange, and a lane whose key is done
// immediately takes the next key. The paper instead serialises a tile over
// its lanes' keys, one bucket read in flight per tile (Sec. V-A).
#pragma once

#include "ght_device.cuh"
#include "ght_find.cuh"

namespace ght {

// ----------------------------------------------------------------------------
// Key and value streams of a build, read like StreamQueue, 32 pairs at a
// time, two chunks ahead. Chunks are either consecutive pieces of the warp's
// static slice, or (dynamic mode) claimed from a global cursor so that all
// warps advance through the input together -- which keeps the in-flight
// inserts of a grouped build inside a small window of the table.
struct PairQueue {
  uint64_t ba, bb, bc;  // input index of entry 0 of chunks a, b, c (warp-uniform)
  uint64_t claim_next;  // dynamic mode: next chunk of the warp's current claim
  uint32_t claim_left;  // chunks left in that claim
  int head;             // next unused entry of chunk a
  uint32_t ka, kb, kc, va, vb, vc;
};

// Dynamic mode: a warp claims kClaimChunks consecutive 32-pair chunks at a
// time from the global cursor (one atomic per claim, not per chunk).
constexpr uint32_t kClaimChunks = 32;

__device__ __forceinline__ uint64_t claim_chunk(PairQueue &q, Ctrl *ctrl, int lane) {
  if (q.claim_left == 0) {
    unsigned long long x = 0ull;
    if (lane == 0) x = atomicAdd(&ctrl->work_cursor, 32ull * kClaimChunks);
    q.claim_next = __shfl_sync(kFull, x, 0);
    q.claim_left = kClaimChunks;
  }
  const uint64_t at = q.claim_next;
  q.claim_next += 32;
  q.claim_left--;
  return at;
}

__device__ __forceinline__ void pair_init(PairQueue &q, const uint32_t *__restrict__ k, const uint32_t *__restrict__ v,
                                          uint64_t beg, uint64_t end, bool dynamic, Ctrl *ctrl, int lane) {
  q.claim_next = 0;
  q.claim_left = 0;
  if (dynamic) {
    q.ba = claim_chunk(q, ctrl, lane);
    q.bb = claim_chunk(q, ctrl, lane);
    q.bc = claim_chunk(q, ctrl, lane);
  } else {
    q.ba = beg;
    q.bb = beg + 32;
    q.bc = beg + 64;
  }
  q.head = 0;
  q.ka = stream_load(k, q.ba + lane, end);
  q.kb = stream_load(k, q.bb + lane, end);
  q.kc = stream_load(k, q.bc + lane, end);
  q.va = stream_load(v, q.ba + lane, end);
  q.vb = stream_load(v, q.bb + lane, end);
  q.vc = stream_load(v, q.bc + lane, end);
}

__device__ __forceinline__ bool pair_exhausted(const PairQueue &q, uint64_t end) { return q.ba + q.head >= end; }

__device__ __forceinline__ uint64_t pair_take(PairQueue &q, const uint32_t *__restrict__ k,
                                              const uint32_t *__restrict__ v, uint64_t end, bool dynamic,
                                              Ctrl *ctrl, unsigned need, unsigned below, int lane,
                                              uint32_t &key, uint32_t &val) {
  const int pos = q.head + __popc(need & below);
  const uint32_t ka = __shfl_sync(kFull, q.ka, pos & 31), kb = __shfl_sync(kFull, q.kb, pos & 31);
  const uint32_t va = __shfl_sync(kFull, q.va, pos & 31), vb = __shfl_sync(kFull, q.vb, pos & 31);
  key = pos < 32 ? ka : kb;
  val = pos < 32 ? va : vb;
  const uint64_t at = pos < 32 ? q.ba + (uint64_t)pos : q.bb + (uint64_t)(pos - 32);
  q.head += __popc(need);
  if (q.head >= 32) {
    q.head -= 32;
    q.ba = q.bb;
    q.bb = q.bc;
    q.bc = dynamic ? claim_chunk(q, ctrl, lane) : q.bc + 32;
    q.ka = q.kb;
    q.kb = q.kc;
    q.va = q.vb;
    q.vb = q.vc;
    q.kc = stream_load(k, q.bc + lane, end);
    q.vc = stream_load(v, q.bc + lane, end);
  }
  return ((need >> lane) & 1u) ? at : ~0ull;
}

// ----------------------------------------------------------------------------
// Bucketed build. Per-lane state machine; every turn of a slot reads one
// bucket per active key, then issues at most one atomic per lane.
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
//
// Each lane runs KPL independent slots. A slot's atomic result is inspected
// only on the slot's next turn, so with KPL = 2 its latency is hidden behind
// the other slot's bucket reads. per_warp = 0 selects dynamic chunks.
//
// Minimum resident blocks per SM the insert is compiled for (0: the
// compiler's choice). The insert is latency-bound, so resident warps matter:
// for 16-pair buckets read by 16 lanes with one key per lane the compiler's
// choice is 112 registers (2 blocks of 256 threads per SM), while a bound of
// 3 blocks gives 80 registers with no spills and inserts 2^28 keys 16-20 %
// faster on GB300. Most other 16-pair shapes already get 80 or fewer; the
// probe-counting build and 32-pair shapes would spill at 80.
template <int B, int G, int KPL, bool COUNT>
constexpr int insert_min_blocks() {
  return B == 16 && G == 16 && KPL == 1 && !COUNT ? 3 : 0;
}

template <int SCHEME, int B, int G, int KPL, bool COUNT, typename S = PairSlot>
__global__ void __launch_bounds__(256, insert_min_blocks<B, G, KPL, COUNT>())
bucketed_insert_kernel(TableView tv, const uint32_t *__restrict__ keys,
                       const uint32_t *__restrict__ values, uint64_t n, uint64_t per_warp) {
  using T = typename S::T;
  constexpr int PPL = B / G;
  T *slots = reinterpret_cast<T *>(tv.slots);
  static_assert(B % G == 0 && 32 % G == 0 && PPL >= 1 && (KPL == 1 || KPL == 2), "tile shape");
  const int lane = threadIdx.x & 31;
  const int r = lane & (G - 1);
  const int tbase = lane - r;
  const unsigned tmask = (G == 32 ? kFull : ((1u << G) - 1u)) << tbase;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t warp = gtid >> 5;
  const bool dynamic = per_warp == 0;
  const uint64_t beg = dynamic ? 0 : warp * per_warp;
  if (beg >= n) return;  // whole warp
  const uint64_t end = dynamic ? n : (beg + per_warp < n ? beg + per_warp : n);
  const unsigned below = lanemask_lt();
  const int h = tv.h;

  uint32_t rng = lane_seed(tv.rng_seed, gtid);
  PairQueue pq;
  pair_init(pq, keys, values, beg, end, dynamic, tv.ctrl, lane);
  // per-slot state
  bool active[KPL], retrying[KPL];
  T pair[KPL], old[KPL];
  uint32_t cur[KPL], chain[KPL], steps[KPL];
  int op[KPL], phase[KPL];
  // remembered reads: P2BHT (l_a, s_a, b_a) = H_0; IHT a = primary, b = H_s0;
  // BCHT_LB best candidate so far in (l_a, s_a, b_a) and `from` in b_b
  int l_a[KPL], s_a[KPL], l_b[KPL], s_b[KPL];
  uint32_t b_a[KPL], b_b[KPL];
#pragma unroll
  for (int s = 0; s < KPL; ++s) {
    active[s] = retrying[s] = false;
    pair[s] = old[s] = 0;
    cur[s] = chain[s] = steps[s] = 0;
    op[s] = phase[s] = 0;
    l_a[s] = l_b[s] = 0;
    s_a[s] = s_b[s] = -1;
    b_a[s] = 0;
    b_b[s] = 0xFFFFFFFFu;
  }
  unsigned long long probes = 0, retries = 0, evictions = 0, longest = 0;
  uint32_t round = 0;

  for (;;) {
    if ((++round & 15u) == 0u) {  // leave early once the build has failed anywhere
      uint32_t st = (lane == 0) ? load_status(tv.ctrl) : 0u;
      st = __shfl_sync(kFull, st, 0);
      if (st & (kStatusBuildFailed | kStatusTimeout | kStatusCorrupt)) break;
    }
#pragma unroll
    for (int s = 0; s < KPL; ++s) {
      // -- resolve the atomic this slot issued on its previous turn
      if (op[s] == 1) {
        if (old[s] == S::kEmpty) {
          active[s] = false;  // stored
          if (COUNT && chain[s] > longest) longest = chain[s];
        } else {
          retrying[s] = true;  // slot taken since the read: read again
          if (SCHEME == kP2BHT || SCHEME == kIHT || SCHEME == kBCHT_LB) {
            phase[s] = 0;
            l_a[s] = B + 1;
            cur[s] = bucket_of(tv.hf, 0, S::key(pair[s]));
          }
        }
      } else if (op[s] == 2) {
        if (COUNT) evictions++;
        chain[s]++;
        if (S::key(old[s]) == kEmptyKey) {
          active[s] = false;  // the slot had been emptied -- cannot happen, but storing is complete
        } else if (SCHEME == kBCHT) {
          const uint32_t from = cur[s];
          pair[s] = old[s];
          const uint32_t k = S::key(old[s]);
          int i = -1;
#pragma unroll
          for (int f = 0; f < 4; ++f)
            if (f < h && i < 0 && bucket_of(tv.hf, f, k) == from) i = f;
          if (i < 0) {
            atomicOr(&tv.ctrl->status, kStatusCorrupt);
            active[s] = false;
          } else {
            cur[s] = bucket_of(tv.hf, (i + 1) % h, k);
          }
        } else {  // kBCHT_LB: evicted pair restarts its candidate scan, excluding b_a
          pair[s] = old[s];
          b_b[s] = b_a[s];
          phase[s] = 0;
          l_a[s] = B + 1;
          cur[s] = bucket_of(tv.hf, 0, S::key(old[s]));
        }
      }
      op[s] = 0;

      // -- refill
      const unsigned need = __ballot_sync(kFull, !active[s]);
      if (need != 0u && !pair_exhausted(pq, end)) {
        uint32_t k, val;
        const uint64_t at = pair_take(pq, keys, values, end, dynamic, tv.ctrl, need, below, lane, k, val);
        if (at < end) {
          if (k == kEmptyKey) {
            atomicOr(&tv.ctrl->status, kStatusSentinel);
          } else {
            pair[s] = S::make(k, val);
            active[s] = true;
            retrying[s] = false;
            chain[s] = 0;
            steps[s] = 0;
            phase[s] = 0;
            b_b[s] = 0xFFFFFFFFu;
            l_a[s] = B + 1;
            cur[s] = bucket_of(tv.hf, SCHEME == kBCHT ? tv.first : 0, k);
          }
        }
      }
      const unsigned act = __ballot_sync(kFull, active[s]);
      if (act == 0u) continue;

      // -- gather the keys of one bucket per active lane of the tile
      uint32_t v[G][PPL];
#pragma unroll
      for (int j = 0; j < G; ++j) {
        const uint32_t bj = __shfl_sync(kFull, cur[s], tbase + j);
        if ((act >> (tbase + j)) & 1u) load_keys_rw<PPL>(slots + (uint64_t)bj * B, r, v[j]);
      }
      // owner learns how many slots are empty and where one of them is
      int my_empty = 0, my_slot = -1;
#pragma unroll
      for (int j = 0; j < G; ++j) {
        const bool aj = (act >> (tbase + j)) & 1u;
        int cnt = 0, slot = -1;
#pragma unroll
        for (int p = 0; p < PPL; ++p) {
          const unsigned em = __ballot_sync(kFull, aj && v[j][p] == kEmptyKey) & tmask;
          cnt += __popc(em);
          if (slot < 0 && em) slot = (__ffs(em) - 1 - tbase) * PPL + p;
        }
        if (lane == tbase + j) {
          my_empty = cnt;
          my_slot = slot;
        }
      }

      // -- decide and issue this slot's atomic
      T *target = nullptr;
      if (active[s]) {
        if (COUNT) {
          if (retrying[s]) retries++;
          else probes++;
        }
        const int load = B - my_empty;
        const uint32_t k = S::key(pair[s]);
        bool fail = false;
        if (++steps[s] > tv.max_steps) {
          atomicOr(&tv.ctrl->status, kStatusTimeout);
          active[s] = false;
        } else if (SCHEME == kBCHT) {
          if (load < B) {
            op[s] = 1;
            target = slots + (uint64_t)cur[s] * B + my_slot;
          } else if (chain[s] >= tv.max_chain) {
            fail = true;
          } else {
            op[s] = 2;
            target = slots + (uint64_t)cur[s] * B + (xorshift32(rng) % B);
          }
        } else if (SCHEME == kP2BHT) {
          if (phase[s] == 0) {
            l_a[s] = load; s_a[s] = my_slot; b_a[s] = cur[s];
            phase[s] = 1;
            cur[s] = bucket_of(tv.hf, 1, k);
          } else if (l_a[s] == B && load == B) {
            fail = true;
          } else {
            op[s] = 1;
            target = (l_a[s] <= load) ? slots + (uint64_t)b_a[s] * B + s_a[s]
                                      : slots + (uint64_t)cur[s] * B + my_slot;
          }
        } else if (SCHEME == kIHT) {
          if (phase[s] == 0) {
            l_a[s] = load; s_a[s] = my_slot; b_a[s] = cur[s];
            if (load + 1 < tv.t) {
              op[s] = 1;
              target = slots + (uint64_t)cur[s] * B + my_slot;
            } else {
              phase[s] = 1;
              cur[s] = bucket_of(tv.hf, 1, k);
            }
          } else if (phase[s] == 1) {
            l_b[s] = load; s_b[s] = my_slot; b_b[s] = cur[s];
            phase[s] = 2;
            cur[s] = bucket_of(tv.hf, 2, k);
          } else if (l_b[s] < B || load < B) {
            op[s] = 1;
            target = (l_b[s] <= load) ? slots + (uint64_t)b_b[s] * B + s_b[s]
                                      : slots + (uint64_t)cur[s] * B + my_slot;
          } else if (l_a[s] < B) {
            op[s] = 1;
            target = slots + (uint64_t)b_a[s] * B + s_a[s];
          } else {
            fail = true;
          }
        } else {  // kBCHT_LB
          if (cur[s] != b_b[s] && load < l_a[s]) {
            l_a[s] = load; s_a[s] = my_slot; b_a[s] = cur[s];
          }
          if (phase[s] + 1 < h) {
            phase[s]++;
            cur[s] = bucket_of(tv.hf, phase[s], k);
          } else if (l_a[s] < B) {
            op[s] = 1;
            target = slots + (uint64_t)b_a[s] * B + s_a[s];
          } else if (l_a[s] > B || chain[s] >= tv.max_chain) {
            fail = true;  // no candidate besides the one it came from, or chain bound
          } else {
            op[s] = 2;
            target = slots + (uint64_t)b_a[s] * B + (xorshift32(rng) % B);
          }
        }
        if (fail) {
          atomicOr(&tv.ctrl->status, kStatusBuildFailed);
          active[s] = false;
          if (COUNT && chain[s] > longest) longest = chain[s];
        }
      }
      // at most one atomic per lane; a warp issues them together and the
      // results are read on the slot's next turn
      if (op[s] == 1) old[s] = cas_slot<T>(target, S::kEmpty, pair[s]);
      else if (op[s] == 2) old[s] = exch_slot<T>(target, pair[s]);
      if (op[s] != 0) retrying[s] = false;
    }
    bool any = false;
#pragma unroll
    for (int s = 0; s < KPL; ++s) any |= active[s];
    if (__ballot_sync(kFull, any) == 0u && pair_exhausted(pq, end)) break;
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
// Ranked first-choice placement: phase 1 of a two-phase BCHT build.
//
// Sequential BCHT (Sec. III-A) may insert the keys in any order. Take the
// order in which, first, every key that arrives at its first-choice bucket
// H_0 while that bucket still has room is inserted, and then all other keys.
// In the first part no bucket is ever full, so each insert is one probe that
// takes the next free slot of H_0 -- and the slot is known without reading
// the bucket: it is the key's arrival rank at H_0. This kernel counts
// arrivals per bucket with one atomic increment on a per-bucket counter
// (4 bytes per bucket, small enough to stay in L2), stores a key of rank
// r < B straight into slot r, and appends keys of rank >= B to an overflow
// list; the overflow keys are then inserted by the BCHT insert kernel, whose
// first probe finds H_0 full and evicts as Sec. V-B prescribes. The table must
// be filled with empty slots and the counters zeroed before the launch.
//
// Blocks claim input tiles from a cursor in the control block (zeroed by the
// fill), so all blocks advance through the input together: on pairs grouped
// by first-choice bucket range, the stores and counter increments in flight
// then stay inside a few MB of the table, whose lines fill up in L2 and
// leave it once, whole. Overflow keys are staged per block in shared memory
// and appended to the list one block tile at a time with a single global
// reservation on the control block's overflow count; entries past `cap` are
// not written (the caller sees the count exceed cap and builds the ordinary
// way). With region > 0 the input is grouped into regions of `region` items
// and only [g * region, ends[g]) of group g's region holds pairs.
constexpr int kPlacePerThread = 4;
constexpr int kPlaceTile = 256 * kPlacePerThread;

template <int B, bool COUNT, typename S = PairSlot>
__global__ void __launch_bounds__(256)
rank_place_kernel(TableView tv, const uint32_t *__restrict__ keys, const uint32_t *__restrict__ values,
                  uint64_t n, uint32_t *__restrict__ counters, uint32_t *__restrict__ ovf_k,
                  uint32_t *__restrict__ ovf_v, uint64_t cap, const uint32_t *__restrict__ ends, uint32_t region,
                  uint64_t region_M) {
  using T = typename S::T;
  T *slots = reinterpret_cast<T *>(tv.slots);
  unsigned long long *ovf_count = &tv.ctrl->reserved[0];
  unsigned long long *tile_cursor = &tv.ctrl->reserved[1];
  __shared__ uint32_t s_k[2 * kPlaceTile], s_v[2 * kPlaceTile];
  __shared__ uint32_t s_n;
  __shared__ unsigned long long s_base, s_tile[2];
  const int lane = threadIdx.x & 31;
  const unsigned below = lanemask_lt();
  if (threadIdx.x == 0) {
    s_n = 0u;
    s_tile[0] = atomicAdd(tile_cursor, (unsigned long long)kPlaceTile);
  }
  __syncthreads();
  unsigned long long placed = 0;
  // Tile i is s_tile[i & 1]; thread 0 claims tile i + 1 into the other entry
  // while tile i is processed (that entry was last read before the barrier
  // that ended tile i - 1). s_n is bumped while a tile is processed, read
  // after barrier (A) and reset inside a flush.
  for (int it = 0;; it ^= 1) {
    const uint64_t t0 = s_tile[it];
    if (t0 >= n) break;  // block-uniform
    if (threadIdx.x == 0) s_tile[it ^ 1] = atomicAdd(tile_cursor, (unsigned long long)kPlaceTile);
    uint32_t k[kPlacePerThread], v[kPlacePerThread], b[kPlacePerThread], r[kPlacePerThread];
    bool ok[kPlacePerThread];
#pragma unroll
    for (int u = 0; u < kPlacePerThread; ++u) {
      const uint64_t i = t0 + (uint64_t)u * blockDim.x + threadIdx.x;  // coalesced
      ok[u] = i < n;
      if (region && ok[u]) ok[u] = (uint32_t)i < __ldg(ends + __umul64hi(region_M, i));  // within its group's pairs
      k[u] = ok[u] ? __ldg(keys + i) : kEmptyKey;
      v[u] = ok[u] ? __ldg(values + i) : 0u;
      if (ok[u] && k[u] == kEmptyKey) {
        atomicOr(&tv.ctrl->status, kStatusSentinel);
        ok[u] = false;
      }
    }
#pragma unroll
    for (int u = 0; u < kPlacePerThread; ++u) {
      b[u] = ok[u] ? bucket_of(tv.hf, 0, k[u]) : 0u;
      r[u] = ok[u] ? atomicAdd(counters + b[u], 1u) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kPlacePerThread; ++u) {
      const bool fits = ok[u] && r[u] < (uint32_t)B;
      if (fits) slots[(uint64_t)b[u] * B + r[u]] = S::make(k[u], v[u]);
      if (COUNT && ok[u]) placed++;  // a visit of H_0, stored or not (the overflow insert starts at H_1)
      // overflow: one shared reservation per warp (< 2 * kPlaceTile entries
      // are staged: they are flushed below once above one tile)
      const unsigned over = __ballot_sync(kFull, ok[u] && !fits);
      if (over) {
        uint32_t at = 0;
        if (lane == 0) at = atomicAdd(&s_n, (uint32_t)__popc(over));
        at = __shfl_sync(kFull, at, 0) + __popc(over & below);
        if ((over >> lane) & 1u) {
          s_k[at] = k[u];
          s_v[at] = v[u];
        }
      }
    }
    __syncthreads();  // (A)
    const uint32_t staged = s_n;
    const bool last = s_tile[it ^ 1] >= n;  // no further tile for this block
    if (staged > (uint32_t)kPlaceTile || (last && staged > 0u)) {
      if (threadIdx.x == 0) s_base = atomicAdd(ovf_count, (unsigned long long)staged);
      __syncthreads();
      const unsigned long long base = s_base;
      for (uint32_t i = threadIdx.x; i < staged; i += blockDim.x) {
        if (base + i < cap) {
          ovf_k[base + i] = s_k[i];
          ovf_v[base + i] = s_v[i];
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) s_n = 0u;
    }
    __syncthreads();
  }
  if (COUNT) {
    placed = warp_sum(placed);
    if ((threadIdx.x & 31) == 0 && placed) atomicAdd(&tv.ctrl->insert_probes, placed);
  }
}

// ----------------------------------------------------------------------------
// Bucket size one cuckoo ("1CHT", Sec. VII; CUDPP style): one thread per
// key, each step a single 64-bit exchange into H_i(k); a displaced pair moves
// on to H_{(i+1) mod h}. With b = 1 the exchange is also the bucket read.
// Sec. III-A fails an insert once the maximum number of exchanges has been
// made and the next bucket is full: so after max_chain displacements the
// next step is a CAS into an empty slot, and a full slot there fails the
// build without displacing another pair.
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
      const bool at_bound = displaced >= tv.max_chain;
      const uint64_t old = at_bound ? cas_pair(tv.slots + cur, kEmptyPair, pair) : exch_pair(tv.slots + cur, pair);
      if (COUNT) probes++;
      if (pair_key(old) == kEmptyKey) break;
      if (at_bound) {
        atomicOr(&tv.ctrl->status, kStatusBuildFailed);
        break;
      }
      ++displaced;
      if (COUNT) {
        evictions++;
        if (displaced > longest) longest = displaced;
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
