// kern_batch.cu -- many independent BCHT tables built and queried by single
// launches (the batched form; the paper builds one table at a time).
//
// All tables live in one allocation, each with a descriptor (slots, bucket
// count, hash constants, status word). Keys, values and queries of all tables
// are concatenated; key_offs / query_offs (T+1 entries) give each table's
// range. Work is split over warps exactly as in the single-table kernels; a
// lane finds the table of the item it takes from a per-chunk hint (one
// uniform binary search per 32 items) and reads that table's descriptor.
#include "ght_batch.h"
#include "ght_find_async.cuh"
#include "ght_kernels.cuh"

namespace ght {

// First table whose range contains index i (uniform search over [lo, hi)).
__device__ __forceinline__ uint32_t table_of(const uint64_t *__restrict__ offs, uint32_t lo, uint32_t hi,
                                             uint64_t i) {
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(offs + mid) <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t advance_table(const uint64_t *__restrict__ offs, uint32_t tb, uint32_t t_hi,
                                                  uint64_t i) {
  while (tb + 1 < t_hi && __ldg(offs + tb + 1) <= i) ++tb;
  return tb;
}

__device__ __forceinline__ uint32_t batch_bucket(const BatchTable &d, int i, uint32_t k) {
  return fastmod(mod_prime((uint64_t)select4(d.a, i) * k + select4(d.c, i)), d.mod);
}

// Input stream of a warp's slice with the table of each chunk's first item.
struct BatchQueue {
  uint64_t base;
  int head;
  uint32_t ta, tb, tc;  // table hint of chunks a, b, c (warp-uniform)
  uint32_t ka, kb, kc, va, vb, vc;
};

template <bool PAIRS>
__device__ __forceinline__ void bq_load(uint32_t &k, uint32_t &v, uint32_t &t, const uint32_t *__restrict__ keys,
                                        const uint32_t *__restrict__ vals, uint64_t at, uint64_t end,
                                        const BatchView &bv, const uint64_t *__restrict__ offs, int lane) {
  k = stream_load(keys, at + lane, end);
  if (PAIRS) v = stream_load(vals, at + lane, end);
  t = at < end ? table_of(offs, bv.t_lo, bv.t_hi, at) : bv.t_lo;
}

template <bool PAIRS>
__device__ __forceinline__ uint64_t bq_take(BatchQueue &q, const uint32_t *__restrict__ keys,
                                            const uint32_t *__restrict__ vals, uint64_t end, const BatchView &bv,
                                            const uint64_t *__restrict__ offs, unsigned need, unsigned below,
                                            int lane, uint32_t &key, uint32_t &val, uint32_t &table) {
  const int pos = q.head + __popc(need & below);
  const uint32_t ka = __shfl_sync(kFull, q.ka, pos & 31), kb = __shfl_sync(kFull, q.kb, pos & 31);
  key = pos < 32 ? ka : kb;
  if (PAIRS) {
    const uint32_t va = __shfl_sync(kFull, q.va, pos & 31), vb = __shfl_sync(kFull, q.vb, pos & 31);
    val = pos < 32 ? va : vb;
  }
  const uint64_t at = q.base + (uint64_t)pos;
  table = pos < 32 ? q.ta : q.tb;
  q.head += __popc(need);
  if (q.head >= 32) {
    q.head -= 32;
    q.base += 32;
    q.ka = q.kb;
    q.kb = q.kc;
    q.va = q.vb;
    q.vb = q.vc;
    q.ta = q.tb;
    q.tb = q.tc;
    bq_load<PAIRS>(q.kc, q.vc, q.tc, keys, vals, q.base + 64, end, bv, offs, lane);
  }
  if (!((need >> lane) & 1u) || at >= end) return ~0ull;
  table = advance_table(offs, table, bv.t_hi, at);
  return at;
}

template <bool PAIRS>
__device__ __forceinline__ void bq_init(BatchQueue &q, const uint32_t *__restrict__ keys,
                                        const uint32_t *__restrict__ vals, uint64_t beg, uint64_t end,
                                        const BatchView &bv, const uint64_t *__restrict__ offs, int lane) {
  q.base = beg;
  q.head = 0;
  bq_load<PAIRS>(q.ka, q.va, q.ta, keys, vals, beg, end, bv, offs, lane);
  bq_load<PAIRS>(q.kb, q.vb, q.tb, keys, vals, beg + 32, end, bv, offs, lane);
  bq_load<PAIRS>(q.kc, q.vc, q.tc, keys, vals, beg + 64, end, bv, offs, lane);
}

// Key/value stream of the batched insert: 32-pair chunks claimed from the
// batch's work cursor (runs of kClaimChunks chunks per claim, as in the
// single-table insert), each with the table of its first pair, kept two
// chunks ahead of use.
struct BatchClaimQueue {
  uint64_t ba, bb, bc;  // index of entry 0 of chunks a, b, c (warp-uniform)
  uint64_t claim_next;  // next chunk of the warp's current claim
  uint32_t claim_left;  // chunks left in that claim
  int head;             // next unused entry of chunk a
  uint32_t ta, tb, tc;  // table of each chunk's first pair
  uint32_t ka, kb, kc, va, vb, vc;
};

__device__ __forceinline__ uint64_t bc_claim(BatchClaimQueue &q, Ctrl *ctrl, uint64_t lo, int lane) {
  if (q.claim_left == 0) {
    unsigned long long x = 0ull;
    if (lane == 0) x = atomicAdd(&ctrl->work_cursor, 32ull * kClaimChunks);
    q.claim_next = lo + __shfl_sync(kFull, x, 0);
    q.claim_left = kClaimChunks;
  }
  const uint64_t at = q.claim_next;
  q.claim_next += 32;
  q.claim_left--;
  return at;
}

__device__ __forceinline__ void bc_init(BatchClaimQueue &q, const uint32_t *__restrict__ keys,
                                        const uint32_t *__restrict__ vals, uint64_t lo, uint64_t hi,
                                        const BatchView &bv, const uint64_t *__restrict__ offs, int lane) {
  q.claim_next = 0;
  q.claim_left = 0;
  q.head = 0;
  q.ba = bc_claim(q, bv.ctrl, lo, lane);
  q.bb = bc_claim(q, bv.ctrl, lo, lane);
  q.bc = bc_claim(q, bv.ctrl, lo, lane);
  bq_load<true>(q.ka, q.va, q.ta, keys, vals, q.ba, hi, bv, offs, lane);
  bq_load<true>(q.kb, q.vb, q.tb, keys, vals, q.bb, hi, bv, offs, lane);
  bq_load<true>(q.kc, q.vc, q.tc, keys, vals, q.bc, hi, bv, offs, lane);
}

// Hand the next popc(need) pairs to the lanes in `need`; returns the pair's
// index (~0 for lanes without one) and its table.
__device__ __forceinline__ uint64_t bc_take(BatchClaimQueue &q, const uint32_t *__restrict__ keys,
                                            const uint32_t *__restrict__ vals, uint64_t lo, uint64_t hi,
                                            const BatchView &bv, const uint64_t *__restrict__ offs, unsigned need,
                                            unsigned below, int lane, uint32_t &key, uint32_t &val, uint32_t &table) {
  const int pos = q.head + __popc(need & below);
  const uint32_t ka = __shfl_sync(kFull, q.ka, pos & 31), kb = __shfl_sync(kFull, q.kb, pos & 31);
  const uint32_t va = __shfl_sync(kFull, q.va, pos & 31), vb = __shfl_sync(kFull, q.vb, pos & 31);
  key = pos < 32 ? ka : kb;
  val = pos < 32 ? va : vb;
  const uint64_t at = pos < 32 ? q.ba + (uint64_t)pos : q.bb + (uint64_t)(pos - 32);
  table = pos < 32 ? q.ta : q.tb;
  q.head += __popc(need);
  if (q.head >= 32) {
    q.head -= 32;
    q.ba = q.bb;
    q.bb = q.bc;
    q.bc = bc_claim(q, bv.ctrl, lo, lane);
    q.ka = q.kb;
    q.kb = q.kc;
    q.va = q.vb;
    q.vb = q.vc;
    q.ta = q.tb;
    q.tb = q.tc;
    bq_load<true>(q.kc, q.vc, q.tc, keys, vals, q.bc, hi, bv, offs, lane);
  }
  if (!((need >> lane) & 1u) || at >= hi) return ~0ull;
  table = advance_table(offs, table, bv.t_hi, at);
  return at;
}

// ----------------------------------------------------------------------------
// Fill the slots of tables [t_lo, t_hi) and clear their status words.
__global__ void __launch_bounds__(256) batch_fill_kernel(BatchView bv, uint4 *__restrict__ slots16, uint64_t n16) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint4 e = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) slots16[i] = e;
  for (uint64_t t = bv.t_lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < bv.t_hi; t += stride)
    bv.tables[t].status = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) bv.ctrl->work_cursor = 0ull;  // the insert's claims start at zero
}

// ----------------------------------------------------------------------------
// BCHT bulk build of every table in [t_lo, t_hi) (Sec. III-A, V-B), with the
// turn structure, chunk claims (the batch's work cursor, zeroed by the fill),
// key-word gathers and register bound of the single-table insert kernel.
template <int G, int KPL, bool COUNT>
__global__ void __launch_bounds__(256, insert_min_blocks<16, G, KPL, COUNT>())
batch_insert_kernel(BatchView bv, const uint32_t *__restrict__ keys, const uint32_t *__restrict__ values) {
  constexpr int B = 16;
  constexpr int PPL = B / G;
  static_assert(B % G == 0 && 32 % G == 0 && (KPL == 1 || KPL == 2), "tile shape");
  const uint64_t *offs = bv.key_offs;
  const int lane = threadIdx.x & 31;
  const int r = lane & (G - 1);
  const int tbase = lane - r;
  const unsigned tmask = (G == 32 ? kFull : ((1u << G) - 1u)) << tbase;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t lo = __ldg(offs + bv.t_lo), hi = __ldg(offs + bv.t_hi);
  const unsigned below = lanemask_lt();
  const int h = bv.h;

  uint32_t rng = lane_seed(bv.rng_seed, gtid);
  BatchClaimQueue q;
  bc_init(q, keys, values, lo, hi, bv, offs, lane);
  bool active[KPL], retrying[KPL];
  uint64_t pair[KPL], old[KPL];
  uint32_t cur[KPL], chain[KPL], steps[KPL], tab[KPL];
  int op[KPL];
#pragma unroll
  for (int s = 0; s < KPL; ++s) {
    active[s] = retrying[s] = false;
    pair[s] = old[s] = 0;
    cur[s] = chain[s] = steps[s] = tab[s] = 0;
    op[s] = 0;
  }
  unsigned long long probes = 0, retries = 0, evictions = 0;

  for (;;) {
#pragma unroll
    for (int s = 0; s < KPL; ++s) {
      // -- resolve the atomic this slot issued on its previous turn
      if (op[s] == 1) {
        if (old[s] == kEmptyPair) active[s] = false;
        else retrying[s] = true;
      } else if (op[s] == 2) {
        if (COUNT) evictions++;
        chain[s]++;
        if (pair_key(old[s]) == kEmptyKey) {
          active[s] = false;
        } else {
          const BatchTable &d = bv.tables[tab[s]];
          const uint32_t from = cur[s], k = pair_key(old[s]);
          pair[s] = old[s];
          int i = -1;
#pragma unroll
          for (int f = 0; f < 4; ++f)
            if (f < h && i < 0 && batch_bucket(d, f, k) == from) i = f;
          if (i < 0) {
            atomicOr(&bv.tables[tab[s]].status, kStatusCorrupt);
            active[s] = false;
          } else {
            cur[s] = batch_bucket(d, (i + 1) % h, k);
          }
        }
      }
      op[s] = 0;
      // -- refill
      const unsigned need = __ballot_sync(kFull, !active[s]);
      if (need != 0u && q.ba + q.head < hi) {
        uint32_t k, val, tb;
        const uint64_t at = bc_take(q, keys, values, lo, hi, bv, offs, need, below, lane, k, val, tb);
        if (at != ~0ull) {
          if (k == kEmptyKey) {
            atomicOr(&bv.tables[tb].status, kStatusSentinel);
          } else {
            pair[s] = ((uint64_t)val << 32) | k;
            tab[s] = tb;
            active[s] = true;
            retrying[s] = false;
            chain[s] = steps[s] = 0;
            cur[s] = batch_bucket(bv.tables[tb], 0, k);
          }
        }
      }
      const unsigned act = __ballot_sync(kFull, active[s]);
      if (act == 0u) continue;
      // -- gather: each member's bucket address (its own table)
      uint64_t *myb = active[s] ? bv.tables[tab[s]].slots + (uint64_t)cur[s] * B : nullptr;
      uint32_t v[G][PPL];  // key words only: emptiness is all an insert reads
#pragma unroll
      for (int j = 0; j < G; ++j) {
        uint64_t *bj = reinterpret_cast<uint64_t *>(__shfl_sync(kFull, reinterpret_cast<uintptr_t>(myb), tbase + j));
        if ((act >> (tbase + j)) & 1u)
          load_keys_rw<PPL>(reinterpret_cast<const unsigned long long *>(bj), r, v[j]);
      }
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
      uint64_t *target = nullptr;
      if (active[s]) {
        if (COUNT) {
          if (retrying[s]) retries++;
          else probes++;
        }
        if (++steps[s] > bv.max_steps) {
          atomicOr(&bv.tables[tab[s]].status, kStatusTimeout);
          active[s] = false;
        } else if (my_empty > 0) {
          op[s] = 1;
          target = myb + my_slot;
        } else if (chain[s] >= bv.max_chain) {
          atomicOr(&bv.tables[tab[s]].status, kStatusBuildFailed);
          active[s] = false;
        } else {
          op[s] = 2;
          target = myb + (xorshift32(rng) % B);
        }
      }
      if (op[s] == 1) old[s] = cas_pair(target, kEmptyPair, pair[s]);
      else if (op[s] == 2) old[s] = exch_pair(target, pair[s]);
      if (op[s] != 0) retrying[s] = false;
    }
    bool any = false;
#pragma unroll
    for (int s = 0; s < KPL; ++s) any |= active[s];
    if (__ballot_sync(kFull, any) == 0u && q.ba + q.head >= hi) break;
  }
  if (COUNT) {
    probes = warp_sum(probes);
    retries = warp_sum(retries);
    evictions = warp_sum(evictions);
    if (lane == 0) {
      atomicAdd(&bv.ctrl->insert_probes, probes);
      atomicAdd(&bv.ctrl->insert_retries, retries);
      atomicAdd(&bv.ctrl->insert_evictions, evictions);
    }
  }
}

// ----------------------------------------------------------------------------
// BCHT bulk find over tables [t_lo, t_hi) (Sec. V-B find, early exit), with
// the structure of the single-table find kernel.
template <int G, int KPL, bool COUNT>
__global__ void __launch_bounds__(256)
batch_find_kernel(BatchView bv, const uint32_t *__restrict__ queries, uint32_t *__restrict__ out,
                  uint64_t per_warp) {
  constexpr int B = 16;
  constexpr int PPL = B / G;
  static_assert(B % G == 0 && 32 % G == 0 && (KPL == 1 || KPL == 2), "tile shape");
  __shared__ uint32_t s_hit[8][32], s_emp[8][32], s_val[8][32];
  const uint64_t *offs = bv.query_offs;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int r = lane & (G - 1);
  const int tbase = lane - r;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t lo = __ldg(offs + bv.t_lo), hi = __ldg(offs + bv.t_hi);
  const uint64_t beg = lo + (gtid >> 5) * per_warp;
  if (beg >= hi) return;
  const uint64_t end = beg + per_warp < hi ? beg + per_warp : hi;
  const unsigned below = lanemask_lt();

  BatchQueue q;
  bq_init<false>(q, queries, nullptr, beg, end, bv, offs, lane);
  bool active[KPL];
  uint32_t key[KPL], act[KPL], tab[KPL];
  uint64_t idx[KPL];
  int probe[KPL];
  uint64_t v[KPL][G][PPL];
#pragma unroll
  for (int s = 0; s < KPL; ++s) {
    active[s] = false;
    key[s] = kEmptyKey;
    act[s] = tab[s] = 0u;
    idx[s] = 0;
    probe[s] = 0;
  }
  unsigned long long probes = 0, answered = 0;

  for (;;) {
#pragma unroll
    for (int s = 0; s < KPL; ++s) {
      const unsigned need = __ballot_sync(kFull, !active[s]);
      if (need != 0u && q.base + q.head < end) {
        uint32_t k, unused, tb;
        const uint64_t at = bq_take<false>(q, queries, nullptr, end, bv, offs, need, below, lane, k, unused, tb);
        if (at != ~0ull) {
          if (COUNT) answered++;
          if (k == kEmptyKey) {
            out[at] = kEmptyKey;
          } else {
            active[s] = true;
            key[s] = k;
            idx[s] = at;
            tab[s] = tb;
            probe[s] = 0;
          }
        }
      }
      act[s] = __ballot_sync(kFull, active[s]);
      if (act[s] != 0u) {
        const uint64_t *myb =
            active[s] ? bv.tables[tab[s]].slots + (uint64_t)batch_bucket(bv.tables[tab[s]], probe[s], key[s]) * B
                      : nullptr;
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const uint64_t *bj =
              reinterpret_cast<const uint64_t *>(__shfl_sync(kFull, reinterpret_cast<uintptr_t>(myb), tbase + j));
          if ((act[s] >> (tbase + j)) & 1u) load_part_ro<PPL>(bj, r, v[s][j]);
        }
      }
      const int e = (KPL == 1) ? s : (s + 1) % KPL;
      if (act[e] != 0u) {
        s_hit[wib][lane] = 0u;
        s_emp[wib][lane] = 0u;
        __syncwarp();
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const int owner = tbase + j;
          const uint32_t kj = __shfl_sync(kFull, key[e], owner);
          if ((act[e] >> owner) & 1u) {
#pragma unroll
            for (int p = 0; p < PPL; ++p) {
              const uint32_t sk = pair_key(v[e][j][p]);
              if (sk == kj) {
                s_hit[wib][owner] = 1u;
                s_val[wib][owner] = pair_value(v[e][j][p]);
              }
              if (sk == kEmptyKey) s_emp[wib][owner] = 1u;
            }
          }
        }
        __syncwarp();
        if ((act[e] >> lane) & 1u) {
          if (COUNT) probes++;
          bool finish = false;
          uint32_t result = kEmptyKey;
          if (s_hit[wib][lane]) {
            result = s_val[wib][lane];
            finish = true;
          } else if (s_emp[wib][lane] || ++probe[e] >= bv.h) {
            finish = true;
          }
          if (finish) {
            out[idx[e]] = result;
            active[e] = false;
          }
        }
        act[e] = 0u;
      }
    }
    bool any = false;
#pragma unroll
    for (int s = 0; s < KPL; ++s) any |= active[s];
    if (__ballot_sync(kFull, any) == 0u && q.base + q.head >= end) break;
  }
  if (COUNT) {
    probes = warp_sum(probes);
    answered = warp_sum(answered);
    if (lane == 0) {
      atomicAdd(&bv.ctrl->find_probes, probes);
      atomicAdd(&bv.ctrl->find_queries, answered);
    }
  }
}

// ----------------------------------------------------------------------------
// The same find with the bucket parts staged in shared memory (the staged
// find of the single-table path, ght_find_async.cuh): 4-lane tiles, KPL
// query sets per lane in flight, each set's buckets copied by cp.async (two
// 16-byte chunks per lane and tile member, chunk positions swizzled by tile)
// and evaluated KPL - 1 steps after its copies were issued. A query's table
// comes with it from the batch queue; its bucket address from the table's
// descriptor. The tables of a batch are each small but are queried all at
// once, so together their slots exceed the L2 and the reads go to DRAM,
// where the deeper pipeline pays.
template <int KPL, int WARPS, bool COUNT>
__global__ void __launch_bounds__(32 * WARPS)
batch_find_async_kernel(BatchView bv, const uint32_t *__restrict__ queries, uint32_t *__restrict__ out,
                        uint64_t per_warp) {
  constexpr int G = 4;
  constexpr int kChunks = 8;  // 16-byte chunks per 16-pair bucket
  extern __shared__ uint4 bfa_smem[];
  const uint64_t *offs = bv.query_offs;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int r = lane & (G - 1);
  const int tbase = lane - r;
  const unsigned swz = (unsigned)(lane >> 2) & 7u;
  const unsigned tmask = ((1u << G) - 1u) << tbase;
  uint4 *wbuf = bfa_smem + (size_t)wib * KPL * 32 * kChunks;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t lo = __ldg(offs + bv.t_lo), hi = __ldg(offs + bv.t_hi);
  const uint64_t beg = lo + (gtid >> 5) * per_warp;
  if (beg >= hi) return;  // whole warp
  const uint64_t end = beg + per_warp < hi ? beg + per_warp : hi;
  const unsigned below = lanemask_lt();

  BatchQueue q;
  bq_init<false>(q, queries, nullptr, beg, end, bv, offs, lane);
  bool active[KPL];
  uint32_t key[KPL], act[KPL], tab[KPL];
  uint64_t idx[KPL];
  int probe[KPL];
#pragma unroll
  for (int s = 0; s < KPL; ++s) {
    active[s] = false;
    key[s] = kEmptyKey;
    act[s] = tab[s] = 0u;
    idx[s] = 0;
    probe[s] = 0;
  }
  unsigned long long probes = 0, answered = 0;

  for (;;) {
#pragma unroll
    for (int s = 0; s < KPL; ++s) {
      // -- refill set s from the stream, then issue the copies of its buckets
      const unsigned need = __ballot_sync(kFull, !active[s]);
      if (need != 0u && q.base + q.head < end) {
        uint32_t k, unused, tb;
        const uint64_t at = bq_take<false>(q, queries, nullptr, end, bv, offs, need, below, lane, k, unused, tb);
        if (at != ~0ull) {
          if (COUNT) answered++;
          if (k == kEmptyKey) {
            out[at] = kEmptyKey;  // the sentinel is never a key
          } else {
            active[s] = true;
            key[s] = k;
            idx[s] = at;
            tab[s] = tb;
            probe[s] = 0;
          }
        }
      }
      act[s] = __ballot_sync(kFull, active[s]);
      if (act[s] != 0u) {
        const uint4 *myb = nullptr;
        if (active[s]) {
          const BatchTable &d = bv.tables[tab[s]];
          myb = reinterpret_cast<const uint4 *>(d.slots) + (uint64_t)batch_bucket(d, probe[s], key[s]) * kChunks;
        }
        uint4 *sbuf = wbuf + (size_t)s * 32 * kChunks;
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const int owner = tbase + j;
          const uint4 *src =
              reinterpret_cast<const uint4 *>(__shfl_sync(kFull, reinterpret_cast<uintptr_t>(myb), owner));
          if ((act[s] >> owner) & 1u) {
            uint4 *row = sbuf + owner * kChunks;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
              const unsigned c = 2u * (unsigned)r + (unsigned)i;
              cp_async16(row + (c ^ swz), src + c);
            }
          }
        }
      }
      cp_async_commit();  // one group per set step, empty or not
      // -- evaluate the set issued KPL - 1 steps ago
      const int e = (s + 1) % KPL;
      cp_async_wait<KPL - 1>();
      __syncwarp();
      if (act[e] != 0u) {
        const uint4 *ebuf = wbuf + (size_t)e * 32 * kChunks;
        bool my_hit = false, my_emp = false;
        uint32_t my_val = kEmptyKey;
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const int owner = tbase + j;
          const uint32_t kj = __shfl_sync(kFull, key[e], owner);
          bool hit = false, emp = false;
          uint32_t hv = 0u;
          if ((act[e] >> owner) & 1u) {
            const uint4 *row = ebuf + owner * kChunks;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
              const uint4 c = row[(2u * (unsigned)r + (unsigned)i) ^ swz];  // pairs (c.x, c.y), (c.z, c.w)
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
          } else if (my_emp || ++probe[e] >= bv.h) {  // BCHT: early exit at a bucket with an empty slot
            finish = true;
          }
          if (finish) {
            out[idx[e]] = result;
            active[e] = false;
          }
        }
        act[e] = 0u;
      }
      __syncwarp();  // set e's buffer is read before the next step reuses it
    }
    bool any = false;
#pragma unroll
    for (int s = 0; s < KPL; ++s) any |= active[s];
    if (__ballot_sync(kFull, any) == 0u && q.base + q.head >= end) break;
  }
  cp_async_wait<0>();
  if (COUNT) {
    probes = warp_sum(probes);
    answered = warp_sum(answered);
    if (lane == 0) {
      atomicAdd(&bv.ctrl->find_probes, probes);
      atomicAdd(&bv.ctrl->find_queries, answered);
    }
  }
}

// ----------------------------------------------------------------------------
template <typename K>
static cudaError_t launch_sliced(K kern, uint64_t items, int blocks_per_sm, cudaStream_t s, int *blocks,
                                 uint64_t *per_warp) {
  cudaError_t e = grid_for(kern, items, blocks_per_sm, blocks);
  if (e != cudaSuccess) return e;
  *per_warp = per_warp_of(items, *blocks);
  return cudaSuccess;
}

cudaError_t launch_batch_fill(const BatchView &bv, uint64_t *slots, uint64_t num_slots, cudaStream_t s) {
  const uint64_t n16 = num_slots / 2;  // every table's slot count is even (b = 16)
  int blocks = 0;
  cudaError_t e = grid_for(batch_fill_kernel, n16 > 0 ? n16 : 1, 0, &blocks);
  if (e != cudaSuccess) return e;
  batch_fill_kernel<<<blocks, kThreads, 0, s>>>(bv, reinterpret_cast<uint4 *>(slots), n16);
  return cudaGetLastError();
}

template <int G, int KPL>
static cudaError_t insert_cfg(const BatchView &bv, const uint32_t *k, const uint32_t *v, uint64_t items,
                              const LaunchOpts &o, cudaStream_t s) {
  auto kern = o.count ? batch_insert_kernel<G, KPL, true> : batch_insert_kernel<G, KPL, false>;
  int blocks = 0;
  cudaError_t e = grid_for(kern, items, o.blocks_per_sm, &blocks);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kThreads, 0, s>>>(bv, k, v);  // claims from bv.ctrl->work_cursor, zeroed by the fill
  return cudaGetLastError();
}

template <int G, int KPL>
static cudaError_t find_cfg(const BatchView &bv, const uint32_t *q, uint32_t *out, uint64_t items,
                            const LaunchOpts &o, cudaStream_t s) {
  auto kern = o.count ? batch_find_kernel<G, KPL, true> : batch_find_kernel<G, KPL, false>;
  int blocks = 0;
  uint64_t pw = 0;
  cudaError_t e = launch_sliced(kern, items, o.blocks_per_sm, s, &blocks, &pw);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kThreads, 0, s>>>(bv, q, out, pw);
  return cudaGetLastError();
}

__device__ __forceinline__ uint32_t segment_of(const uint64_t *__restrict__ offs, uint32_t segs, uint64_t i) {
  uint32_t lo = 0, hi = segs;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(offs + mid) <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(256)
segment_gather_kernel(const uint32_t *const *__restrict__ src, const uint64_t *__restrict__ offs, uint32_t segs,
                      uint32_t *__restrict__ dst, uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t sg = segment_of(offs, segs, i);
    dst[i] = __ldg(src[sg] + (i - __ldg(offs + sg)));
  }
}

__global__ void __launch_bounds__(256)
segment_scatter_kernel(const uint32_t *__restrict__ src, uint32_t *const *__restrict__ dst,
                       const uint64_t *__restrict__ offs, uint32_t segs, uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t sg = segment_of(offs, segs, i);
    dst[sg][i - __ldg(offs + sg)] = src[i];
  }
}

cudaError_t launch_segment_gather(const uint32_t *const *src, const uint64_t *offs, uint32_t segs, uint32_t *dst,
                                  uint64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int blocks = 0;
  cudaError_t e = grid_for(segment_gather_kernel, n, 0, &blocks);
  if (e != cudaSuccess) return e;
  segment_gather_kernel<<<blocks, kThreads, 0, s>>>(src, offs, segs, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_segment_scatter(const uint32_t *src, uint32_t *const *dst, const uint64_t *offs, uint32_t segs,
                                   uint64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int blocks = 0;
  cudaError_t e = grid_for(segment_scatter_kernel, n, 0, &blocks);
  if (e != cudaSuccess) return e;
  segment_scatter_kernel<<<blocks, kThreads, 0, s>>>(src, dst, offs, segs, n);
  return cudaGetLastError();
}

bool batch_shape_supported(int G, int kpl) {
  return (G == 4 || G == 8 || G == 16) && (kpl == 1 || kpl == 2);
}

bool batch_find_shape_supported(int G, int kpl) { return batch_shape_supported(G, kpl) || (G == 4 && kpl == 6); }

// staged find: 6 query sets per lane, 2-warp blocks (24 KB of shared memory per warp)
static cudaError_t find_staged(const BatchView &bv, const uint32_t *q, uint32_t *out, uint64_t items,
                               const LaunchOpts &o, cudaStream_t s) {
  constexpr int kKpl = 6, kWarps = 2;
  auto kern = o.count ? batch_find_async_kernel<kKpl, kWarps, true> : batch_find_async_kernel<kKpl, kWarps, false>;
  const size_t smem = kWarps * find_async_smem_per_warp<kKpl>();
  int blocks = 0;
  cudaError_t e = grid_for_smem(kern, 32 * kWarps, smem, items, o.blocks_per_sm, &blocks);
  if (e != cudaSuccess) return e;
  const uint64_t warps = (uint64_t)blocks * kWarps;
  kern<<<blocks, 32 * kWarps, smem, s>>>(bv, q, out, (items + warps - 1) / warps);
  return cudaGetLastError();
}

cudaError_t launch_batch_insert(const BatchView &bv, const uint32_t *k, const uint32_t *v, uint64_t items,
                                const LaunchOpts &o, cudaStream_t s) {
  if (items == 0) return cudaSuccess;
  const int g = o.tile_lanes, kpl = o.keys_per_lane;
  if (g == 16) return kpl == 1 ? insert_cfg<16, 1>(bv, k, v, items, o, s) : insert_cfg<16, 2>(bv, k, v, items, o, s);
  if (g == 8) return kpl == 1 ? insert_cfg<8, 1>(bv, k, v, items, o, s) : insert_cfg<8, 2>(bv, k, v, items, o, s);
  if (g == 4) return kpl == 1 ? insert_cfg<4, 1>(bv, k, v, items, o, s) : insert_cfg<4, 2>(bv, k, v, items, o, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_batch_find(const BatchView &bv, const uint32_t *q, uint32_t *out, uint64_t items,
                              const LaunchOpts &o, cudaStream_t s) {
  if (items == 0) return cudaSuccess;
  const int g = o.tile_lanes, kpl = o.keys_per_lane;
  if (g == 16) return kpl == 1 ? find_cfg<16, 1>(bv, q, out, items, o, s) : find_cfg<16, 2>(bv, q, out, items, o, s);
  if (g == 8) return kpl == 1 ? find_cfg<8, 1>(bv, q, out, items, o, s) : find_cfg<8, 2>(bv, q, out, items, o, s);
  if (g == 4 && kpl == 6) return find_staged(bv, q, out, items, o, s);
  if (g == 4) return kpl == 1 ? find_cfg<4, 1>(bv, q, out, items, o, s) : find_cfg<4, 2>(bv, q, out, items, o, s);
  return cudaErrorInvalidValue;
}

}  // namespace ght
