// kern_gfind.cu -- grouped bulk find of 16-pair buckets, for query batches
// many times larger than the table's bucket count.
//
// What it computes is the find of Sec. V (BCHT, Sec. V-B: probe H_0, H_1, ...,
// stop at the bucket holding the key or, with early exit, at a bucket with
// an empty slot; P2BHT, IHT and the load-balanced BCHT, Sec. V-C/V-D and
// Sec. III-A: read on until the key is found or the last candidate): every
// query makes the same bucket reads, in the same order, with the same stop
// rule, as in the per-query find. Only the schedule differs: round r makes
// probe r of every query still open, with the queries grouped by the 32 KB
// of table (256 buckets) their H_r bucket lies in.
//
// Why (a GB300 measure, not the paper's design): a random 128-byte bucket
// read costs one DRAM access, and this GPU's DRAM serves about 42 G random
// line reads per second, 80 % of its copy bandwidth in bytes. When a batch
// holds many queries per bucket, one round reads each table line once, in
// order, into a 32 KB shared-memory image of the sub-group's buckets, and the
// queries move through two streaming grouping passes instead. The answers
// return to query order through two more grouping passes by position and a
// shared-memory window per 8192 positions (window_write_kernel): scattered
// 4-byte stores would cost a DRAM read-modify-write each.
#include "ght_bulk.cuh"
#include "ght_internal.h"
#include "ght_kernels.cuh"

namespace ght {

namespace {

constexpr int kGLThreads = 256;
constexpr int kGLPer = 4;                  // items a thread evaluates per batch
constexpr uint32_t kGLImageBytes = 128u << kGFindFineShift;  // one sub-group's buckets
constexpr uint32_t kGLSparse = 128;        // fewer items: their buckets are read directly
constexpr uint32_t kGLWaitPolls = 1u << 26;  // bounded wait for a sub-group's image
constexpr int kWinThreads = 512;

// Bucket evaluation for one key: the 16 pairs as eight 16-byte chunks, lane
// L starting at chunk L mod 8 (in shared memory the 32 lanes of a warp then
// spread over the eight bank groups: four wavefronts per read, the least a
// 512-byte warp read takes). A bucket has an empty slot iff the largest key
// word in it is the empty key (no key is 0xFFFFFFFF).
template <typename Row>
__device__ __forceinline__ void eval_bucket(Row row, int lane, uint32_t key, bool &hit, bool &emp, uint32_t &val) {
  uint32_t mx = 0u;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint4 x = row((c + lane) & 7);
    if (x.x == key) {
      hit = true;
      val = x.y;
    }
    if (x.z == key) {
      hit = true;
      val = x.w;
    }
    mx = max(mx, max(x.x, x.z));
  }
  emp = mx == kEmptyKey;
}

}  // namespace

// One round of the grouped find: block per sub-group of 2^fine_shift <= 256
// buckets (claimed from fl.claim), whose items are [f * region, ends[f]) of
// (gk, gp, gb): keys, query positions and each key's H_round bucket within
// the sub-group, split by sub-group by the grouping pass that also computed
// the buckets. A block copies the sub-group's buckets (32 KB) into shared
// memory with one bulk copy and each thread evaluates whole buckets for its
// items there; a sub-group with fewer than kGLSparse items (the late rounds,
// where most queries are answered) reads its items' buckets from global
// memory instead. Four blocks share an SM, so one block's image copy
// overlaps the others' evaluation. An item is answered (found; or, with
// early exit, a bucket with an empty slot; or its last candidate) into the
// answer list (position, value), or moves on to the next round's list (key,
// position). Both lists are appended per batch of the block: one atomic per
// list and batch.
template <bool EARLY, bool COUNT>
__global__ void __launch_bounds__(kGLThreads, 4)
grouped_lookup_kernel(TableView tv, int round, const uint32_t *__restrict__ gk, const uint32_t *__restrict__ gp,
                      const uint8_t *__restrict__ gb, const uint32_t *__restrict__ ends, uint32_t region,
                      uint32_t bins, int fine_shift, GroupedFindLists fl) {
  extern __shared__ uint4 gl_img[];  // [buckets of the sub-group][8 chunks]
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_bin;
  __shared__ int s_abort;
  __shared__ uint32_t warp_tot[kGLThreads / 32];
  __shared__ unsigned long long s_res_base, s_cont_base;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t m = tv.m;
  const bool last = round + 1 >= tv.h;
  const uint4 *slots4 = reinterpret_cast<const uint4 *>(tv.slots);
  unsigned long long probes = 0;
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
    s_abort = 0;
  }
  __syncthreads();
  uint32_t loads = 0;  // images loaded so far (the barrier's phase)
  for (;;) {
    if (tid == 0) s_bin = (uint32_t)min(atomicAdd(fl.claim, 1ull), (unsigned long long)bins);
    __syncthreads();
    const uint32_t f = s_bin;
    if (f >= bins) break;  // block-uniform
    // a sub-group's cursor passes its region's end when items spilled
    const uint32_t s0 = f * region, s1 = min(ends[f], s0 + region);
    const uint32_t b0 = f << fine_shift;
    const uint32_t nb = min(m - b0, 1u << fine_shift);
    const bool staged = s1 >= s0 + kGLSparse;  // block-uniform
    if (staged) {
      if (tid == 0) {
        fence_proxy_async_smem();  // the last sub-group's reads of the image come first
        mbar_arrive_expect_tx(&bar, nb * 128u);
        bulk_g2s(gl_img, slots4 + (uint64_t)b0 * 8u, nb * 128u, &bar);
      }
      if (!mbar_wait_bounded(&bar, loads & 1u, kGLWaitPolls)) s_abort = 1;
      ++loads;
      __syncthreads();
      if (s_abort) {
        if (tid == 0) atomicOr(&tv.ctrl->status, kStatusTimeout);
        return;
      }
    }
    for (uint32_t i0 = s0; i0 < s1; i0 += kGLThreads * kGLPer) {
      uint32_t key[kGLPer], pos[kGLPer], val[kGLPer], lbs[kGLPer];
      int state[kGLPer];  // 0: no item, 1: answered, 2: next round
#pragma unroll
      for (int u = 0; u < kGLPer; ++u) {
        const uint32_t i = i0 + (uint32_t)u * kGLThreads + tid;
        state[u] = 0;
        key[u] = kEmptyKey;
        pos[u] = 0u;
        val[u] = kEmptyKey;
        lbs[u] = 0u;
        if (i < s1) {
          key[u] = __ldg(gk + i);
          pos[u] = __ldg(gp + i);
          lbs[u] = __ldg(gb + i);
          state[u] = 1;
        }
      }
      uint32_t nres = 0, ncont = 0;
#pragma unroll
      for (int u = 0; u < kGLPer; ++u) {
        if (state[u] == 0) continue;
        if (key[u] == kEmptyKey) {  // the sentinel is never a key: answered without a probe
          ++nres;
          continue;
        }
        const uint32_t lb = lbs[u];
        if (lb >= nb) {  // not this sub-group's bucket: a grouping fault
          atomicOr(&tv.ctrl->status, kStatusCorrupt);
          state[u] = 0;
          continue;
        }
        if (COUNT) probes++;
        bool hit = false, emp = false;
        uint32_t hv = kEmptyKey;
        if (staged) {
          const uint4 *row = gl_img + lb * 8u;
          eval_bucket([&](int c) { return row[c]; }, lane, key[u], hit, emp, hv);
        } else {
          const uint4 *row = slots4 + (uint64_t)(b0 + lb) * 8u;
          eval_bucket([&](int c) { return __ldg(row + c); }, lane, key[u], hit, emp, hv);
        }
        if (hit || (EARLY && emp) || last) {
          val[u] = hv;
          ++nres;
        } else {
          state[u] = 2;
          ++ncont;
        }
      }
      // block-wide offsets of this batch's answers and carried items
      const uint32_t packed = nres | (ncont << 16);
      uint32_t incl = packed;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane == 31) warp_tot[wid] = incl;
      __syncthreads();
      if (tid == 0) {
        uint32_t tot = 0;
        for (int w = 0; w < kGLThreads / 32; ++w) {
          const uint32_t x = warp_tot[w];
          warp_tot[w] = tot;
          tot += x;
        }
        s_res_base = (tot & 0xFFFFu) ? atomicAdd(fl.res_count, (unsigned long long)(tot & 0xFFFFu)) : 0ull;
        s_cont_base = (tot >> 16) ? atomicAdd(fl.cont_count, (unsigned long long)(tot >> 16)) : 0ull;
      }
      __syncthreads();
      const uint32_t before = warp_tot[wid] + incl - packed;
      unsigned long long rb = s_res_base + (before & 0xFFFFu), cb = s_cont_base + (before >> 16);
#pragma unroll
      for (int u = 0; u < kGLPer; ++u) {
        if (state[u] == 1) {
          if (rb < fl.cap) {
            fl.res_p[rb] = pos[u];
            fl.res_v[rb] = val[u];
          }
          ++rb;
        } else if (state[u] == 2) {
          if (cb < fl.cap) {
            fl.cont_k[cb] = key[u];
            fl.cont_p[cb] = pos[u];
          }
          ++cb;
        }
      }
      __syncthreads();  // warp_tot and the bases are reused by the next batch
    }
    __syncthreads();  // the image and s_bin are reused by the next sub-group
  }
  if (COUNT) {
    probes = warp_sum(probes);
    if (lane == 0 && probes) atomicAdd(&tv.ctrl->find_probes, probes);
  }
}

// Items the groupings could not place in their regions (queries whose
// buckets crowd far beyond a random hash's, e.g. one key asked many times):
// each is answered here from probe `round` on, reading buckets from global
// memory one 16-byte chunk at a time; its answer joins the answer list. Also
// adds the batch's n queries to the table's query count.
template <bool EARLY, bool COUNT>
__global__ void __launch_bounds__(256)
grouped_spill_kernel(TableView tv, SpillList spill, GroupedFindLists fl, uint64_t n_queries) {
  const unsigned long long n = min(*spill.count, spill.cap);
  unsigned long long probes = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t key = spill.k[i], pos = spill.v[i];
    uint32_t val = kEmptyKey;
    if (key != kEmptyKey) {
      for (int p = (int)spill.round[i]; p < tv.h; ++p) {
        if (COUNT) probes++;
        const uint4 *row = reinterpret_cast<const uint4 *>(tv.slots) + (uint64_t)bucket_of(tv.hf, p, key) * 8u;
        bool hit = false, emp = false;
        for (int c = 0; c < 8; ++c) {
          const uint4 x = row[c];
          if (x.x == key) {
            hit = true;
            val = x.y;
          }
          if (x.z == key) {
            hit = true;
            val = x.w;
          }
          emp |= (x.x == kEmptyKey) | (x.z == kEmptyKey);
        }
        if (hit || (EARLY && emp)) break;
      }
    }
    const unsigned long long at = atomicAdd(fl.res_count, 1ull);
    if (at < fl.cap) {
      fl.res_p[at] = pos;
      fl.res_v[at] = val;
    }
  }
  if (COUNT) {
    probes = warp_sum(probes);
    if ((threadIdx.x & 31) == 0 && probes) atomicAdd(&tv.ctrl->find_probes, probes);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&tv.ctrl->find_queries, (unsigned long long)n_queries);
  }
}

// Last step of the return to query order: window f holds positions [8192 f,
// 8192 f + 8192), whose (position, answer) items are [8192 f, ends[f]) of
// (rp, rv) -- each position exactly once. The answers are placed in a
// shared-memory image of the window and the window leaves as 16-byte stores.
__global__ void __launch_bounds__(kWinThreads)
window_write_kernel(const uint32_t *__restrict__ rp, const uint32_t *__restrict__ rv, const uint32_t *__restrict__ ends,
                    uint64_t n, uint32_t *__restrict__ out) {
  constexpr uint32_t kWin = 1u << kGFindWindowLog2;
  __shared__ __align__(16) uint32_t win[kWin];
  const uint32_t windows = (uint32_t)((n + kWin - 1) / kWin);
  const bool vec = (reinterpret_cast<uintptr_t>(out) & 15u) == 0u;
  for (uint32_t f = blockIdx.x; f < windows; f += gridDim.x) {
    const uint32_t s0 = f * kWin, s1 = min(ends[f], s0 + kWin);
    for (uint32_t i = s0 + threadIdx.x; i < s1; i += kWinThreads) win[__ldg(rp + i) & (kWin - 1u)] = __ldg(rv + i);
    __syncthreads();
    const uint64_t base = (uint64_t)f * kWin;
    const uint32_t cnt = (uint32_t)min((uint64_t)kWin, n - base);
    if (vec && cnt == kWin) {
      uint4 *o4 = reinterpret_cast<uint4 *>(out + base);
      const uint4 *w4 = reinterpret_cast<const uint4 *>(win);
      for (uint32_t i = threadIdx.x; i < kWin / 4; i += kWinThreads) o4[i] = w4[i];
    } else {
      for (uint32_t i = threadIdx.x; i < cnt; i += kWinThreads) out[base + i] = win[i];
    }
    __syncthreads();
  }
}

cudaError_t launch_grouped_lookup(const TableView &tv, int round, bool early_exit, bool count, const uint32_t *gk,
                                  const uint32_t *gp, const uint8_t *gb, const uint32_t *ends, uint32_t region,
                                  uint32_t bins, int fine_shift, const GroupedFindLists &fl, cudaStream_t s) {
  if (fine_shift < 0 || fine_shift > kGFindFineShift || bins == 0 || round < 0 || round >= tv.h || !gb)
    return cudaErrorInvalidValue;
  auto kern = early_exit ? (count ? grouped_lookup_kernel<true, true> : grouped_lookup_kernel<true, false>)
                         : (count ? grouped_lookup_kernel<false, true> : grouped_lookup_kernel<false, false>);
  int blocks = 0;
  cudaError_t e = grid_for_smem(kern, kGLThreads, kGLImageBytes, (uint64_t)bins * kGLThreads, 0, &blocks);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kGLThreads, kGLImageBytes, s>>>(tv, round, gk, gp, gb, ends, region, bins, fine_shift, fl);
  return cudaGetLastError();
}

cudaError_t launch_grouped_spill(const TableView &tv, bool early_exit, bool count, const SpillList &spill,
                                 const GroupedFindLists &fl, uint64_t n_queries, cudaStream_t s) {
  auto kern = early_exit ? (count ? grouped_spill_kernel<true, true> : grouped_spill_kernel<true, false>)
                         : (count ? grouped_spill_kernel<false, true> : grouped_spill_kernel<false, false>);
  // a small grid: the list is empty unless queries crowd far beyond a random hash's
  int blocks = 0;
  cudaError_t e = grid_for(kern, 1ull << 20, 0, &blocks);
  if (e != cudaSuccess) return e;
  kern<<<blocks, 256, 0, s>>>(tv, spill, fl, n_queries);
  return cudaGetLastError();
}

cudaError_t launch_window_write(const uint32_t *rp, const uint32_t *rv, const uint32_t *ends, uint64_t n,
                                uint32_t *out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (n > 0xFFFFFFFFull) return cudaErrorInvalidValue;
  const uint64_t windows = (n + (1u << kGFindWindowLog2) - 1) >> kGFindWindowLog2;
  int sms = 0, dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const uint64_t cap = (uint64_t)sms * 4u;  // 32 KB of shared memory each: four blocks per SM
  window_write_kernel<<<(unsigned)(windows < cap ? windows : cap), kWinThreads, 0, s>>>(rp, rv, ends, n, out);
  return cudaGetLastError();
}

}  // namespace ght
