// kern_place.cu -- first-choice placement of a two-phase bucketed cuckoo
// build, one thread block per sub-group of consecutive first-choice buckets
// (phase 1 of the build; the overflow is inserted by the cuckoo insert).
//
// What it computes is the ranked placement of reading R18 (Sec. III-A with
// the keys that reach their first-choice bucket H_0 while it has room
// inserted first): a key whose arrival rank r at H_0 is below b is stored in
// slot r of H_0, every other key goes to the overflow list. The arrival
// order here is the order of a block's shared-memory atomics.
//
// How (a GB300 design): the pairs arrive split by sub-group (two grouping
// passes), so a sub-group's pairs are contiguous and touch only its
// 2^fine_shift buckets -- 64 KB of table. A block claims the next sub-group,
// fills a 64 KB image of its buckets in shared memory with empty slots, ranks
// each key with a per-bucket counter in shared memory, stores ranks < b into
// the image and stages the rest for the overflow list, and then writes the
// image over the table with 16-byte stores. A placement that stores each
// pair into the table by itself is bound by the L2's rate of scattered
// 8-byte stores (about 80 G/s on GB300, whether its ranks come from L2 or
// shared-memory counters); here every table line leaves the SM as whole
// vector stores, once, and the table needs no fill.
#include "ght_internal.h"
#include "ght_kernels.cuh"

namespace ght {

namespace {

constexpr int kBPThreads = 512;
constexpr int kBPBatch = 8;          // pairs a thread loads before ranking them
constexpr int kBPStage = 2048;       // overflow pairs staged per block
constexpr uint32_t kBPImageBytes = 65536;

}  // namespace

template <typename S, int B, bool COUNT>
__global__ void __launch_bounds__(kBPThreads, 2)
block_place_kernel(TableView tv, const uint32_t *__restrict__ pk, const uint32_t *__restrict__ pv,
                   const uint32_t *__restrict__ ends, uint32_t region, uint32_t bins, int fine_shift,
                   uint32_t *__restrict__ ovf_k, uint32_t *__restrict__ ovf_v, uint64_t cap) {
  using T = typename S::T;
  constexpr int kMaxBuckets = (int)(kBPImageBytes / (B * sizeof(T)));
  constexpr int kVecB = (int)(B * sizeof(T) / 16);  // 16-byte vectors per bucket
  extern __shared__ uint4 bp_img[];                 // [kBPImageBytes / 16]
  T *img = reinterpret_cast<T *>(bp_img);
  __shared__ uint32_t bcnt[kMaxBuckets];
  __shared__ uint32_t ok[kBPStage], ov[kBPStage];
  __shared__ uint32_t s_bin, s_novf;
  __shared__ unsigned long long s_obase;
  unsigned long long *ovf_count = &tv.ctrl->reserved[0];
  unsigned long long *bin_cursor = &tv.ctrl->reserved[1];
  const int tid = threadIdx.x;
  const uint32_t m = tv.m;
  unsigned long long placed = 0;
  if (tid == 0) s_novf = 0u;

  // move the staged overflow pairs to the global list (whole block)
  auto flush = [&](uint32_t staged) {
    if (tid == 0) s_obase = atomicAdd(ovf_count, (unsigned long long)staged);
    __syncthreads();
    const unsigned long long base = s_obase;
    for (uint32_t i = tid; i < staged; i += kBPThreads)
      if (base + i < cap) {
        ovf_k[base + i] = ok[i];
        ovf_v[base + i] = ov[i];
      }
    __syncthreads();
    if (tid == 0) s_novf = 0u;
    __syncthreads();
  };

  for (;;) {
    if (tid == 0) s_bin = (uint32_t)min(atomicAdd(bin_cursor, 1ull), (unsigned long long)bins);
    __syncthreads();
    const uint32_t f = s_bin;
    if (f >= bins) break;  // block-uniform
    const uint32_t b0 = f << fine_shift;
    const uint32_t nb = min(m - b0, 1u << fine_shift);
    const uint4 e = make_uint4(kEmptyKey, kEmptyKey, kEmptyKey, kEmptyKey);
    for (uint32_t i = tid; i < nb * kVecB; i += kBPThreads) bp_img[i] = e;
    for (uint32_t i = tid; i < nb; i += kBPThreads) bcnt[i] = 0u;
    __syncthreads();
    // a sub-group's cursor passes its region's end when it overflowed (the
    // pairs beyond were not written; the build regroups exactly)
    const uint32_t s0 = f * region, s1 = min(ends[f], s0 + region);
    for (uint32_t i0 = s0; i0 < s1; i0 += kBPBatch * kBPThreads) {
      uint32_t k[kBPBatch], v[kBPBatch];
#pragma unroll
      for (int u = 0; u < kBPBatch; ++u) {
        const uint32_t i = i0 + u * kBPThreads + tid;
        k[u] = i < s1 ? __ldg(pk + i) : kEmptyKey;
        v[u] = i < s1 ? __ldg(pv + i) : 0u;
        if (i < s1 && k[u] == kEmptyKey) atomicOr(&tv.ctrl->status, kStatusSentinel);
      }
#pragma unroll
      for (int u = 0; u < kBPBatch; ++u) {
        if (k[u] == kEmptyKey) continue;
        const uint32_t lb = bucket_of(tv.hf, 0, k[u]) - b0;
        const uint32_t r = atomicAdd(&bcnt[lb], 1u);
        if (COUNT) placed++;  // a visit of H_0, stored or not (the overflow insert starts at H_1)
        if (r < (uint32_t)B) {
          img[lb * B + r] = S::make(k[u], v[u]);
        } else {
          const uint32_t at = atomicAdd(&s_novf, 1u);
          if (at < (uint32_t)kBPStage) {
            ok[at] = k[u];
            ov[at] = v[u];
          } else {  // staging full: straight to the list
            const unsigned long long g = atomicAdd(ovf_count, 1ull);
            if (g < cap) {
              ovf_k[g] = k[u];
              ovf_v[g] = v[u];
            }
          }
        }
      }
    }
    __syncthreads();
    uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<T *>(tv.slots) + (uint64_t)b0 * B);
    for (uint32_t i = tid; i < nb * kVecB; i += kBPThreads) dst[i] = bp_img[i];
    const uint32_t staged = s_novf;
    __syncthreads();
    if (staged > (uint32_t)(kBPStage / 2)) flush(min(staged, (uint32_t)kBPStage));
  }
  const uint32_t staged = s_novf;
  __syncthreads();
  if (staged) flush(min(staged, (uint32_t)kBPStage));
  if (COUNT) {
    placed = warp_sum(placed);
    if ((tid & 31) == 0 && placed) atomicAdd(&tv.ctrl->insert_probes, placed);
  }
}

int block_place_fine_shift(int B, bool key_slots) {
  const uint32_t bucket_bytes = (uint32_t)B * (key_slots ? 4u : 8u);
  int shift = 0;
  while ((1u << (shift + 1)) * bucket_bytes <= kBPImageBytes) ++shift;
  return shift;
}

template <typename S, int B>
static cudaError_t place_blocks(const TableView &tv, const uint32_t *pk, const uint32_t *pv, const uint32_t *ends,
                                uint32_t region, uint32_t bins, int fine_shift, const PlaceBuffers &pb, bool count,
                                cudaStream_t s) {
  auto kern = count ? block_place_kernel<S, B, true> : block_place_kernel<S, B, false>;
  int blocks = 0;
  cudaError_t e = grid_for_smem(kern, kBPThreads, kBPImageBytes, (uint64_t)bins * kBPThreads, 0, &blocks);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kBPThreads, kBPImageBytes, s>>>(tv, pk, pv, ends, region, bins, fine_shift, pb.ovf_k, pb.ovf_v,
                                                 pb.cap);
  return cudaGetLastError();
}

cudaError_t launch_block_place(int B, bool key_slots, const TableView &tv, const uint32_t *pk, const uint32_t *pv,
                               const uint32_t *ends, uint32_t region, uint32_t bins, int fine_shift,
                               const PlaceBuffers &pb, bool count, cudaStream_t s) {
  if (fine_shift < 0 || fine_shift > block_place_fine_shift(B, key_slots) || bins == 0) return cudaErrorInvalidValue;
  if (key_slots) {
    if (B != 32) return cudaErrorInvalidValue;
    return place_blocks<KeySlot, 32>(tv, pk, pv, ends, region, bins, fine_shift, pb, count, s);
  }
  if (B == 16) return place_blocks<PairSlot, 16>(tv, pk, pv, ends, region, bins, fine_shift, pb, count, s);
  if (B == 32) return place_blocks<PairSlot, 32>(tv, pk, pv, ends, region, bins, fine_shift, pb, count, s);
  return cudaErrorInvalidValue;
}

}  // namespace ght
