// kern_set.cu -- keys-only BCHT (a membership set): 32 four-byte keys per
// 128-byte bucket, three hash functions, the BCHT insert and find of
// ght_kernels.cuh with 32-bit slots (the paper's tables "storing keys",
// Sec. I and Sec. III-A).
#include "ght_internal.h"
#include "ght_kernels.cuh"
#include "ght_find_async.cuh"

namespace ght {

template <int KPL>
static cudaError_t set_insert(const TableView &tv, const uint32_t *k, const uint32_t *v, uint64_t n,
                              const LaunchOpts &o, cudaStream_t s) {
  auto kern = o.count ? bucketed_insert_kernel<kBCHT, 32, 8, KPL, true, KeySlot>
                      : bucketed_insert_kernel<kBCHT, 32, 8, KPL, false, KeySlot>;
  int blocks = 0;
  cudaError_t e = grid_for(kern, n, o.blocks_per_sm, &blocks);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kThreads, 0, s>>>(tv, k, v, n, o.dynamic ? 0 : per_warp_of(n, blocks));
  return cudaGetLastError();
}

template <int KPL>
static cudaError_t set_find(const TableView &tv, const uint32_t *q, uint32_t *out, uint64_t n, const LaunchOpts &o,
                            cudaStream_t s) {
  auto kern = o.count ? bucketed_find_kernel<kBCHT, 32, 8, KPL, true, KeySlot>
                      : bucketed_find_kernel<kBCHT, 32, 8, KPL, false, KeySlot>;
  int blocks = 0;
  cudaError_t e = grid_for(kern, n, o.blocks_per_sm, &blocks);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kThreads, 0, s>>>(tv, q, out, n, per_warp_of(n, blocks));
  return cudaGetLastError();
}

bool set_shape_supported(int B, int G) { return B == 32 && G == 8; }

cudaError_t launch_place_set(const TableView &tv, const uint32_t *k, uint64_t n, const PlaceBuffers &pb, bool count,
                             cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  auto kern = count ? rank_place_kernel<32, true, KeySlot> : rank_place_kernel<32, false, KeySlot>;
  int blocks = 0;
  cudaError_t e = grid_for(kern, (n + kPlacePerThread - 1) / kPlacePerThread, 0, &blocks);
  if (e != cudaSuccess) return e;
  // a set has no values: the key array stands in for them and is ignored
  kern<<<blocks, kThreads, 0, s>>>(tv, k, k, n, pb.counters, pb.ovf_k, pb.ovf_v, pb.cap, pb.ends, pb.region,
                                       pb.region_M);
  return cudaGetLastError();
}

cudaError_t launch_insert_set(const TableView &tv, const uint32_t *k, const uint32_t *v, uint64_t n,
                              const LaunchOpts &o, cudaStream_t s) {
  if (o.tile_lanes != 8) return cudaErrorInvalidValue;
  return o.keys_per_lane == 1 ? set_insert<1>(tv, k, v, n, o, s) : set_insert<2>(tv, k, v, n, o, s);
}

cudaError_t launch_find_set(const TableView &tv, const uint32_t *q, uint32_t *out, uint64_t n, const LaunchOpts &o,
                            cudaStream_t s) {
  if (o.tile_lanes != 8) return cudaErrorInvalidValue;
  return o.keys_per_lane == 1 ? set_find<1>(tv, q, out, n, o, s) : set_find<2>(tv, q, out, n, o, s);
}

// The staged find (bucket parts in shared memory, 4-lane tiles, keys_per_lane
// sets in flight) on the set's 32-key buckets.
cudaError_t launch_find_set_async(const TableView &tv, const uint32_t *q, uint32_t *out, uint64_t n,
                                  const LaunchOpts &o, cudaStream_t s) {
  if (o.tile_lanes != 4) return cudaErrorInvalidValue;
  return launch_staged_find_kpl<KeySlot>(tv, q, out, n, o.keys_per_lane, o.count, o.blocks_per_sm, true, s);
}

}  // namespace ght
