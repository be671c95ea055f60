// kern_bcht.cu -- instantiations and launchers of the BCHT kernels for every
// supported tile shape (bucket of 16 or 32 pairs; 4, 8 or 16 lanes per tile).
#include "ght_internal.h"
#include "ght_find_async.cuh"
#include "ght_kernels.cuh"

namespace ght {

template <int B, int G, int KPL>
static cudaError_t insert_kpl(const TableView &tv, const uint32_t *k, const uint32_t *v,
                              uint64_t n, const LaunchOpts &o, cudaStream_t s) {
  auto kern = o.count ? bucketed_insert_kernel<kBCHT, B, G, KPL, true> : bucketed_insert_kernel<kBCHT, B, G, KPL, false>;
  int blocks = 0;
  cudaError_t e = grid_for(kern, n, o.blocks_per_sm, &blocks);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kThreads, 0, s>>>(tv, k, v, n, o.dynamic ? 0 : per_warp_of(n, blocks));
  return cudaGetLastError();
}

template <int B, int G>
static cudaError_t insert_shape(const TableView &tv, const uint32_t *k, const uint32_t *v,
                                uint64_t n, const LaunchOpts &o, cudaStream_t s) {
  return o.keys_per_lane == 1 ? insert_kpl<B, G, 1>(tv, k, v, n, o, s) : insert_kpl<B, G, 2>(tv, k, v, n, o, s);
}

template <int B, int G, int KPL>
static cudaError_t find_kpl(const TableView &tv, const uint32_t *q, uint32_t *out, uint64_t n,
                            const LaunchOpts &o, cudaStream_t s) {
  auto kern = o.count ? bucketed_find_kernel<kBCHT, B, G, KPL, true> : bucketed_find_kernel<kBCHT, B, G, KPL, false>;
  int blocks = 0;
  cudaError_t e = grid_for(kern, n, o.blocks_per_sm, &blocks);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kThreads, 0, s>>>(tv, q, out, n, per_warp_of(n, blocks));
  return cudaGetLastError();
}

template <int B, int G>
static cudaError_t find_shape(const TableView &tv, const uint32_t *q, uint32_t *out, uint64_t n,
                              const LaunchOpts &o, cudaStream_t s) {
  return o.keys_per_lane == 1 ? find_kpl<B, G, 1>(tv, q, out, n, o, s) : find_kpl<B, G, 2>(tv, q, out, n, o, s);
}

template <int B>
static cudaError_t place_b(const TableView &tv, const uint32_t *k, const uint32_t *v, uint64_t n,
                          const PlaceBuffers &pb, bool count, cudaStream_t s) {
  auto kern = count ? rank_place_kernel<B, true> : rank_place_kernel<B, false>;
  int blocks = 0;
  cudaError_t e = grid_for(kern, (n + kPlacePerThread - 1) / kPlacePerThread, 0, &blocks);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kThreads, 0, s>>>(tv, k, v, n, pb.counters, pb.ovf_k, pb.ovf_v, pb.cap, pb.ends, pb.region,
                                       pb.region_M);
  return cudaGetLastError();
}

cudaError_t launch_place_bcht(int B, const TableView &tv, const uint32_t *k, const uint32_t *v, uint64_t n,
                              const PlaceBuffers &pb, bool count, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (B == 16) return place_b<16>(tv, k, v, n, pb, count, s);
  if (B == 32) return place_b<32>(tv, k, v, n, pb, count, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_find_bcht_async(int B, const TableView &tv, const uint32_t *q, uint32_t *out, uint64_t n,
                                   const LaunchOpts &o, cudaStream_t s, bool early_exit) {
  if (o.tile_lanes != 4) return cudaErrorInvalidValue;
  if (B == 16)
    return launch_staged_find_kpl<PairSlot, 1>(tv, q, out, n, o.keys_per_lane, o.count, o.blocks_per_sm, early_exit, s);
  if (B == 32)
    return launch_staged_find_kpl<PairSlot, 2>(tv, q, out, n, o.keys_per_lane, o.count, o.blocks_per_sm, early_exit, s);
  return cudaErrorInvalidValue;
}

bool bcht_shape_supported(int B, int G) {
  return (B == 16 && (G == 4 || G == 8 || G == 16)) || (B == 32 && (G == 8 || G == 16));
}

cudaError_t launch_insert_bcht(int B, const TableView &tv, const uint32_t *k, const uint32_t *v,
                               uint64_t n, const LaunchOpts &o, cudaStream_t s) {
  if (B == 16 && o.tile_lanes == 8) return insert_shape<16, 8>(tv, k, v, n, o, s);
  if (B == 16 && o.tile_lanes == 4) return insert_shape<16, 4>(tv, k, v, n, o, s);
  if (B == 16 && o.tile_lanes == 16) return insert_shape<16, 16>(tv, k, v, n, o, s);
  if (B == 32 && o.tile_lanes == 8) return insert_shape<32, 8>(tv, k, v, n, o, s);
  if (B == 32 && o.tile_lanes == 16) return insert_shape<32, 16>(tv, k, v, n, o, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_find_bcht(int B, const TableView &tv, const uint32_t *q, uint32_t *out,
                             uint64_t n, const LaunchOpts &o, cudaStream_t s) {
  if (B == 16 && o.tile_lanes == 8) return find_shape<16, 8>(tv, q, out, n, o, s);
  if (B == 16 && o.tile_lanes == 4) return find_shape<16, 4>(tv, q, out, n, o, s);
  if (B == 16 && o.tile_lanes == 16) return find_shape<16, 16>(tv, q, out, n, o, s);
  if (B == 32 && o.tile_lanes == 8) return find_shape<32, 8>(tv, q, out, n, o, s);
  if (B == 32 && o.tile_lanes == 16) return find_shape<32, 16>(tv, q, out, n, o, s);
  return cudaErrorInvalidValue;
}

}  // namespace ght
