// kern_other.cu -- instantiations and launchers of the P2BHT, IHT,
// load-balanced BCHT and bucket-size-one cuckoo kernels, plus fill and hash.
#include "ght_internal.h"
#include "ght_kernels.cuh"

namespace ght {

// ----------------------------------------------------------------------------
// Fill (Sec. III-A: initialise all buckets to empty) and reset the control
// block. slots16 covers the 16-byte aligned body; tail8 the last odd pair.
__global__ void fill_kernel(uint4 *__restrict__ slots16, uint64_t n16, uint64_t *__restrict__ tail8,
                            Ctrl *__restrict__ ctrl) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint4 e = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride)
    slots16[i] = e;
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0 && tail8) *tail8 = kEmptyPair;
    if (threadIdx.x < sizeof(Ctrl) / 8) reinterpret_cast<unsigned long long *>(ctrl)[threadIdx.x] = 0ull;
  }
}

// Bucket indices under each hash function (diagnostic; out is n x h).
__global__ void hash_kernel(TableView tv, const uint32_t *__restrict__ keys, uint32_t *__restrict__ out,
                            uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t k = keys[i];
    for (int f = 0; f < tv.h; ++f) out[i * tv.h + f] = bucket_of(tv.hf, f, k);
  }
}

template <int S, int B, int G, int KPL>
static cudaError_t insert_kpl(const TableView &tv, const uint32_t *k, const uint32_t *v,
                              uint64_t n, const LaunchOpts &o, cudaStream_t s) {
  auto kern = o.count ? bucketed_insert_kernel<S, B, G, KPL, true> : bucketed_insert_kernel<S, B, G, KPL, false>;
  int blocks = 0;
  cudaError_t e = grid_for(kern, n, o.blocks_per_sm, &blocks);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kThreads, 0, s>>>(tv, k, v, n, o.dynamic ? 0 : per_warp_of(n, blocks));
  return cudaGetLastError();
}

template <int S, int B, int G>
static cudaError_t insert_shape(const TableView &tv, const uint32_t *k, const uint32_t *v,
                                uint64_t n, const LaunchOpts &o, cudaStream_t s) {
  return o.keys_per_lane == 1 ? insert_kpl<S, B, G, 1>(tv, k, v, n, o, s) : insert_kpl<S, B, G, 2>(tv, k, v, n, o, s);
}

template <int S, int B, int G, int KPL>
static cudaError_t find_kpl(const TableView &tv, const uint32_t *q, uint32_t *out, uint64_t n,
                            const LaunchOpts &o, cudaStream_t s) {
  auto kern = o.count ? bucketed_find_kernel<S, B, G, KPL, true> : bucketed_find_kernel<S, B, G, KPL, false>;
  int blocks = 0;
  cudaError_t e = grid_for(kern, n, o.blocks_per_sm, &blocks);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kThreads, 0, s>>>(tv, q, out, n, per_warp_of(n, blocks));
  return cudaGetLastError();
}

template <int S, int B, int G>
static cudaError_t find_shape(const TableView &tv, const uint32_t *q, uint32_t *out, uint64_t n,
                              const LaunchOpts &o, cudaStream_t s) {
  return o.keys_per_lane == 1 ? find_kpl<S, B, G, 1>(tv, q, out, n, o, s) : find_kpl<S, B, G, 2>(tv, q, out, n, o, s);
}

bool other_shape_supported(int scheme, int B, int G) {
  if (scheme == kCuckoo1) return B == 1;
  if (scheme == kP2BHT || scheme == kIHT || scheme == kBCHT_LB) return (B == 16 || B == 32) && G == 8;
  return false;
}

#define GHT_DISPATCH_BUCKETED(FN, ...)                                              \
  switch (scheme) {                                                                 \
    case kP2BHT: return B == 16 ? FN<kP2BHT, 16, 8>(__VA_ARGS__) : FN<kP2BHT, 32, 8>(__VA_ARGS__); \
    case kIHT: return B == 16 ? FN<kIHT, 16, 8>(__VA_ARGS__) : FN<kIHT, 32, 8>(__VA_ARGS__);       \
    case kBCHT_LB: return B == 16 ? FN<kBCHT_LB, 16, 8>(__VA_ARGS__) : FN<kBCHT_LB, 32, 8>(__VA_ARGS__); \
    default: return cudaErrorInvalidValue;                                          \
  }

cudaError_t launch_insert_other(int scheme, int B, const TableView &tv, const uint32_t *k,
                                const uint32_t *v, uint64_t n, const LaunchOpts &o, cudaStream_t s) {
  if (scheme == kCuckoo1) {
    auto kern = o.count ? cuckoo1_insert_kernel<true> : cuckoo1_insert_kernel<false>;
    int blocks = 0;
    cudaError_t e = grid_for(kern, n, o.blocks_per_sm, &blocks);
    if (e != cudaSuccess) return e;
    kern<<<blocks, kThreads, 0, s>>>(tv, k, v, n);
    return cudaGetLastError();
  }
  if (!other_shape_supported(scheme, B, o.tile_lanes)) return cudaErrorInvalidValue;
  GHT_DISPATCH_BUCKETED(insert_shape, tv, k, v, n, o, s)
}

cudaError_t launch_find_other(int scheme, int B, const TableView &tv, const uint32_t *q,
                              uint32_t *out, uint64_t n, const LaunchOpts &o, cudaStream_t s) {
  if (scheme == kCuckoo1) {
    auto kern = o.count ? cuckoo1_find_kernel<true> : cuckoo1_find_kernel<false>;
    int blocks = 0;
    cudaError_t e = grid_for(kern, n, o.blocks_per_sm, &blocks);
    if (e != cudaSuccess) return e;
    kern<<<blocks, kThreads, 0, s>>>(tv, q, out, n);
    return cudaGetLastError();
  }
  if (!other_shape_supported(scheme, B, o.tile_lanes)) return cudaErrorInvalidValue;
  GHT_DISPATCH_BUCKETED(find_shape, tv, q, out, n, o, s)
}

// Debug check after a successful build (keys must be unique, Sec. VII): every
// scheme stores a key only in its candidate buckets H_0 .. H_{h-1}, so an
// input key with more than one copy across its distinct candidate buckets was
// passed more than once. Thread per key, every slot of every candidate read.
template <typename S>
__global__ void __launch_bounds__(256)
dup_check_kernel(TableView tv, int B, const uint32_t *__restrict__ keys, uint64_t n) {
  using T = typename S::T;
  const T *slots = reinterpret_cast<const T *>(tv.slots);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t k = __ldg(keys + i);
    if (k == kEmptyKey) continue;  // rejected by the build already
    uint32_t seen[4];
    int copies = 0;
    for (int f = 0; f < tv.h && f < 4; ++f) {
      const uint32_t b = bucket_of(tv.hf, f, k);
      bool again = false;
      for (int g = 0; g < f; ++g) again |= seen[g] == b;
      seen[f] = b;
      if (again) continue;
      for (int j = 0; j < B; ++j) copies += S::key(slots[(uint64_t)b * B + j]) == k;
    }
    if (copies > 1) atomicOr(&tv.ctrl->status, (uint32_t)kStatusDuplicate);
  }
}

cudaError_t launch_dup_check(const TableView &tv, int B, bool key_slots, const uint32_t *keys, uint64_t n,
                             cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (B < 1 || B > 32) return cudaErrorInvalidValue;
  int blocks = 0;
  auto kern = key_slots ? dup_check_kernel<KeySlot> : dup_check_kernel<PairSlot>;
  cudaError_t e = grid_for(kern, n, 0, &blocks);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kThreads, 0, s>>>(tv, B, keys, n);
  return cudaGetLastError();
}

cudaError_t launch_fill(const TableView &tv, uint64_t num_slots, cudaStream_t s) {
  const uint64_t n16 = num_slots / 2;  // slots start 256-byte aligned
  uint64_t *tail = (num_slots & 1) ? tv.slots + (num_slots - 1) : nullptr;
  int blocks = 0;
  cudaError_t e = grid_for(fill_kernel, n16 > 0 ? n16 : 1, 0, &blocks);
  if (e != cudaSuccess) return e;
  fill_kernel<<<blocks, kThreads, 0, s>>>(reinterpret_cast<uint4 *>(tv.slots), n16, tail, tv.ctrl);
  return cudaGetLastError();
}

cudaError_t launch_hash(const TableView &tv, const uint32_t *k, uint32_t *out, uint64_t n,
                        cudaStream_t s) {
  int blocks = 0;
  cudaError_t e = grid_for(hash_kernel, n, 0, &blocks);
  if (e != cudaSuccess) return e;
  hash_kernel<<<blocks, kThreads, 0, s>>>(tv, k, out, n);
  return cudaGetLastError();
}

}  // namespace ght
