// ght_shard.cu -- host side of the sharding entry points (include/ght.h):
// the partition of keys or queries over G shards by a partition hash, and
// the return of answers to query order. The paper's method runs on one GPU;
// these are the steps that spread one table over several.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "ght.h"
#include "ght_host.h"
#include "ght_internal.h"

using ght::host::cuda_fail;
using ght::host::fail;
using ght::host::pool_alloc;
using ght::host::wait_event;

extern "C" {

int ght_partition_constants(uint64_t seed, uint32_t *a, uint32_t *c) {
  if (!a || !c) return fail(GHT_ERR_INVALID_ARG, "a or c is NULL");
  // the tables' derivation from a seed of its own, so g is independent of every h_i
  uint32_t aa[4], cc[4];
  ght::host::derive_constants(seed ^ GHT_PARTITION_SEED_SALT, 0, 1, aa, cc);
  *a = aa[0];
  *c = cc[0];
  return GHT_OK;
}

int ght_partition(const uint32_t *d_keys, const uint32_t *d_values, uint64_t n, uint64_t seed, uint32_t shards,
                  uint32_t *d_out_keys, uint32_t *d_out_values, uint64_t *h_counts, void *cuda_stream) {
  if (shards == 0 || shards > 4096) return fail(GHT_ERR_INVALID_ARG, "shards %u outside [1, 4096]", shards);
  if (!h_counts) return fail(GHT_ERR_INVALID_ARG, "h_counts is NULL");
  if (n > 0xFFFFFFFFull) return fail(GHT_ERR_INVALID_ARG, "n = %llu exceeds 2^32 - 1", (unsigned long long)n);
  if (n > 0 && (!d_keys || !d_out_keys || !d_out_values))
    return fail(GHT_ERR_INVALID_ARG, "keys or outputs are NULL");
  if ((reinterpret_cast<uintptr_t>(d_keys) | reinterpret_cast<uintptr_t>(d_values)) & 15u)
    return fail(GHT_ERR_INVALID_ARG, "keys and values must be 16-byte aligned");
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  ght::TableView tv;
  memset(&tv, 0, sizeof tv);
  uint32_t a = 0, c = 0;
  ght_partition_constants(seed, &a, &c);
  tv.hf.a[0] = a;
  tv.hf.c[0] = c;
  tv.hf.mod = ght::make_fastmod(shards);
  tv.m = shards;
  tv.h = 1;
  // scratch: control block (status of the scatter's bounded waits), counts, cursors
  const uint64_t bytes = sizeof(ght::Ctrl) + 2ull * ((shards * 4ull + 255ull) & ~255ull);
  void *scr = nullptr;
  cudaError_t e = pool_alloc(&scr, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(GHT_ERR_OOM, "partition scratch: %s", cudaGetErrorString(e));
  }
  tv.ctrl = static_cast<ght::Ctrl *>(scr);
  uint32_t *counts = reinterpret_cast<uint32_t *>(static_cast<char *>(scr) + sizeof(ght::Ctrl));
  uint32_t *cursors = counts + ((shards * 4ull + 255ull) & ~255ull) / 4;
  std::vector<uint32_t> h32(shards, 0u);
  ght::Ctrl h_ctrl;
  memset(&h_ctrl, 0, sizeof h_ctrl);
  int rc = GHT_OK;
  if ((e = cudaMemsetAsync(tv.ctrl, 0, sizeof(ght::Ctrl), s)) != cudaSuccess ||
      (e = ght::launch_group(tv, d_keys, d_values, n, 0, shards, counts, cursors, d_out_keys, d_out_values, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(h32.data(), counts, shards * 4ull, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&h_ctrl, tv.ctrl, sizeof h_ctrl, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    rc = cuda_fail(e, "launching the partition");
  cudaFreeAsync(scr, s);
  if (rc) return rc;
  cudaEvent_t done = nullptr;
  if ((e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "creating an event");
  rc = (e = cudaEventRecord(done, s)) == cudaSuccess ? wait_event(done) : cuda_fail(e, "recording an event");
  cudaEventDestroy(done);
  if (rc) return rc;
  if (h_ctrl.status & ght::kStatusTimeout) return fail(GHT_ERR_DEVICE_TIMEOUT, "the partition's copies did not complete");
  for (uint32_t i = 0; i < shards; ++i) h_counts[i] = h32[i];
  return GHT_OK;
}

int ght_unpermute(const uint32_t *d_src, const uint32_t *d_pos, uint64_t n, uint32_t *d_dst, void *cuda_stream) {
  if (n == 0) return GHT_OK;
  if (!d_src || !d_pos || !d_dst) return fail(GHT_ERR_INVALID_ARG, "src, pos or dst is NULL");
  const cudaError_t e = ght::launch_unpermute(d_src, d_pos, n, d_dst, static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? GHT_OK : cuda_fail(e, "launching the unpermute");
}

}  // extern "C"
