// ght_batch_api.cu -- host side of the batched-table C ABI (include/ght.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "ght.h"
#include "ght_batch.h"
#include "ght_host.h"

using ght::host::cuda_fail;
using ght::host::fail;
using ght::host::wait_event;

struct ght_batch {
  uint32_t T = 0;
  uint64_t seed = 0;
  int h = 3;
  uint32_t max_chain = 1000, max_attempts = 50;
  ght::LaunchOpts find_o, build_o;
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;  // private stream the graph is captured on
  // device memory: slots of all tables, then descriptors, offsets, control block
  void *slots_mem = nullptr, *meta_mem = nullptr;
  uint64_t total_slots = 0, slot_bytes = 0;
  ght::BatchTable *d_tables = nullptr;
  uint64_t *d_key_offs = nullptr, *d_query_offs = nullptr;
  ght::Ctrl *d_ctrl = nullptr;
  // host state
  ght::BatchTable *h_tables = nullptr;  // pinned mirror of the descriptors
  std::vector<uint64_t> caps, m, slot_off, key_offs, query_offs;
  std::vector<uint32_t> attempt;
  bool layout_set = false;
  // graph of one run
  cudaGraphExec_t exec = nullptr;
  const void *g_keys = nullptr, *g_values = nullptr, *g_queries = nullptr, *g_out = nullptr;
  int g_shape = -1;
  cudaEvent_t done = nullptr, ev0 = nullptr, ev1 = nullptr;
  // stats
  uint32_t tables_failed = 0, rebuilds = 0;
  int tuned = 0;
  double last_run_ms = -1.0;
  uint64_t graph_launches = 0;

  uint64_t table_seed(uint32_t t) const { return seed + (uint64_t)t * 0x9E3779B97F4A7C15ull; }

  void set_constants(uint32_t t, uint32_t att) {
    attempt[t] = att;
    ght::host::derive_constants(table_seed(t), att, h, h_tables[t].a, h_tables[t].c);
  }

  ght::BatchView view(uint32_t lo, uint32_t hi) const {
    ght::BatchView v;
    v.tables = d_tables;
    v.key_offs = d_key_offs;
    v.query_offs = d_query_offs;
    v.ctrl = d_ctrl;
    v.t_lo = lo;
    v.t_hi = hi;
    v.h = h;
    v.max_chain = max_chain;
    v.max_steps = (uint32_t)std::min<uint64_t>(((uint64_t)max_chain + 2ull) * 3ull * 18ull + 64ull, 0xFFFFFFF0ull);
    v.rng_seed = ght::host::derive_rng_seed(seed, 0);
    return v;
  }

  int shape_sig() const {
    return ((build_o.blocks_per_sm * 64 + find_o.blocks_per_sm) * 100 + build_o.tile_lanes) * 1000 +
           build_o.keys_per_lane * 100 + find_o.tile_lanes * 10 + find_o.keys_per_lane;
  }

  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
  }
};

namespace {

int check_ready(const ght_batch *b) {
  if (!b) return fail(GHT_ERR_INVALID_ARG, "batch is NULL");
  if (!b->layout_set) return fail(GHT_ERR_INVALID_ARG, "ght_batch_set_layout has not been called");
  return GHT_OK;
}

int upload_tables(ght_batch *b, uint32_t lo, uint32_t hi) {
  const cudaError_t e = cudaMemcpyAsync(b->d_tables + lo, b->h_tables + lo, (hi - lo) * sizeof(ght::BatchTable),
                                        cudaMemcpyHostToDevice, b->stream);
  return e == cudaSuccess ? GHT_OK : cuda_fail(e, "uploading table descriptors");
}

int download_tables(ght_batch *b, uint32_t lo, uint32_t hi) {
  cudaError_t e = cudaMemcpyAsync(b->h_tables + lo, b->d_tables + lo, (hi - lo) * sizeof(ght::BatchTable),
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading table status");
  e = cudaEventRecord(b->done, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "recording an event");
  return wait_event(b->done);
}

// Fill + insert of tables [lo, hi) (no wait).
int launch_build(ght_batch *b, uint32_t lo, uint32_t hi, const uint32_t *k, const uint32_t *v) {
  const ght::BatchView bv = b->view(lo, hi);
  uint64_t *slots = static_cast<uint64_t *>(b->slots_mem) + b->slot_off[lo];
  const uint64_t nslots = b->slot_off[hi] - b->slot_off[lo];
  cudaError_t e = ght::launch_batch_fill(bv, slots, nslots, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "launching batch fill");
  e = ght::launch_batch_insert(bv, k, v, b->key_offs[hi] - b->key_offs[lo], b->build_o, b->stream);
  return e == cudaSuccess ? GHT_OK : cuda_fail(e, "launching batch insert");
}

int launch_find(const ght_batch *b, uint32_t lo, uint32_t hi, const uint32_t *q, uint32_t *out) {
  const ght::BatchView bv = b->view(lo, hi);
  const cudaError_t e =
      ght::launch_batch_find(bv, q, out, b->query_offs[hi] - b->query_offs[lo], b->find_o, b->stream);
  return e == cudaSuccess ? GHT_OK : cuda_fail(e, "launching batch find");
}

// After the mirror holds fresh status words: rebuild each failed table alone
// with its next constants; optionally answer its queries again.
int repair(ght_batch *b, const uint32_t *k, const uint32_t *v, const uint32_t *q, uint32_t *out) {
  b->tables_failed = 0;
  for (uint32_t t = 0; t < b->T; ++t) {
    uint32_t st = b->h_tables[t].status;
    if (st & ght::kStatusSentinel) return fail(GHT_ERR_SENTINEL_KEY, "table %u: an input key is the sentinel", t);
    if (st & ght::kStatusTimeout) return fail(GHT_ERR_DEVICE_TIMEOUT, "table %u: a key exceeded the step bound", t);
    if (st & ght::kStatusCorrupt) return fail(GHT_ERR_CUDA, "table %u: corrupt", t);
    while (st != 0u && b->attempt[t] + 1 < b->max_attempts) {
      b->set_constants(t, b->attempt[t] + 1);
      b->rebuilds++;
      int rc = upload_tables(b, t, t + 1);
      if (!rc) rc = launch_build(b, t, t + 1, k, v);
      if (!rc) rc = download_tables(b, t, t + 1);
      if (rc) return rc;
      st = b->h_tables[t].status;
    }
    if (st != 0u) {
      b->tables_failed++;
      continue;
    }
    if (q && b->rebuilds && b->attempt[t] > 0) {
      const int rc = launch_find(b, t, t + 1, q, out);
      if (rc) return rc;
    }
  }
  if (q) {
    const cudaError_t e = cudaEventRecord(b->done, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "recording an event");
    const int rc = wait_event(b->done);
    if (rc) return rc;
  }
  if (b->tables_failed) return fail(GHT_ERR_BUILD_FAILED, "%u tables failed in %u attempts", b->tables_failed,
                                    b->max_attempts);
  return GHT_OK;
}

int reset_constants(ght_batch *b) {
  for (uint32_t t = 0; t < b->T; ++t) b->set_constants(t, 0);
  return GHT_OK;
}

}  // namespace

extern "C" {

ght_batch *ght_batch_create(uint32_t num_tables, const uint64_t *h_capacities, const double *h_load_factors,
                            uint64_t seed, const ght_config *cfg) {
  if (num_tables == 0 || !h_capacities || !h_load_factors) {
    fail(GHT_ERR_INVALID_ARG, "num_tables, capacities and load factors are required");
    return nullptr;
  }
  ght_batch *b = new (std::nothrow) ght_batch();
  if (!b) {
    fail(GHT_ERR_OOM, "host allocation failed");
    return nullptr;
  }
  b->T = num_tables;
  b->seed = seed;
  b->find_o.tile_lanes = 4;
  b->find_o.keys_per_lane = 2;
  b->build_o.tile_lanes = 16;
  b->build_o.keys_per_lane = 1;
  if (cfg) {
    if (cfg->bucket_size && cfg->bucket_size != 16) {
      fail(GHT_ERR_INVALID_ARG, "batched tables use 16-pair buckets");
      delete b;
      return nullptr;
    }
    if (cfg->num_hashes && cfg->num_hashes != 3) {
      fail(GHT_ERR_INVALID_ARG, "batched tables use three hash functions");
      delete b;
      return nullptr;
    }
    if (cfg->max_chain) b->max_chain = cfg->max_chain;
    if (cfg->max_attempts) b->max_attempts = cfg->max_attempts;
    if (cfg->tile_lanes) b->find_o.tile_lanes = cfg->tile_lanes;
    if (cfg->keys_per_lane) b->find_o.keys_per_lane = cfg->keys_per_lane;
    if (cfg->build_tile_lanes) b->build_o.tile_lanes = cfg->build_tile_lanes;
    if (cfg->build_keys_per_lane) b->build_o.keys_per_lane = cfg->build_keys_per_lane;
    b->find_o.blocks_per_sm = cfg->blocks_per_sm;
    b->build_o.blocks_per_sm = cfg->build_blocks_per_sm;
    b->find_o.count = b->build_o.count = cfg->count_probes != 0;
  }
  if (!ght::batch_find_shape_supported(b->find_o.tile_lanes, b->find_o.keys_per_lane) ||
      !ght::batch_shape_supported(b->build_o.tile_lanes, b->build_o.keys_per_lane)) {
    fail(GHT_ERR_INVALID_ARG, "unsupported launch shape");
    delete b;
    return nullptr;
  }
  b->caps.assign(h_capacities, h_capacities + num_tables);
  b->m.resize(num_tables);
  b->slot_off.assign(num_tables + 1, 0);
  b->attempt.assign(num_tables, 0);
  for (uint32_t t = 0; t < num_tables; ++t) {
    const double lf = h_load_factors[t];
    if (!(lf > 0.0) || !(lf <= 1.0)) {
      fail(GHT_ERR_INVALID_ARG, "table %u: load factor %g is not in (0, 1]", t, lf);
      delete b;
      return nullptr;
    }
    double want = std::ceil((double)h_capacities[t] / (lf * 16.0));  // Sec. III sizing
    if (want < 1.0) want = 1.0;
    if (want > 4294967295.0) {
      fail(GHT_ERR_INVALID_ARG, "table %u needs more than 2^32-1 buckets", t);
      delete b;
      return nullptr;
    }
    b->m[t] = (uint64_t)want;
    b->slot_off[t + 1] = b->slot_off[t] + b->m[t] * 16ull;
  }
  b->total_slots = b->slot_off[num_tables];
  b->slot_bytes = b->total_slots * 8ull;
  const uint64_t meta = num_tables * sizeof(ght::BatchTable) + 2ull * (num_tables + 1) * 8ull + sizeof(ght::Ctrl);
  cudaError_t e = cudaMalloc(&b->slots_mem, b->slot_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&b->meta_mem, meta);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&b->h_tables), num_tables * sizeof(ght::BatchTable));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(GHT_ERR_OOM, "batch allocation (%llu slot bytes): %s", (unsigned long long)b->slot_bytes,
         cudaGetErrorString(e));
    ght_batch_destroy(b);
    return nullptr;
  }
  char *p = static_cast<char *>(b->meta_mem);
  b->d_tables = reinterpret_cast<ght::BatchTable *>(p);
  p += num_tables * sizeof(ght::BatchTable);
  b->d_key_offs = reinterpret_cast<uint64_t *>(p);
  p += (num_tables + 1) * 8ull;
  b->d_query_offs = reinterpret_cast<uint64_t *>(p);
  p += (num_tables + 1) * 8ull;
  b->d_ctrl = reinterpret_cast<ght::Ctrl *>(p);
  for (uint32_t t = 0; t < num_tables; ++t) {
    ght::BatchTable &d = b->h_tables[t];
    memset(&d, 0, sizeof d);
    d.slots = static_cast<uint64_t *>(b->slots_mem) + b->slot_off[t];
    d.m = (uint32_t)b->m[t];
    d.mod = ght::make_fastmod(d.m);
    b->set_constants(t, 0);
  }
  e = cudaMemset(b->d_ctrl, 0, sizeof(ght::Ctrl));
  if (e != cudaSuccess) {
    cuda_fail(e, "clearing the control block");
    ght_batch_destroy(b);
    return nullptr;
  }
  return b;
}

int ght_batch_set_stream(ght_batch *b, void *cuda_stream) {
  if (!b) return fail(GHT_ERR_INVALID_ARG, "batch is NULL");
  if (b->stream != reinterpret_cast<cudaStream_t>(cuda_stream)) b->drop_graph();
  b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  return GHT_OK;
}

int ght_batch_set_layout(ght_batch *b, const uint64_t *h_key_offsets, const uint64_t *h_query_offsets) {
  if (!b || !h_key_offsets || !h_query_offsets) return fail(GHT_ERR_INVALID_ARG, "batch and offsets are required");
  if (h_key_offsets[0] != 0 || h_query_offsets[0] != 0) return fail(GHT_ERR_INVALID_ARG, "offsets must start at 0");
  for (uint32_t t = 0; t < b->T; ++t) {
    if (h_key_offsets[t + 1] < h_key_offsets[t] || h_query_offsets[t + 1] < h_query_offsets[t])
      return fail(GHT_ERR_INVALID_ARG, "offsets must be non-decreasing (table %u)", t);
    if (h_key_offsets[t + 1] - h_key_offsets[t] > b->caps[t])
      return fail(GHT_ERR_CAPACITY, "table %u: %llu keys exceed capacity %llu", t,
                  (unsigned long long)(h_key_offsets[t + 1] - h_key_offsets[t]), (unsigned long long)b->caps[t]);
  }
  b->key_offs.assign(h_key_offsets, h_key_offsets + b->T + 1);
  b->query_offs.assign(h_query_offsets, h_query_offsets + b->T + 1);
  cudaError_t e = cudaMemcpy(b->d_key_offs, h_key_offsets, (b->T + 1) * 8ull, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_query_offs, h_query_offsets, (b->T + 1) * 8ull, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "uploading offsets");
  b->layout_set = true;
  b->drop_graph();
  return GHT_OK;
}

int ght_batch_build(ght_batch *b, const uint32_t *d_keys, const uint32_t *d_values) {
  int rc = check_ready(b);
  if (rc) return rc;
  if (b->key_offs[b->T] > 0 && (!d_keys || !d_values)) return fail(GHT_ERR_INVALID_ARG, "keys or values is NULL");
  b->rebuilds = 0;
  reset_constants(b);
  if ((rc = upload_tables(b, 0, b->T))) return rc;
  cudaEventRecord(b->ev0, b->stream);
  if ((rc = launch_build(b, 0, b->T, d_keys, d_values))) return rc;
  cudaEventRecord(b->ev1, b->stream);
  if ((rc = download_tables(b, 0, b->T))) return rc;
  return repair(b, d_keys, d_values, nullptr, nullptr);
}

int ght_batch_find(const ght_batch *b, const uint32_t *d_queries, uint32_t *d_out) {
  const int rc = check_ready(b);
  if (rc) return rc;
  if (b->tables_failed) return fail(GHT_ERR_NOT_BUILT, "%u tables have no successful build", b->tables_failed);
  if (b->query_offs[b->T] > 0 && (!d_queries || !d_out)) return fail(GHT_ERR_INVALID_ARG, "queries or out is NULL");
  return launch_find(b, 0, b->T, d_queries, d_out);
}

int ght_batch_run(ght_batch *b, const uint32_t *d_keys, const uint32_t *d_values, const uint32_t *d_queries,
                  uint32_t *d_out) {
  int rc = check_ready(b);
  if (rc) return rc;
  if ((b->key_offs[b->T] > 0 && (!d_keys || !d_values)) || (b->query_offs[b->T] > 0 && (!d_queries || !d_out)))
    return fail(GHT_ERR_INVALID_ARG, "arrays are NULL");
  if (b->exec && (b->g_keys != d_keys || b->g_values != d_values || b->g_queries != d_queries ||
                  b->g_out != d_out || b->g_shape != b->shape_sig()))
    b->drop_graph();
  cudaError_t e;
  if (!b->exec) {
    // One graph: descriptors in, fill, insert, find, descriptors (status) out.
    // Captured on the batch's private stream (the legacy default stream
    // cannot be captured), launched on the caller's stream.
    cudaGraph_t graph = nullptr;
    const cudaStream_t user = b->stream;
    b->stream = b->capture_stream;
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      b->stream = user;
      return cuda_fail(e, "beginning graph capture");
    }
    int crc = upload_tables(b, 0, b->T);
    // external event-record nodes, so the events time the graph's execution
    if (!crc && cudaEventRecordWithFlags(b->ev0, b->stream, cudaEventRecordExternal) != cudaSuccess)
      crc = fail(GHT_ERR_CUDA, "event in capture");
    if (!crc) crc = launch_build(b, 0, b->T, d_keys, d_values);
    if (!crc) crc = launch_find(b, 0, b->T, d_queries, d_out);
    if (!crc && cudaEventRecordWithFlags(b->ev1, b->stream, cudaEventRecordExternal) != cudaSuccess)
      crc = fail(GHT_ERR_CUDA, "event in capture");
    if (!crc) {
      e = cudaMemcpyAsync(b->h_tables, b->d_tables, b->T * sizeof(ght::BatchTable), cudaMemcpyDeviceToHost, b->stream);
      if (e != cudaSuccess) crc = cuda_fail(e, "status read-back in capture");
    }
    e = cudaStreamEndCapture(b->stream, &graph);
    b->stream = user;
    if (crc) {
      if (graph) cudaGraphDestroy(graph);
      return crc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "ending graph capture");
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      return cuda_fail(e, "instantiating the batch graph");
    }
    b->g_keys = d_keys;
    b->g_values = d_values;
    b->g_queries = d_queries;
    b->g_out = d_out;
    b->g_shape = b->shape_sig();
  }
  b->rebuilds = 0;
  reset_constants(b);  // the graph copies the pinned descriptors in when it runs
  e = cudaGraphLaunch(b->exec, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "launching the batch graph");
  b->graph_launches++;
  e = cudaEventRecord(b->done, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "recording an event");
  if ((rc = wait_event(b->done))) return rc;
  float ms = 0.f;
  b->last_run_ms = cudaEventElapsedTime(&ms, b->ev0, b->ev1) == cudaSuccess ? ms : -1.0;
  cudaGetLastError();
  return repair(b, d_keys, d_values, d_queries, d_out);
}

int ght_batch_autotune(ght_batch *b, const uint32_t *d_keys, const uint32_t *d_values, const uint32_t *d_queries,
                       uint32_t *d_out) {
  int rc = check_ready(b);
  if (rc) return rc;
  // tile shapes (lanes per bucket, keys per lane), then the grid (resident
  // blocks per SM; 0 = as many as fit) of the chosen shape
  static const int kBuild[][2] = {{16, 1}, {8, 1}, {8, 2}, {4, 2}};
  static const int kFind[][2] = {{4, 2}, {4, 1}, {8, 2}, {8, 1}, {16, 1}, {4, 6}};  // {4, 6}: the staged find
  static const int kGrid[] = {0, 1, 2, 3, 4};
  if (b->build_o.blocks_per_sm < 0 || b->find_o.blocks_per_sm < 0) return fail(GHT_ERR_INVALID_ARG, "negative grid");
  auto time_between = [&](float *out_ms) -> int {
    const cudaError_t e = cudaEventSynchronize(b->ev1);
    if (e != cudaSuccess) return cuda_fail(e, "timing a candidate");
    return cudaEventElapsedTime(out_ms, b->ev0, b->ev1) == cudaSuccess ? GHT_OK : fail(GHT_ERR_CUDA, "event timing");
  };
  auto time_build = [&](float *total) -> int {
    *total = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
      int r = ght_batch_build(b, d_keys, d_values);
      if (r) return r;
      float ms = 0.f;
      if ((r = time_between(&ms))) return r;
      if (rep > 0) *total += ms;  // the first repetition warms up
    }
    return GHT_OK;
  };
  auto time_find = [&](float *total) -> int {
    *total = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(b->ev0, b->stream);
      int r = launch_find(b, 0, b->T, d_queries, d_out);
      if (r) return r;
      cudaEventRecord(b->ev1, b->stream);
      float ms = 0.f;
      if ((r = time_between(&ms))) return r;
      if (rep > 0) *total += ms;
    }
    return GHT_OK;
  };
  float best = 3.0e38f, total = 0.f;
  ght::LaunchOpts best_o = b->build_o;
  b->build_o.blocks_per_sm = 0;
  for (const auto &c : kBuild) {
    b->build_o.tile_lanes = c[0];
    b->build_o.keys_per_lane = c[1];
    if ((rc = time_build(&total))) return rc;
    if (total < best) {
      best = total;
      best_o = b->build_o;
    }
  }
  for (int g : kGrid) {
    if (g == 0) continue;  // measured with the shapes
    b->build_o = best_o;
    b->build_o.blocks_per_sm = g;
    if ((rc = time_build(&total))) return rc;
    if (total < best) {
      best = total;
      best_o = b->build_o;
    }
  }
  b->build_o = best_o;
  if ((rc = ght_batch_build(b, d_keys, d_values))) return rc;
  best = 3.0e38f;
  best_o = b->find_o;
  b->find_o.blocks_per_sm = 0;
  for (const auto &c : kFind) {
    b->find_o.tile_lanes = c[0];
    b->find_o.keys_per_lane = c[1];
    if ((rc = time_find(&total))) return rc;
    if (total < best) {
      best = total;
      best_o = b->find_o;
    }
  }
  for (int g : kGrid) {
    if (g == 0) continue;
    b->find_o = best_o;
    b->find_o.blocks_per_sm = g;
    if ((rc = time_find(&total))) return rc;
    if (total < best) {
      best = total;
      best_o = b->find_o;
    }
  }
  b->find_o = best_o;
  b->tuned = 1;
  b->drop_graph();
  return GHT_OK;
}

int ght_batch_stats(const ght_batch *b, ght_batch_stats_t *out) {
  if (!b || !out) return fail(GHT_ERR_INVALID_ARG, "batch or out is NULL");
  memset(out, 0, sizeof *out);
  out->num_tables = b->T;
  out->tables_failed = b->tables_failed;
  out->total_keys = b->layout_set ? b->key_offs[b->T] : 0;
  out->total_queries = b->layout_set ? b->query_offs[b->T] : 0;
  out->total_slots = b->total_slots;
  out->table_bytes = b->slot_bytes;
  out->rebuilds = b->rebuilds;
  out->tuned = b->tuned;
  out->tile_lanes = b->find_o.tile_lanes;
  out->keys_per_lane = b->find_o.keys_per_lane;
  out->build_tile_lanes = b->build_o.tile_lanes;
  out->build_keys_per_lane = b->build_o.keys_per_lane;
  out->last_run_ms = b->last_run_ms;
  out->graph_launches = b->graph_launches;
  out->blocks_per_sm = b->find_o.blocks_per_sm;
  out->build_blocks_per_sm = b->build_o.blocks_per_sm;
  return GHT_OK;
}

int ght_batch_table_stats(const ght_batch *b, uint32_t table, ght_stats_t *out) {
  if (!b || !out || table >= b->T) return fail(GHT_ERR_INVALID_ARG, "batch, table or out invalid");
  memset(out, 0, sizeof *out);
  out->scheme = GHT_BCHT;
  out->bucket_size = 16;
  out->num_hashes = b->h;
  out->num_buckets = b->m[table];
  out->num_slots = b->m[table] * 16ull;
  out->capacity = b->caps[table];
  out->n_stored = b->layout_set && b->h_tables[table].status == 0u ? b->key_offs[table + 1] - b->key_offs[table] : 0;
  out->load_factor = (double)out->n_stored / (double)out->num_slots;
  out->attempts = b->attempt[table] + 1;
  out->max_chain = b->max_chain;
  for (int i = 0; i < 4; ++i) {
    out->hash_a[i] = b->h_tables[table].a[i];
    out->hash_c[i] = b->h_tables[table].c[i];
  }
  out->table_bytes = b->m[table] * 128ull;
  out->built = b->h_tables[table].status == 0u ? 1 : 0;
  out->tile_lanes = b->find_o.tile_lanes;
  out->keys_per_lane = b->find_o.keys_per_lane;
  out->build_tile_lanes = b->build_o.tile_lanes;
  out->build_keys_per_lane = b->build_o.keys_per_lane;
  out->last_fill_ms = out->last_insert_ms = out->last_find_ms = out->last_group_ms = -1.0;
  return GHT_OK;
}

int ght_batch_export(const ght_batch *b, uint32_t table, uint64_t *h_slots, uint64_t n_slots) {
  if (!b || !h_slots || table >= b->T) return fail(GHT_ERR_INVALID_ARG, "batch, table or slots invalid");
  const uint64_t total = b->m[table] * 16ull;
  if (n_slots < total) return fail(GHT_ERR_INVALID_ARG, "h_slots too small");
  cudaError_t e = cudaMemcpyAsync(h_slots, static_cast<uint64_t *>(b->slots_mem) + b->slot_off[table], total * 8ull,
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "exporting slots");
  e = cudaEventRecord(b->done, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "recording an event");
  return wait_event(b->done);
}

void ght_batch_destroy(ght_batch *b) {
  if (!b) return;
  b->drop_graph();
  cudaStreamSynchronize(b->stream);
  if (b->slots_mem) cudaFree(b->slots_mem);
  if (b->meta_mem) cudaFree(b->meta_mem);
  if (b->h_tables) cudaFreeHost(b->h_tables);
  if (b->done) cudaEventDestroy(b->done);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  delete b;
}

}  // extern "C"
