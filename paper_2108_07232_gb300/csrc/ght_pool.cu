// ght_pool.cu -- a served pool of device-resident BCHT tables (C ABI in
// include/ght.h). Not in the paper: it serves the paper's tables to a stream
// of requests.
//
// Two host threads drive the device:
//   * the find scheduler keeps up to two batched launches in flight. Whenever
//     one completes it packs every pending find request whose table is ready
//     (oldest first, up to a query cap) into the next launch: one upload of
//     per-request descriptors, a gather of the requests' queries into one
//     array, one batched find, a scatter of the answers. Requests that arrive
//     while launches run join the next launch (continuous batching).
//   * the build worker admits build requests in arrival order when the table
//     fits in the HBM budget, allocates its storage from the library pool and
//     builds it on its own stream, so builds overlap finds on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ght.h"
#include "ght_batch.h"
#include "ght_host.h"

using ght::host::cuda_fail;
using ght::host::fail;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum TableState { kPending = 0, kBuilding, kReady, kFailed, kDropped };
enum Kind { kFind = 0, kBuild = 1 };

struct PoolTable {
  ght_table *t = nullptr;
  void *storage = nullptr;
  uint64_t bytes = 0;
  int state = kPending;
  int refs = 0;  // in-flight find launches that read the table
  ght::BatchTable desc;
};

struct Req {
  int kind = kFind;
  uint32_t table = 0;
  const uint32_t *in = nullptr, *values = nullptr;
  uint32_t *out = nullptr;
  uint64_t n = 0;
  uint64_t capacity = 0, seed = 0;
  double lf = 0.0;
  double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
  int status = -1;  // < 0 while pending
  int launch_requests = 0;
};

constexpr int kMaxInFlight = 2;
constexpr uint32_t kMaxReqPerLaunch = 4096;

// Host and device blocks of one launch: descriptors, query offsets, source
// and destination pointers; staging for the packed queries and answers.
struct Slot {
  bool busy = false;
  void *pinned = nullptr;  // host: [desc R][offs R+1][src R][dst R]
  void *dev = nullptr;     // device copy of the same layout
  void *staging = nullptr;
  uint64_t staging_bytes = 0;
  cudaEvent_t ev = nullptr;
  std::vector<uint64_t> tickets;
  std::vector<uint32_t> tables;
};

constexpr uint64_t kSlotBytes =
    kMaxReqPerLaunch * (sizeof(ght::BatchTable) + 8ull + 8ull + 8ull) + 8ull;

}  // namespace

struct ght_pool {
  uint64_t budget = 0, used = 0;
  ght_config cfg;
  ght::LaunchOpts find_o;
  uint64_t max_batch_queries = 1ull << 22;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_find, cv_build, cv_done;
  std::deque<PoolTable> tables;  // a deque: submit_build appends while workers hold references
  std::unordered_map<uint64_t, Req> reqs;
  std::deque<uint64_t> find_q, build_q;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread find_thr, build_thr;
  cudaStream_t find_stream = nullptr, build_stream = nullptr;
  Slot slots[kMaxInFlight];
  // stats
  uint64_t find_launches = 0, finds_done = 0, queries_done = 0, builds_done = 0, builds_refused = 0;
  uint64_t requests_packed = 0;
  int thread_error = 0;

  void complete(uint64_t ticket, int status) {
    auto it = reqs.find(ticket);
    if (it == reqs.end()) return;
    it->second.status = status;
    it->second.t_done = now_s();
  }

  void release_table(uint32_t id) {  // with mu held
    PoolTable &pt = tables[id];
    if (pt.state == kDropped && pt.refs == 0 && pt.t) {
      ght_destroy(pt.t);
      pt.t = nullptr;
      if (pt.storage) cudaFreeAsync(pt.storage, build_stream);
      pt.storage = nullptr;
      used -= pt.bytes;
      pt.bytes = 0;
      cv_build.notify_all();
    }
  }

  void find_loop();
  void build_loop();
  int launch_finds(Slot &sl, std::vector<uint64_t> &batch);
};

int ght_pool::launch_finds(Slot &sl, std::vector<uint64_t> &batch) {
  const uint32_t R = (uint32_t)batch.size();
  char *h = static_cast<char *>(sl.pinned);
  ght::BatchTable *desc = reinterpret_cast<ght::BatchTable *>(h);
  uint64_t *offs = reinterpret_cast<uint64_t *>(h + R * sizeof(ght::BatchTable));
  const uint32_t **src = reinterpret_cast<const uint32_t **>(offs + R + 1);
  uint32_t **dst = reinterpret_cast<uint32_t **>(offs + R + 1 + R);
  offs[0] = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (uint32_t i = 0; i < R; ++i) {
      Req &r = reqs[batch[i]];
      desc[i] = tables[r.table].desc;
      offs[i + 1] = offs[i] + r.n;
      src[i] = r.in;
      dst[i] = r.out;
      r.t_start = now_s();
      r.launch_requests = (int)R;
    }
  }
  const uint64_t total = offs[R];
  const uint64_t layout = R * sizeof(ght::BatchTable) + (R + 1) * 8ull + 2ull * R * 8ull;
  char *d = static_cast<char *>(sl.dev);
  ght::BatchTable *d_desc = reinterpret_cast<ght::BatchTable *>(d);
  uint64_t *d_offs = reinterpret_cast<uint64_t *>(d + R * sizeof(ght::BatchTable));
  const uint32_t *const *d_src = reinterpret_cast<const uint32_t *const *>(d_offs + R + 1);
  uint32_t *const *d_dst = reinterpret_cast<uint32_t *const *>(d_offs + R + 1 + R);
  const uint64_t need = 2ull * total * sizeof(uint32_t) + 512;
  if (sl.staging_bytes < need) {
    if (sl.staging) cudaFreeAsync(sl.staging, find_stream);
    sl.staging = nullptr;
    sl.staging_bytes = 0;
    const uint64_t want = std::max<uint64_t>(need, 2ull * max_batch_queries * sizeof(uint32_t) + 512);
    cudaError_t e = ght::host::pool_alloc(&sl.staging, want, find_stream);
    if (e != cudaSuccess) return cuda_fail(e, "pool staging");
    sl.staging_bytes = want;
  }
  uint32_t *q = static_cast<uint32_t *>(sl.staging);
  uint32_t *o = q + ((total + 63) & ~63ull);
  cudaError_t e = cudaMemcpyAsync(sl.dev, sl.pinned, layout, cudaMemcpyHostToDevice, find_stream);
  if (e == cudaSuccess) e = ght::launch_segment_gather(d_src, d_offs, R, q, total, find_stream);
  if (e == cudaSuccess) {
    ght::BatchView bv;
    memset(&bv, 0, sizeof bv);
    bv.tables = d_desc;
    bv.key_offs = d_offs;
    bv.query_offs = d_offs;
    bv.ctrl = nullptr;
    bv.t_lo = 0;
    bv.t_hi = R;
    bv.h = 3;
    e = ght::launch_batch_find(bv, q, o, total, find_o, find_stream);
  }
  if (e == cudaSuccess) e = ght::launch_segment_scatter(o, d_dst, d_offs, R, total, find_stream);
  if (e == cudaSuccess) e = cudaEventRecord(sl.ev, find_stream);
  if (e != cudaSuccess) return cuda_fail(e, "launching pooled finds");
  sl.busy = true;
  sl.tickets.swap(batch);
  return GHT_OK;
}

void ght_pool::find_loop() {
  cudaSetDevice(device);
  std::vector<uint64_t> batch;
  for (;;) {
    // retire completed launches
    bool progressed = false;
    for (auto &sl : slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.ev);
      if (q == cudaErrorNotReady) continue;
      std::lock_guard<std::mutex> lock(mu);
      const int st = q == cudaSuccess ? GHT_OK : GHT_ERR_CUDA;
      for (uint64_t tk : sl.tickets) {
        auto it = reqs.find(tk);
        if (it != reqs.end()) {
          queries_done += it->second.n;
          PoolTable &pt = tables[it->second.table];
          pt.refs--;
          release_table(it->second.table);
        }
        complete(tk, st);
        finds_done++;
      }
      sl.tickets.clear();
      sl.busy = false;
      progressed = true;
      cv_done.notify_all();
    }
    // pack the next launch into a free slot
    Slot *free_slot = nullptr;
    for (auto &sl : slots)
      if (!sl.busy) free_slot = &sl;
    bool any_busy = false;
    for (auto &sl : slots) any_busy |= sl.busy;
    {
      std::unique_lock<std::mutex> lock(mu);
      if (stop && find_q.empty() && !any_busy) return;
      batch.clear();
      if (free_slot) {
        uint64_t total = 0;
        for (auto it = find_q.begin(); it != find_q.end() && batch.size() < kMaxReqPerLaunch;) {
          Req &r = reqs[*it];
          const PoolTable &pt = tables[r.table];
          if (pt.state == kFailed || pt.state == kDropped) {
            complete(*it, GHT_ERR_NOT_BUILT);
            it = find_q.erase(it);
            cv_done.notify_all();
            continue;
          }
          if (pt.state != kReady) {
            ++it;
            continue;
          }
          if (!batch.empty() && total + r.n > max_batch_queries) break;
          total += r.n;
          batch.push_back(*it);
          tables[r.table].refs++;
          it = find_q.erase(it);
        }
        if (!batch.empty()) {
          find_launches++;
          requests_packed += batch.size();
        }
      }
      if (batch.empty() && !progressed) {
        if (any_busy) {
          lock.unlock();
          std::this_thread::yield();
        } else {
          cv_find.wait_for(lock, std::chrono::microseconds(200));
        }
        continue;
      }
    }
    if (!batch.empty()) {
      const int rc = launch_finds(*free_slot, batch);
      if (rc) {
        std::lock_guard<std::mutex> lock(mu);
        thread_error = rc;
        for (uint64_t tk : batch) {
          tables[reqs[tk].table].refs--;
          complete(tk, rc);
        }
        cv_done.notify_all();
      }
    }
  }
}

void ght_pool::build_loop() {
  cudaSetDevice(device);
  for (;;) {
    uint64_t tk = 0;
    Req r;
    PoolTable *ptp = nullptr;  // element address taken under the lock (stable in a deque)
    {
      std::unique_lock<std::mutex> lock(mu);
      for (;;) {
        if (stop) return;
        if (!build_q.empty()) {
          Req &head = reqs[build_q.front()];
          const uint64_t bytes = ght_table_bytes(GHT_BCHT, head.capacity, head.lf, &cfg);
          if (bytes == 0 || bytes > budget) {  // can never fit: refuse
            builds_refused++;
            tables[head.table].state = kFailed;
            complete(build_q.front(), bytes == 0 ? GHT_ERR_INVALID_ARG : GHT_ERR_OOM);
            build_q.pop_front();
            cv_done.notify_all();
            continue;
          }
          if (used + bytes <= budget) {  // admitted: reserve the budget
            tk = build_q.front();
            build_q.pop_front();
            used += bytes;
            tables[head.table].bytes = bytes;
            tables[head.table].state = kBuilding;
            head.t_start = now_s();
            r = head;
            ptp = &tables[head.table];
            break;
          }
        }
        cv_build.wait_for(lock, std::chrono::milliseconds(2));
      }
    }
    PoolTable &pt = *ptp;
    int rc = GHT_OK;
    void *storage = nullptr;
    cudaError_t e = ght::host::pool_alloc(&storage, pt.bytes, build_stream);
    ght_table *t = nullptr;
    if (e != cudaSuccess) {
      cudaGetLastError();
      rc = fail(GHT_ERR_OOM, "pool table allocation: %s", cudaGetErrorString(e));
    } else {
      t = ght_create_ex(GHT_BCHT, r.capacity, r.lf, r.seed, &cfg, storage, pt.bytes);
      if (!t) rc = GHT_ERR_INVALID_ARG;
    }
    if (rc == GHT_OK) rc = ght_set_stream(t, build_stream);
    if (rc == GHT_OK) rc = ght_build(t, r.values ? r.in : nullptr, r.values, r.n);
    std::lock_guard<std::mutex> lock(mu);
    pt.t = t;
    pt.storage = storage;
    if (rc == GHT_OK && ght::table_descriptor(t, &pt.desc)) {
      pt.state = kReady;
      builds_done++;
    } else {
      pt.state = kDropped;
      if (!t && storage) {
        cudaFreeAsync(storage, build_stream);
        pt.storage = nullptr;
        used -= pt.bytes;
        pt.bytes = 0;
      }
      release_table(r.table);
      pt.state = kFailed;
      if (rc == GHT_OK) rc = GHT_ERR_INVALID_ARG;
    }
    complete(tk, rc);
    cv_done.notify_all();
    cv_find.notify_all();
  }
}

extern "C" {

ght_pool *ght_pool_create(uint64_t hbm_budget_bytes, const ght_config *cfg) {
  ght_pool *p = new (std::nothrow) ght_pool();
  if (!p) {
    fail(GHT_ERR_OOM, "host allocation failed");
    return nullptr;
  }
  p->budget = hbm_budget_bytes;
  ght_default_config(GHT_BCHT, &p->cfg);
  if (cfg) {
    if (cfg->max_chain) p->cfg.max_chain = cfg->max_chain;
    if (cfg->max_attempts) p->cfg.max_attempts = cfg->max_attempts;
    if (cfg->build_tile_lanes) p->cfg.build_tile_lanes = cfg->build_tile_lanes;
    if (cfg->build_keys_per_lane) p->cfg.build_keys_per_lane = cfg->build_keys_per_lane;
    if (cfg->tile_lanes) p->cfg.tile_lanes = cfg->tile_lanes;
    if (cfg->keys_per_lane) p->cfg.keys_per_lane = cfg->keys_per_lane;
  }
  p->find_o.tile_lanes = p->cfg.tile_lanes;
  p->find_o.keys_per_lane = p->cfg.keys_per_lane;
  if (!ght::batch_find_shape_supported(p->find_o.tile_lanes, p->find_o.keys_per_lane)) {
    fail(GHT_ERR_INVALID_ARG, "unsupported find shape");
    delete p;
    return nullptr;
  }
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->find_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->build_stream, cudaStreamNonBlocking);
  for (auto &sl : p->slots) {
    if (e == cudaSuccess) e = cudaMallocHost(&sl.pinned, kSlotBytes);
    if (e == cudaSuccess) e = cudaMalloc(&sl.dev, kSlotBytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    cuda_fail(e, "creating the pool");
    ght_pool_destroy(p);
    return nullptr;
  }
  p->find_thr = std::thread([p] { p->find_loop(); });
  p->build_thr = std::thread([p] { p->build_loop(); });
  return p;
}

uint64_t ght_pool_submit_build(ght_pool *p, uint64_t capacity, double load_factor, uint64_t seed,
                               const uint32_t *d_keys, const uint32_t *d_values, uint64_t n, uint32_t *table_id) {
  if (!p || !table_id || n > capacity || (n > 0 && (!d_keys || !d_values))) {
    fail(GHT_ERR_INVALID_ARG, "pool, table_id, keys and values are required and n <= capacity");
    return 0;
  }
  std::lock_guard<std::mutex> lock(p->mu);
  const uint64_t tk = p->next_ticket++;
  Req r;
  r.kind = kBuild;
  r.table = (uint32_t)p->tables.size();
  r.in = d_keys;
  r.values = d_values;
  r.n = n;
  r.capacity = capacity;
  r.lf = load_factor;
  r.seed = seed;
  r.t_submit = now_s();
  p->tables.emplace_back();
  p->reqs.emplace(tk, r);
  p->build_q.push_back(tk);
  *table_id = r.table;
  p->cv_build.notify_all();
  return tk;
}

uint64_t ght_pool_submit_find(ght_pool *p, uint32_t table_id, const uint32_t *d_queries, uint32_t *d_out,
                              uint64_t n) {
  if (!p || (n > 0 && (!d_queries || !d_out))) {
    fail(GHT_ERR_INVALID_ARG, "pool, queries and out are required");
    return 0;
  }
  std::lock_guard<std::mutex> lock(p->mu);
  if (table_id >= p->tables.size()) {
    fail(GHT_ERR_INVALID_ARG, "no table %u", table_id);
    return 0;
  }
  const uint64_t tk = p->next_ticket++;
  Req r;
  r.kind = kFind;
  r.table = table_id;
  r.in = d_queries;
  r.out = d_out;
  r.n = n;
  r.t_submit = now_s();
  p->reqs.emplace(tk, r);
  if (n == 0) {
    p->complete(tk, GHT_OK);
  } else {
    p->find_q.push_back(tk);
    p->cv_find.notify_all();
  }
  return tk;
}

static void fill_result(const Req &r, ght_pool_result_t *out) {
  if (!out) return;
  out->status = r.status;
  out->kind = r.kind;
  out->table = r.table;
  out->n = r.n;
  out->queue_s = r.t_start > 0.0 ? r.t_start - r.t_submit : 0.0;
  out->latency_s = r.t_done - r.t_submit;
  out->launch_requests = r.launch_requests;
}

int ght_pool_wait(ght_pool *p, uint64_t ticket, double timeout_s, ght_pool_result_t *out) {
  if (!p) return fail(GHT_ERR_INVALID_ARG, "pool is NULL");
  std::unique_lock<std::mutex> lock(p->mu);
  auto it = p->reqs.find(ticket);
  if (it == p->reqs.end()) return fail(GHT_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (it->second.status < 0) {
    if (p->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && it->second.status < 0)
      return fail(GHT_ERR_DEVICE_TIMEOUT, "request %llu not done within %.3f s", (unsigned long long)ticket,
                  timeout_s);
    it = p->reqs.find(ticket);
  }
  fill_result(it->second, out);
  const int st = it->second.status;
  p->reqs.erase(it);
  if (st != GHT_OK) return fail(st, "request %llu failed with status %d", (unsigned long long)ticket, st);
  return GHT_OK;
}

int ght_pool_drop_table(ght_pool *p, uint32_t table_id) {
  if (!p) return fail(GHT_ERR_INVALID_ARG, "pool is NULL");
  std::lock_guard<std::mutex> lock(p->mu);
  if (table_id >= p->tables.size()) return fail(GHT_ERR_INVALID_ARG, "no table %u", table_id);
  PoolTable &pt = p->tables[table_id];
  if (pt.state == kPending || pt.state == kBuilding) return fail(GHT_ERR_INVALID_ARG, "table %u is being built", table_id);
  pt.state = kDropped;
  p->release_table(table_id);
  return GHT_OK;
}

int ght_pool_stats(ght_pool *p, ght_pool_stats_t *out) {
  if (!p || !out) return fail(GHT_ERR_INVALID_ARG, "pool or out is NULL");
  std::lock_guard<std::mutex> lock(p->mu);
  memset(out, 0, sizeof *out);
  out->budget_bytes = p->budget;
  out->used_bytes = p->used;
  out->tables = (uint32_t)p->tables.size();
  for (const auto &pt : p->tables) out->tables_ready += pt.state == kReady;
  out->find_launches = p->find_launches;
  out->finds_done = p->finds_done;
  out->queries_done = p->queries_done;
  out->builds_done = p->builds_done;
  out->builds_refused = p->builds_refused;
  out->mean_requests_per_launch = p->find_launches ? (double)p->requests_packed / (double)p->find_launches : 0.0;
  out->pending_finds = p->find_q.size();
  out->pending_builds = p->build_q.size();
  return p->thread_error;
}

// Replay a request trace against the pool (serial = 0) or with plain calls,
// one request at a time in arrival order (serial = 1), measuring each
// request's latency from its scheduled arrival to its completion.
int ght_pool_replay(ght_pool *p, const ght_pool_request_t *trace, uint64_t count, int serial, double *latency_s,
                    int32_t *status, double *makespan_s) {
  if (!p || (count > 0 && !trace)) return fail(GHT_ERR_INVALID_ARG, "pool and trace are required");
  std::vector<uint64_t> tickets(count, 0);
  const double t0 = now_s();
  auto wait_until = [&](double at) {
    while (now_s() < t0 + at) {
      if (t0 + at - now_s() > 200e-6) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  };
  int rc_all = GHT_OK;
  if (!serial) {
    for (uint64_t i = 0; i < count; ++i) {
      const ght_pool_request_t &q = trace[i];
      wait_until(q.arrival_s);
      uint32_t id = 0;
      tickets[i] = q.kind == 1 ? ght_pool_submit_build(p, q.capacity, q.load_factor, q.seed, q.d_in, q.d_values, q.n, &id)
                               : ght_pool_submit_find(p, q.table, q.d_in, q.d_out, q.n);
      if (tickets[i]) {  // the arrival time is the latency origin
        std::lock_guard<std::mutex> lock(p->mu);
        auto it = p->reqs.find(tickets[i]);
        if (it != p->reqs.end()) it->second.t_submit = t0 + q.arrival_s;
      }
    }
    double last = t0;
    for (uint64_t i = 0; i < count; ++i) {
      ght_pool_result_t r;
      memset(&r, 0, sizeof r);
      int rc = tickets[i] ? ght_pool_wait(p, tickets[i], 600.0, &r) : GHT_ERR_INVALID_ARG;
      if (rc && rc_all == GHT_OK) rc_all = rc;
      if (latency_s) latency_s[i] = r.latency_s;
      if (status) status[i] = rc;
      last = std::max(last, t0 + trace[i].arrival_s + r.latency_s);
    }
    if (makespan_s) *makespan_s = last - t0;
    return rc_all;
  }
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "creating a stream");
  cudaEvent_t ev = nullptr;
  e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaStreamDestroy(s);
    return cuda_fail(e, "creating an event");
  }
  double last = t0;
  for (uint64_t i = 0; i < count; ++i) {
    const ght_pool_request_t &q = trace[i];
    wait_until(q.arrival_s);
    int rc = GHT_OK;
    if (q.kind == 1) {
      uint32_t id = 0;
      const uint64_t tk = ght_pool_submit_build(p, q.capacity, q.load_factor, q.seed, q.d_in, q.d_values, q.n, &id);
      rc = tk ? ght_pool_wait(p, tk, 600.0, nullptr) : GHT_ERR_INVALID_ARG;
    } else {
      ght_table *t = nullptr;
      {
        std::lock_guard<std::mutex> lock(p->mu);
        if (q.table < p->tables.size() && p->tables[q.table].state == kReady) t = p->tables[q.table].t;
      }
      if (!t) rc = fail(GHT_ERR_NOT_BUILT, "table %u is not ready", q.table);
      if (rc == GHT_OK) rc = ght_set_stream(t, s);
      if (rc == GHT_OK) rc = ght_find(t, q.d_in, q.d_out, q.n);
      if (rc == GHT_OK) {
        e = cudaEventRecord(ev, s);
        rc = e == cudaSuccess ? ght::host::wait_event(ev) : cuda_fail(e, "recording an event");
      }
    }
    const double done = now_s();
    if (latency_s) latency_s[i] = done - (t0 + q.arrival_s);
    if (status) status[i] = rc;
    if (rc && rc_all == GHT_OK) rc_all = rc;
    last = done;
  }
  if (makespan_s) *makespan_s = last - t0;
  cudaEventDestroy(ev);
  cudaStreamDestroy(s);
  return rc_all;
}

void ght_pool_destroy(ght_pool *p) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lock(p->mu);
    p->stop = true;
  }
  p->cv_find.notify_all();
  p->cv_build.notify_all();
  if (p->find_thr.joinable()) p->find_thr.join();
  if (p->build_thr.joinable()) p->build_thr.join();
  if (p->find_stream) cudaStreamSynchronize(p->find_stream);
  if (p->build_stream) cudaStreamSynchronize(p->build_stream);
  for (auto &pt : p->tables) {
    if (pt.t) ght_destroy(pt.t);
    if (pt.storage) cudaFreeAsync(pt.storage, p->build_stream);
  }
  for (auto &sl : p->slots) {
    if (sl.staging) cudaFreeAsync(sl.staging, p->find_stream);
    if (sl.pinned) cudaFreeHost(sl.pinned);
    if (sl.dev) cudaFree(sl.dev);
    if (sl.ev) cudaEventDestroy(sl.ev);
  }
  if (p->find_stream) {
    cudaStreamSynchronize(p->find_stream);
    cudaStreamDestroy(p->find_stream);
  }
  if (p->build_stream) {
    cudaStreamSynchronize(p->build_stream);
    cudaStreamDestroy(p->build_stream);
  }
  delete p;
}

}  // extern "C"
