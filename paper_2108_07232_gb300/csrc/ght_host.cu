// ght_host.cu -- host helpers shared by the C-ABI translation units.
#include "ght_host.h"

#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>

#include "ght.h"
#include "ght_device.cuh"

namespace ght {
namespace host {

namespace {
thread_local std::string g_err;
}

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  return fail(GHT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

const char *last_error() { return g_err.c_str(); }

uint64_t splitmix64(uint64_t &state) {
  state += 0x9E3779B97F4A7C15ull;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void derive_constants(uint64_t seed, uint32_t attempt, int h, uint32_t a[4], uint32_t c[4]) {
  uint64_t st = seed ^ ((uint64_t)attempt * 0x9E3779B97F4A7C15ull);
  for (int i = 0; i < h; ++i) {
    const uint64_t x = splitmix64(st), y = splitmix64(st);
    a[i] = (uint32_t)(1u + x % (uint64_t)(kPrime - 1u));
    c[i] = (uint32_t)(y % (uint64_t)kPrime);
  }
  for (int i = h; i < 4; ++i) a[i] = c[i] = 0;
}

uint32_t derive_rng_seed(uint64_t seed, uint32_t attempt) {
  uint64_t r = seed ^ 0x4B45524E454Cull ^ ((uint64_t)attempt << 32);
  return (uint32_t)splitmix64(r) | 1u;
}

int wait_event(cudaEvent_t ev) {
  const char *env = getenv("GHT_WAIT_TIMEOUT_S");
  const double limit = env && atof(env) > 0.0 ? atof(env) : 300.0;
  const auto t0 = std::chrono::steady_clock::now();
  for (uint64_t spins = 0;; ++spins) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return GHT_OK;
    if (e != cudaErrorNotReady) return cuda_fail(e, "waiting for the device");
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > limit)
      return fail(GHT_ERR_DEVICE_TIMEOUT, "device work did not finish within %.0f s", limit);
    if (spins > 1000) std::this_thread::sleep_for(std::chrono::microseconds(20));
    else std::this_thread::yield();
  }
}

// The library's own stream-ordered pool (one per device) for staging and
// scratch; freed blocks stay cached in it, so repeated calls do not return
// to the driver.
cudaError_t pool_alloc(void **p, uint64_t bytes, cudaStream_t s) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
      cudaMemPoolProps props;
      memset(&props, 0, sizeof props);
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&pools[dev], &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pool = pools[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

}  // namespace host
}  // namespace ght
