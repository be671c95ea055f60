// ght_host.h -- host helpers shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ght {
namespace host {

// Record a thread-local error message and return `code`.
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
const char *last_error();

// SplitMix64 step (Steele, Lea, Flood, OOPSLA 2014).
uint64_t splitmix64(uint64_t &state);

// Hash constants of (seed, attempt): a_i = 1 + x mod (p-1), c_i = y mod p,
// drawn a_0, c_0, a_1, ... from SplitMix64 seeded with
// seed XOR (attempt * 0x9E3779B97F4A7C15); entries beyond h are zero.
void derive_constants(uint64_t seed, uint32_t attempt, int h, uint32_t a[4], uint32_t c[4]);

// Per-attempt seed of the eviction xorshift.
uint32_t derive_rng_seed(uint64_t seed, uint32_t attempt);

// Wait for `ev` by polling with a deadline (GHT_WAIT_TIMEOUT_S, default 300 s).
int wait_event(cudaEvent_t ev);

// Stream-ordered allocation from the library's own pool (one per device).
cudaError_t pool_alloc(void **p, uint64_t bytes, cudaStream_t s);

}  // namespace host
}  // namespace ght
