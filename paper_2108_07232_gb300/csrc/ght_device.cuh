// ght_device.cuh -- device primitives of the GB300 hash tables: the hash
// family, integer remainder helpers, bucket loads and pair atomics.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ght {

constexpr uint32_t kPrime = 4294967291u;  // 2^32 - 5 (Sec. VII setup)
constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;
constexpr uint64_t kEmptyPair = 0xFFFFFFFFFFFFFFFFull;
constexpr unsigned kFull = 0xFFFFFFFFu;

enum Scheme : int { kBCHT = 0, kP2BHT = 1, kIHT = 2, kCuckoo1 = 3, kBCHT_LB = 4 };

// Status bits written by kernels into the control block.
enum : uint32_t {
  kStatusBuildFailed = 1u,  // chain bound hit or all candidate buckets full
  kStatusTimeout = 2u,      // a per-key step bound ran out
  kStatusSentinel = 4u,     // an input key was the sentinel
  kStatusCorrupt = 8u,      // an evicted key did not hash to its bucket
  kStatusDuplicate = 16u    // the duplicate check found a key stored twice
};

// Device control block, at the start of a table's storage (256 bytes).
struct Ctrl {
  uint32_t status;
  uint32_t pad0;
  unsigned long long insert_probes;
  unsigned long long insert_retries;
  unsigned long long insert_evictions;
  unsigned long long find_probes;
  unsigned long long find_queries;
  unsigned long long longest_chain;
  unsigned long long work_cursor;  // next input index claimed by a dynamic-chunk build
  unsigned long long reserved[24];
};
static_assert(sizeof(Ctrl) == 256, "control block is 256 bytes");

// Remainder by a runtime divisor d in [1, 2^32) without a divide, after
// Lemire, Kaser and Kurz, "Faster remainder by direct computation" (Software:
// Practice and Experience, 2019): with M = ceil(2^64 / d), x mod d is the
// high 64 bits of (M * x mod 2^64) * d, exact for every 32-bit x and d.
struct FastMod {
  uint64_t M;
  uint32_t d;
  uint32_t pad;
};

__host__ __device__ inline FastMod make_fastmod(uint32_t d) {
  FastMod f;
  f.M = 0xFFFFFFFFFFFFFFFFull / d + 1ull;  // wraps to 0 for d = 1, which yields 0
  f.d = d;
  f.pad = 0;
  return f;
}

__host__ __device__ __forceinline__ uint32_t fastmod(uint32_t x, const FastMod &f) {
  const uint64_t low = f.M * (uint64_t)x;
  const uint32_t lo = (uint32_t)low, hi = (uint32_t)(low >> 32);
  // high word of low * d, from 32-bit halves (no 128-bit type needed)
  const uint64_t t = (uint64_t)hi * f.d + (((uint64_t)lo * f.d) >> 32);
  return (uint32_t)(t >> 32);
}

// x mod p for any 64-bit x, from 2^32 = p + 5: fold the high word twice,
// then one conditional subtraction.
__host__ __device__ __forceinline__ uint32_t mod_prime(uint64_t x) {
  const uint64_t y = (x >> 32) * 5ull + (x & 0xFFFFFFFFull);  // < 6 * 2^32
  const uint64_t z = (y >> 32) * 5ull + (y & 0xFFFFFFFFull);  // <= 2^32 + 24
  return (uint32_t)(z >= kPrime ? z - kPrime : z);
}

struct HashFamily {
  uint32_t a[4];
  uint32_t c[4];
  FastMod mod;  // remainder by the number of buckets m
};

// Select x[i] for a runtime i without indexing: keeps kernel parameters out
// of local memory.
__host__ __device__ __forceinline__ uint32_t select4(const uint32_t (&x)[4], int i) {
  return i == 0 ? x[0] : (i == 1 ? x[1] : (i == 2 ? x[2] : x[3]));
}

// h_i(k) = ((a_i k + c_i) mod p) mod m  (Sec. VII setup)
__host__ __device__ __forceinline__ uint32_t bucket_of(const HashFamily &hf, int i, uint32_t k) {
  return fastmod(mod_prime((uint64_t)select4(hf.a, i) * k + select4(hf.c, i)), hf.mod);
}

// Everything a kernel needs to address a table; passed by value.
struct TableView {
  uint64_t *slots;     // m * b pairs, bucket-major
  Ctrl *ctrl;
  HashFamily hf;
  uint32_t m;
  int32_t h;           // number of hash functions
  int32_t t;           // IHT threshold
  uint32_t max_chain;  // cuckoo exchanges per insert
  uint32_t rng_seed;   // eviction xorshift seed
  uint32_t max_steps;  // per-key bound on build rounds (timeout)
  int32_t first;       // BCHT: hash index a new key starts at (1 for keys whose H_0 is known to be full)
};

__device__ __forceinline__ uint32_t pair_key(uint64_t p) { return (uint32_t)p; }
__device__ __forceinline__ uint32_t pair_value(uint64_t p) { return (uint32_t)(p >> 32); }

// Slot kinds of a bucketed table. PairSlot: 64-bit (value << 32) | key, a
// find returns the value or the sentinel. KeySlot: a 32-bit key only (a
// membership set), a find returns 1 (present) or 0 (absent).
struct PairSlot {
  using T = unsigned long long;
  static constexpr T kEmpty = 0xFFFFFFFFFFFFFFFFull;
  __device__ static uint32_t key(T s) { return (uint32_t)s; }
  __device__ static uint32_t found(T s) { return (uint32_t)(s >> 32); }
  __device__ static T make(uint32_t k, uint32_t v) { return ((T)v << 32) | k; }
  __device__ static uint32_t missing() { return kEmptyKey; }
};

struct KeySlot {
  using T = unsigned int;
  static constexpr T kEmpty = 0xFFFFFFFFu;
  __device__ static uint32_t key(T s) { return s; }
  __device__ static uint32_t found(T) { return 1u; }
  __device__ static T make(uint32_t k, uint32_t) { return k; }
  __device__ static uint32_t missing() { return 0u; }
};

// Marsaglia xorshift32 (13, 17, 5), "Xorshift RNGs" (2003), the eviction-slot
// generator of Sec. V-B.
__device__ __forceinline__ uint32_t xorshift32(uint32_t &s) {
  s ^= s << 13;
  s ^= s >> 17;
  s ^= s << 5;
  return s;
}

// Per-lane xorshift seed: a 32-bit integer mixer of (table seed, lane id),
// forced odd so the state is never zero.
__device__ __forceinline__ uint32_t lane_seed(uint32_t seed, uint64_t gid) {
  uint32_t x = seed ^ (uint32_t)gid ^ (uint32_t)(gid >> 32) * 0x9E3779B9u;
  x ^= x >> 16;
  x *= 0x7FEB352Du;
  x ^= x >> 15;
  x *= 0x846CA68Bu;
  x ^= x >> 16;
  return x | 1u;
}

// ---- bucket part loads --------------------------------------------------
// A tile of G lanes reads one bucket of B pairs; lane r reads pairs
// [r*PPL, (r+1)*PPL), PPL = B/G, with 16-byte vector loads where PPL >= 2.

// Find path: the table is immutable while finds run, so the read-only
// (non-coherent) data path is used.
template <int PPL>
__device__ __forceinline__ void load_part_ro(const uint64_t *bucket, int r, uint64_t (&v)[PPL]) {
  const uint64_t *p = bucket + r * PPL;
  if constexpr (PPL == 1) {
    v[0] = __ldg(reinterpret_cast<const unsigned long long *>(p));
  } else {
#pragma unroll
    for (int i = 0; i < PPL; i += 2) {
      const ulonglong2 x = __ldg(reinterpret_cast<const ulonglong2 *>(p + i));
      v[i] = x.x;
      v[i + 1] = x.y;
    }
  }
}

// Build path: other SMs update the table concurrently, so loads must not be
// served from a stale L1 line (a CAS retry would spin on it): relaxed,
// GPU-scope loads are performed at L2, where the atomics are.
template <int PPL>
__device__ __forceinline__ void load_part_rw(const uint64_t *bucket, int r, uint64_t (&v)[PPL]) {
  const uint64_t *p = bucket + r * PPL;
  if constexpr (PPL == 1) {
    unsigned long long x;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(x) : "l"(p) : "memory");
    v[0] = x;
  } else {
#pragma unroll
    for (int i = 0; i < PPL; i += 2) {
      unsigned long long x, y;
      asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];"
                   : "=l"(x), "=l"(y)
                   : "l"(p + i)
                   : "memory");
      v[i] = x;
      v[i + 1] = y;
    }
  }
}

// Generic part loads: lane r of a tile reads slots [r*PPL, (r+1)*PPL) of a
// bucket of slot type T, with 16-byte vector loads when the part allows.
template <int PPL, typename T>
__device__ __forceinline__ void load_slots_ro(const T *bucket, int r, T (&v)[PPL]) {
  if constexpr (sizeof(T) == 8) {
    load_part_ro<PPL>(reinterpret_cast<const uint64_t *>(bucket), r, reinterpret_cast<uint64_t(&)[PPL]>(v));
  } else {
    static_assert(PPL % 4 == 0, "32-bit slots are read 4 at a time");
    const uint4 *p = reinterpret_cast<const uint4 *>(bucket + r * PPL);
#pragma unroll
    for (int i = 0; i < PPL / 4; ++i) {
      const uint4 x = __ldg(p + i);
      v[4 * i] = x.x;
      v[4 * i + 1] = x.y;
      v[4 * i + 2] = x.z;
      v[4 * i + 3] = x.w;
    }
  }
}

template <int PPL, typename T>
__device__ __forceinline__ void load_slots_rw(const T *bucket, int r, T (&v)[PPL]) {
  if constexpr (sizeof(T) == 8) {
    load_part_rw<PPL>(reinterpret_cast<const uint64_t *>(bucket), r, reinterpret_cast<uint64_t(&)[PPL]>(v));
  } else {
    static_assert(PPL % 4 == 0, "32-bit slots are read 4 at a time");
    const T *p = bucket + r * PPL;
#pragma unroll
    for (int i = 0; i < PPL; i += 4) {
      unsigned a, b, c, d;
      asm volatile("ld.relaxed.gpu.global.v4.b32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
                   : "l"(p + i)
                   : "memory");
      v[i] = a;
      v[i + 1] = b;
      v[i + 2] = c;
      v[i + 3] = d;
    }
  }
}

// Keys only of slots [r*PPL, (r+1)*PPL) of a bucket, for inserts, which need
// to know which slots are empty and nothing else. For one 64-bit pair per
// lane this loads the key word alone: half the registers per load in flight,
// the same sectors.
template <int PPL, typename T>
__device__ __forceinline__ void load_keys_rw(const T *bucket, int r, uint32_t (&k)[PPL]) {
  if constexpr (sizeof(T) == 8 && PPL == 1) {
    const uint32_t *p = reinterpret_cast<const uint32_t *>(bucket + r);  // key = low word
    uint32_t x;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(x) : "l"(p) : "memory");
    k[0] = x;
  } else {
    T v[PPL];
    load_slots_rw<PPL>(bucket, r, v);
#pragma unroll
    for (int i = 0; i < PPL; ++i) k[i] = (uint32_t)v[i];
  }
}

template <typename T>
__device__ __forceinline__ T cas_slot(T *slot, T expect, T desired) {
  return atomicCAS(slot, expect, desired);
}

template <typename T>
__device__ __forceinline__ T exch_slot(T *slot, T desired) {
  return atomicExch(slot, desired);
}

__device__ __forceinline__ uint64_t cas_pair(uint64_t *slot, uint64_t expect, uint64_t desired) {
  return atomicCAS(reinterpret_cast<unsigned long long *>(slot), expect, desired);
}

__device__ __forceinline__ uint64_t exch_pair(uint64_t *slot, uint64_t desired) {
  return atomicExch(reinterpret_cast<unsigned long long *>(slot), desired);
}

__device__ __forceinline__ uint32_t load_status(const Ctrl *c) {
  uint32_t s;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(s) : "l"(&c->status) : "memory");
  return s;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

}  // namespace ght
