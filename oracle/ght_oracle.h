/*
 * ght_oracle.h -- plain, slow, single-threaded CPU oracle for the static
 * bucketed hash tables of Awad, Ashkiani, Porumbescu, Farach-Colton, Owens,
 * "Better GPU Hash Tables" (arXiv 2108.07232).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links, loads or calls
 * this code: only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do. It shares no code, header, table or constant generator with the CUDA
 * library; the two meet only through the seeded arrays of the input module.
 *
 * Conventions (paper Section V opening paragraph and Section III):
 *   - 32-bit keys and values; a slot is a 64-bit pair (value << 32) | key.
 *   - the empty key and the empty value are both 0xFFFFFFFF, so an empty
 *     slot is the all-ones pair.
 *   - a table is m buckets of b slots, capacity C = m*b, load factor n/C.
 *   - hash family h_i(k) = ((a_i*k + c_i) mod p) mod m, p = 4294967291
 *     (Section VII, experimental setup). The paper calls the additive constant
 *     "b"; here it is c_i so it cannot be confused with the bucket size.
 */
#ifndef GHT_ORACLE_H
#define GHT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_PRIME 4294967291u
#define ORC_EMPTY_KEY 0xFFFFFFFFu
#define ORC_EMPTY_PAIR 0xFFFFFFFFFFFFFFFFull

/* Schemes (Section III; 1CHT is BCHT with b = 1, Section VII variant list). */
enum {
  ORC_BCHT = 0,    /* bucketed cuckoo, first-bucket placement, early-exit find */
  ORC_P2BHT = 1,   /* bucketed power-of-two-choices, least loaded of H0/H1 */
  ORC_IHT = 2,     /* iceberg: primary below threshold t, else two choices */
  ORC_CUCKOO1 = 3, /* bucket size one cuckoo (CUDPP-style 1CHT) */
  ORC_BCHT_LB = 4  /* load-balanced BCHT: least loaded of the h buckets (Sec. III-A, last paragraph) */
};

typedef struct {
  int32_t scheme;
  int32_t b;           /* slots per bucket */
  int32_t h;           /* number of hash functions, 1..4 */
  int32_t t;           /* IHT threshold t: the primary takes a key while it would
                        * hold fewer than t keys afterwards */
  uint64_t m;          /* number of buckets, 1 .. 2^32-1 */
  uint32_t a[4];       /* multiplicative constants, 1 <= a_i < p */
  uint32_t c[4];       /* additive constants, 0 <= c_i < p */
  uint32_t max_chain;  /* cuckoo eviction bound (exchanges per insert) */
  uint32_t rng_seed;   /* xorshift seed for the eviction slot */
  /* Optional explicit hash values for hand-made examples: when non-NULL,
   * H_i(k) = explicit_buckets[k*h + i] for k < explicit_n. */
  const uint32_t *explicit_buckets;
  uint64_t explicit_n;
} orc_params;

typedef struct {
  uint64_t probes;        /* bucket reads (sequential count, Sec. VII-D) */
  uint64_t evictions;     /* cuckoo exchanges */
  uint64_t longest_chain; /* most exchanges one insert needed */
  uint64_t inserted;      /* keys fully placed */
  int64_t failed_at;      /* index of the key whose insert failed, or -1 */
} orc_build_stats;

/* ((a*k + c) mod p) mod m, the textbook definition in 64-bit arithmetic. */
uint32_t orc_hash(uint32_t a, uint32_t c, uint64_t m, uint32_t k);

/* Bucket of key k under hash function i of the table. */
uint32_t orc_bucket(const orc_params *P, int i, uint32_t k);

/* SplitMix64 (Steele, Lea, Flood 2014): advance *state, return the output. */
uint64_t orc_splitmix64(uint64_t *state);

/* Hash constants for (seed, attempt): generator state starts at
 * seed XOR (attempt * 0x9E3779B97F4A7C15); draws in order a_0, c_0, a_1, ...;
 * a_i = 1 + x mod (p-1), c_i = x mod p. */
void orc_derive_constants(uint64_t seed, uint32_t attempt, int h,
                          uint32_t *a, uint32_t *c);

/* m = ceil(capacity / (lf * b)) in IEEE double, at least 1; 0 if invalid. */
uint64_t orc_num_buckets(uint64_t capacity, double lf, int b);

/* Default parameters of a scheme (b, h, t, max_chain) plus sizing and
 * constants. Returns 0 on success, -1 on invalid arguments. */
int orc_default_params(int scheme, uint64_t capacity, double lf, uint64_t seed,
                       uint32_t attempt, orc_params *out);

/* Number of non-empty slots in bucket `bucket`. */
int orc_bucket_load(const orc_params *P, const uint64_t *slots, uint64_t bucket);

/* Sequential build in input order into slots[m*b] (filled to empty first).
 * Returns 1 on success, 0 on failure (chain bound hit, or no candidate
 * bucket has room), -1 on a precondition violation (sentinel key). */
int orc_build(const orc_params *P, uint64_t *slots, const uint32_t *keys,
              const uint32_t *values, uint64_t n, orc_build_stats *st);

/* Insert one pair into an existing table (used for hand-made examples).
 * rng_state is the eviction xorshift state. Same return codes as orc_build. */
int orc_insert(const orc_params *P, uint64_t *slots, uint32_t key, uint32_t value,
               uint32_t *rng_state, orc_build_stats *st);

/* Scheme find over a built table; out[i] = value or 0xFFFFFFFF. If
 * probes_each is non-NULL it receives the bucket reads of each query.
 * Returns the total number of bucket reads. */
uint64_t orc_find(const orc_params *P, const uint64_t *slots,
                  const uint32_t *queries, uint32_t *out, uint64_t nq,
                  uint8_t *probes_each);

/* Definitional lookup, independent of any table: out[j] = v if (q_j, v) is
 * an input pair, else 0xFFFFFFFF. Keys must be unique. */
int orc_lookup(const uint32_t *keys, const uint32_t *values, uint64_t n,
               const uint32_t *queries, uint32_t *out, uint64_t nq);

/* Layout validator. Returns 1 if every invariant holds, else 0 with a
 * message in msg. Checks: no half-empty pair; the sentinel is never a key;
 * each stored key lies in one of its candidate buckets; no key twice; the
 * non-empty count equals n; stored pairs equal the input pairs; plus the
 * scheme-specific placement invariants. keys/values may be NULL to skip the
 * input comparison (then n is only the expected count). */
int orc_validate(const orc_params *P, const uint64_t *slots,
                 const uint32_t *keys, const uint32_t *values, uint64_t n,
                 char *msg, int msg_len);

/* Marsaglia xorshift32 (13, 17, 5); state must be non-zero. */
uint32_t orc_xorshift32(uint32_t *state);

#ifdef __cplusplus
}
#endif
#endif
