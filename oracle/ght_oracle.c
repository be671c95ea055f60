/*
 * ght_oracle.c -- plain, slow, single-threaded CPU oracle (test infrastructure
 * only; see ght_oracle.h). Every function follows the paper's definitions in
 * the paper's order, with no blocking, fusion or reordering. Citations are to
 * sections, listings and tables of arXiv 2108.07232.
 */
#include "ght_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static uint32_t key_of(uint64_t pair) { return (uint32_t)(pair & 0xFFFFFFFFull); }
static uint32_t value_of(uint64_t pair) { return (uint32_t)(pair >> 32); }
static uint64_t make_pair(uint32_t k, uint32_t v) { return ((uint64_t)v << 32) | k; }

/* Section VII setup: h(k; a, b) = ((a k + b) mod p) mod L with p = 4294967291.
 * a, c < 2^32 and k < 2^32, so a*k + c < 2^64: plain unsigned 64-bit
 * arithmetic is exact. */
uint32_t orc_hash(uint32_t a, uint32_t c, uint64_t m, uint32_t k) {
  uint64_t x = (uint64_t)a * (uint64_t)k + (uint64_t)c;
  return (uint32_t)((x % (uint64_t)ORC_PRIME) % m);
}

uint32_t orc_bucket(const orc_params *P, int i, uint32_t k) {
  if (P->explicit_buckets && (uint64_t)k < P->explicit_n)
    return P->explicit_buckets[(uint64_t)k * (uint64_t)P->h + (uint64_t)i];
  return orc_hash(P->a[i], P->c[i], P->m, k);
}

/* SplitMix64, Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators" (OOPSLA 2014): golden-gamma increment, then the variant-13
 * finaliser. Used only to turn a seed into the "randomly generated" a and b
 * of Section VII. */
uint64_t orc_splitmix64(uint64_t *state) {
  uint64_t z;
  *state += 0x9E3779B97F4A7C15ull;
  z = *state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void orc_derive_constants(uint64_t seed, uint32_t attempt, int h, uint32_t *a,
                          uint32_t *c) {
  uint64_t state = seed ^ ((uint64_t)attempt * 0x9E3779B97F4A7C15ull);
  int i;
  for (i = 0; i < h; i++) {
    uint64_t x = orc_splitmix64(&state);
    uint64_t y = orc_splitmix64(&state);
    a[i] = (uint32_t)(1u + x % (uint64_t)(ORC_PRIME - 1u));
    c[i] = (uint32_t)(y % (uint64_t)ORC_PRIME);
  }
}

/* Section III: capacity C = m * b and load factor n / C, so a table sized
 * for `capacity` keys at load factor lf has m = ceil(capacity / (lf * b)). */
uint64_t orc_num_buckets(uint64_t capacity, double lf, int b) {
  double want;
  if (!(lf > 0.0) || !(lf <= 1.0) || b < 1) return 0;
  want = ceil((double)capacity / (lf * (double)b));
  if (want < 1.0) want = 1.0;
  if (want > 4294967295.0) return 0;
  return (uint64_t)want;
}

int orc_default_params(int scheme, uint64_t capacity, double lf, uint64_t seed,
                       uint32_t attempt, orc_params *out) {
  uint64_t st;
  memset(out, 0, sizeof(*out));
  out->scheme = scheme;
  switch (scheme) {
  case ORC_BCHT:    /* b = 16, three hash functions (Sec. VII recommendations) */
    out->b = 16; out->h = 3; out->max_chain = 1000; break;
  case ORC_P2BHT:   /* two choices */
    out->b = 16; out->h = 2; break;
  case ORC_IHT:     /* primary + two secondaries (Sec. III-C); t = ceil(0.8 b) */
    out->b = 16; out->h = 3; out->t = 13; break;
  case ORC_CUCKOO1: /* bucket size one, three hash functions */
    out->b = 1; out->h = 3; out->max_chain = 1000; break;
  case ORC_BCHT_LB:
    out->b = 16; out->h = 3; out->max_chain = 1000; break;
  default:
    return -1;
  }
  out->m = orc_num_buckets(capacity, lf, out->b);
  if (out->m == 0) return -1;
  orc_derive_constants(seed, attempt, out->h, out->a, out->c);
  st = seed ^ 0x6F7261636C65ull ^ ((uint64_t)attempt << 32);
  out->rng_seed = (uint32_t)orc_splitmix64(&st) | 1u;
  return 0;
}

int orc_bucket_load(const orc_params *P, const uint64_t *slots, uint64_t bucket) {
  int s, load = 0;
  for (s = 0; s < P->b; s++)
    if (key_of(slots[bucket * (uint64_t)P->b + (uint64_t)s]) != ORC_EMPTY_KEY) load++;
  return load;
}

static int first_empty_slot(const orc_params *P, const uint64_t *slots, uint64_t bucket) {
  int s;
  for (s = 0; s < P->b; s++)
    if (key_of(slots[bucket * (uint64_t)P->b + (uint64_t)s]) == ORC_EMPTY_KEY) return s;
  return -1;
}

/* Marsaglia, "Xorshift RNGs", J. Stat. Softw. 8(14), 2003: the (13, 17, 5)
 * 32-bit generator. Section V-B draws the eviction slot from it. */
uint32_t orc_xorshift32(uint32_t *state) {
  uint32_t x = *state;
  x ^= x << 13;
  x ^= x >> 17;
  x ^= x << 5;
  *state = x;
  return x;
}

/* Bucketed cuckoo insert (Section III-A, Section V-B): start at H_0(k); if the
 * bucket has an empty slot, store there; if it is full, exchange with a random
 * slot and continue with the evicted pair at H_{(i+1) mod h}, where i is the
 * lowest index with H_i(evicted) equal to the current bucket (Section III-A
 * footnote). Fail once max_chain exchanges have been made. Also serves 1CHT
 * (b = 1: the only slot is always the one exchanged). */
static int insert_cuckoo(const orc_params *P, uint64_t *slots, uint64_t pair,
                         uint32_t *rng, orc_build_stats *st) {
  uint32_t bucket = orc_bucket(P, 0, key_of(pair));
  uint32_t chain = 0;
  for (;;) {
    int s;
    st->probes++;
    s = first_empty_slot(P, slots, bucket);
    if (s >= 0) {
      slots[(uint64_t)bucket * (uint64_t)P->b + (uint64_t)s] = pair;
      if (chain > st->longest_chain) st->longest_chain = chain;
      return 1;
    }
    if (chain == P->max_chain) {
      if (chain > st->longest_chain) st->longest_chain = chain;
      return 0;
    }
    {
      uint32_t r = (P->b == 1) ? 0u : orc_xorshift32(rng) % (uint32_t)P->b;
      uint64_t *slot = &slots[(uint64_t)bucket * (uint64_t)P->b + r];
      uint64_t evicted = *slot;
      int i = 0;
      *slot = pair;
      pair = evicted;
      chain++;
      st->evictions++;
      while (i < P->h && orc_bucket(P, i, key_of(pair)) != bucket) i++;
      if (i == P->h) return -2; /* the evicted key did not hash here: corrupt table */
      bucket = orc_bucket(P, (i + 1) % P->h, key_of(pair));
    }
  }
}

/* Bucketed power-of-two-choices insert (Section III-B, Section V-C): read
 * both candidate buckets, fail if both are full, else store in the less
 * loaded one, ties to H_0. */
static int insert_p2(const orc_params *P, uint64_t *slots, uint64_t pair,
                     orc_build_stats *st) {
  uint32_t b0 = orc_bucket(P, 0, key_of(pair));
  uint32_t b1 = orc_bucket(P, 1, key_of(pair));
  int l0 = orc_bucket_load(P, slots, b0);
  int l1 = orc_bucket_load(P, slots, b1);
  uint32_t target;
  st->probes += 2;
  if (l0 == P->b && l1 == P->b) return 0;
  target = (l0 <= l1) ? b0 : b1;
  slots[(uint64_t)target * (uint64_t)P->b + (uint64_t)first_empty_slot(P, slots, target)] = pair;
  return 1;
}

/* Iceberg insert (Section III-C insertion steps; Section V-D): the primary
 * bucket H_p = H_0 takes the key while it would still hold fewer than t keys
 * afterwards (t = 13 for b = 16, the threshold the paper states for its
 * sector measurements; this reading reproduces the paper's probe counts of
 * Section VII-A3 for t at 20, 40, 60 and 80 % of b); otherwise the less full
 * of the secondaries H_s0 = H_1, H_s1 = H_2 (ties to H_s0); if both
 * secondaries are full, the primary if it still has room; else the build
 * fails. */
static int insert_iceberg(const orc_params *P, uint64_t *slots, uint64_t pair,
                          orc_build_stats *st) {
  uint32_t bp = orc_bucket(P, 0, key_of(pair));
  int lp = orc_bucket_load(P, slots, bp);
  uint32_t target;
  st->probes += 1;
  if (lp + 1 < P->t) {
    target = bp;
  } else {
    uint32_t b0 = orc_bucket(P, 1, key_of(pair));
    uint32_t b1 = orc_bucket(P, 2, key_of(pair));
    int l0 = orc_bucket_load(P, slots, b0);
    int l1 = orc_bucket_load(P, slots, b1);
    st->probes += 2;
    if (l0 < P->b || l1 < P->b)
      target = (l0 <= l1) ? b0 : b1;
    else if (lp < P->b)
      target = bp;
    else
      return 0;
  }
  slots[(uint64_t)target * (uint64_t)P->b + (uint64_t)first_empty_slot(P, slots, target)] = pair;
  return 1;
}

/* Load-balanced bucketed cuckoo insert (Section III-A, last paragraph): read
 * all h candidate buckets and store in the least loaded one (ties to the
 * lowest index). When all are full, exchange with a random slot of the
 * current bucket -- starting from H_0 -- and continue with the evicted pair,
 * whose own candidates exclude the bucket it was evicted from. */
static int insert_lb(const orc_params *P, uint64_t *slots, uint64_t pair,
                     uint32_t *rng, orc_build_stats *st) {
  uint32_t chain = 0;
  int64_t from = -1; /* bucket the current pair was evicted from */
  for (;;) {
    int i, best = -1, best_load = P->b + 1;
    uint32_t cand[4];
    for (i = 0; i < P->h; i++) {
      int l;
      cand[i] = orc_bucket(P, i, key_of(pair));
      l = orc_bucket_load(P, slots, cand[i]);
      st->probes++;
      if ((int64_t)cand[i] == from) continue;
      if (l < best_load) { best_load = l; best = i; }
    }
    if (best >= 0 && best_load < P->b) {
      uint32_t t = cand[best];
      slots[(uint64_t)t * (uint64_t)P->b + (uint64_t)first_empty_slot(P, slots, t)] = pair;
      if (chain > st->longest_chain) st->longest_chain = chain;
      return 1;
    }
    if (chain == P->max_chain || best < 0) {
      if (chain > st->longest_chain) st->longest_chain = chain;
      return 0;
    }
    {
      uint32_t r = orc_xorshift32(rng) % (uint32_t)P->b;
      uint32_t victim_bucket = cand[best];
      uint64_t *slot = &slots[(uint64_t)victim_bucket * (uint64_t)P->b + r];
      uint64_t evicted = *slot;
      *slot = pair;
      pair = evicted;
      from = victim_bucket;
      chain++;
      st->evictions++;
    }
  }
}

int orc_insert(const orc_params *P, uint64_t *slots, uint32_t key, uint32_t value,
               uint32_t *rng_state, orc_build_stats *st) {
  uint64_t pair = make_pair(key, value);
  int ok;
  if (key == ORC_EMPTY_KEY) return -1;
  switch (P->scheme) {
  case ORC_BCHT:
  case ORC_CUCKOO1: ok = insert_cuckoo(P, slots, pair, rng_state, st); break;
  case ORC_P2BHT: ok = insert_p2(P, slots, pair, st); break;
  case ORC_IHT: ok = insert_iceberg(P, slots, pair, st); break;
  case ORC_BCHT_LB: ok = insert_lb(P, slots, pair, rng_state, st); break;
  default: return -1;
  }
  return ok < 0 ? -1 : ok;
}

int orc_build(const orc_params *P, uint64_t *slots, const uint32_t *keys,
              const uint32_t *values, uint64_t n, orc_build_stats *st) {
  uint64_t i, total = P->m * (uint64_t)P->b;
  uint32_t rng = P->rng_seed ? P->rng_seed : 1u;
  orc_build_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  st->failed_at = -1;
  /* Section III-A: initialise all buckets to empty. */
  for (i = 0; i < total; i++) slots[i] = ORC_EMPTY_PAIR;
  for (i = 0; i < n; i++) {
    int ok = orc_insert(P, slots, keys[i], values[i], &rng, st);
    if (ok != 1) { st->failed_at = (int64_t)i; return ok; }
    st->inserted++;
  }
  return 1;
}

/* Find (Section V-B find; Section V-C and V-D find paragraphs). Probe the
 * candidate buckets in hash order and stop when the key is found. BCHT and
 * 1CHT also stop at the first probed bucket that has an empty slot (valid
 * because keys are placed in H_0 first and buckets never lose keys); P2BHT,
 * IHT and the load-balanced BCHT cannot exit early. The sentinel is never a
 * key: querying it returns the sentinel without a probe. */
uint64_t orc_find(const orc_params *P, const uint64_t *slots,
                  const uint32_t *queries, uint32_t *out, uint64_t nq,
                  uint8_t *probes_each) {
  uint64_t j, total = 0;
  int early_exit = (P->scheme == ORC_BCHT || P->scheme == ORC_CUCKOO1);
  for (j = 0; j < nq; j++) {
    uint32_t q = queries[j];
    uint32_t result = ORC_EMPTY_KEY;
    int i, probes = 0;
    if (q != ORC_EMPTY_KEY) {
      for (i = 0; i < P->h; i++) {
        uint64_t bucket = orc_bucket(P, i, q);
        int s, found = 0, has_empty = 0;
        probes++;
        for (s = 0; s < P->b; s++) {
          uint64_t pair = slots[bucket * (uint64_t)P->b + (uint64_t)s];
          if (key_of(pair) == q) { result = value_of(pair); found = 1; break; }
          if (key_of(pair) == ORC_EMPTY_KEY) has_empty = 1;
        }
        if (found) break;
        if (early_exit && has_empty) break;
      }
    }
    out[j] = result;
    if (probes_each) probes_each[j] = (uint8_t)probes;
    total += (uint64_t)probes;
  }
  return total;
}

typedef struct { uint32_t key; uint64_t pos; } qpos;

static int cmp_qpos(const void *x, const void *y) {
  const qpos *a = (const qpos *)x, *b = (const qpos *)y;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->pos < b->pos ? -1 : (a->pos > b->pos);
}

/* The result every correct table must return (Section I: a lookup returns
 * the value associated with the key; Section V: the sentinel otherwise).
 * Plain sort of the queries plus one binary search per input pair. */
int orc_lookup(const uint32_t *keys, const uint32_t *values, uint64_t n,
               const uint32_t *queries, uint32_t *out, uint64_t nq) {
  uint64_t i;
  qpos *sq;
  for (i = 0; i < nq; i++) out[i] = ORC_EMPTY_KEY;
  if (nq == 0) return 0;
  sq = (qpos *)malloc(nq * sizeof(qpos));
  if (!sq) return -1;
  for (i = 0; i < nq; i++) { sq[i].key = queries[i]; sq[i].pos = i; }
  qsort(sq, nq, sizeof(qpos), cmp_qpos);
  for (i = 0; i < n; i++) {
    uint64_t lo = 0, hi = nq;
    if (keys[i] == ORC_EMPTY_KEY) { free(sq); return -1; }
    while (lo < hi) { /* first position with key >= keys[i] */
      uint64_t mid = lo + (hi - lo) / 2;
      if (sq[mid].key < keys[i]) lo = mid + 1; else hi = mid;
    }
    while (lo < nq && sq[lo].key == keys[i]) { out[sq[lo].pos] = values[i]; lo++; }
  }
  free(sq);
  return 0;
}

static int cmp_u64(const void *x, const void *y) {
  uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
  return a < b ? -1 : (a > b);
}

/* pair stored with the key in the high word so that sorting orders by key */
static uint64_t key_major(uint64_t pair) { return ((uint64_t)key_of(pair) << 32) | value_of(pair); }

int orc_validate(const orc_params *P, const uint64_t *slots,
                 const uint32_t *keys, const uint32_t *values, uint64_t n,
                 char *msg, int msg_len) {
  uint64_t total = P->m * (uint64_t)P->b, bkt, cnt = 0, i;
  uint64_t *stored = NULL, *input = NULL;
  int ok = 0;
  if (msg && msg_len > 0) msg[0] = 0;
#define FAIL(...) do { if (msg) snprintf(msg, (size_t)msg_len, __VA_ARGS__); goto done; } while (0)
  stored = (uint64_t *)malloc((total ? total : 1) * sizeof(uint64_t));
  if (!stored) FAIL("out of memory");
  for (bkt = 0; bkt < P->m; bkt++) {
    int s;
    for (s = 0; s < P->b; s++) {
      uint64_t pair = slots[bkt * (uint64_t)P->b + (uint64_t)s];
      uint32_t k = key_of(pair);
      int i2, j = -1;
      if (k == ORC_EMPTY_KEY) {
        if (pair != ORC_EMPTY_PAIR) FAIL("half-empty pair at bucket %llu slot %d", (unsigned long long)bkt, s);
        continue;
      }
      for (i2 = 0; i2 < P->h; i2++)
        if (orc_bucket(P, i2, k) == bkt) { j = i2; break; }
      if (j < 0) FAIL("key %u at bucket %llu is in none of its candidate buckets", k, (unsigned long long)bkt);
      if (P->scheme == ORC_BCHT || P->scheme == ORC_CUCKOO1) {
        /* early-exit invariant: every H_0 .. H_{j-1} of the key is full */
        for (i2 = 0; i2 < j; i2++)
          if (orc_bucket_load(P, slots, orc_bucket(P, i2, k)) != P->b)
            FAIL("key %u stored at H_%d but H_%d is not full", k, j, i2);
      }
      if (P->scheme == ORC_IHT && j != 0) {
        if (orc_bucket_load(P, slots, orc_bucket(P, 0, k)) + 1 < P->t)
          FAIL("key %u stored in a secondary bucket while its primary holds fewer than t-1 keys", k);
      }
      stored[cnt++] = key_major(pair);
    }
  }
  if (cnt != n) FAIL("table holds %llu keys, expected %llu", (unsigned long long)cnt, (unsigned long long)n);
  qsort(stored, cnt, sizeof(uint64_t), cmp_u64);
  for (i = 1; i < cnt; i++)
    if ((stored[i] >> 32) == (stored[i - 1] >> 32)) FAIL("key %u stored twice", (uint32_t)(stored[i] >> 32));
  if (keys && values) {
    input = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!input) FAIL("out of memory");
    for (i = 0; i < n; i++) input[i] = ((uint64_t)keys[i] << 32) | values[i];
    qsort(input, n, sizeof(uint64_t), cmp_u64);
    for (i = 0; i < n; i++)
      if (input[i] != stored[i]) FAIL("stored pairs differ from the input near key %u", (uint32_t)(input[i] >> 32));
  }
  ok = 1;
#undef FAIL
done:
  free(stored);
  free(input);
  return ok;
}
