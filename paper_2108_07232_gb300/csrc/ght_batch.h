// ght_batch.h -- device-side view of a batch of BCHT tables (kern_batch.cu).
#pragma once

#include "ght.h"
#include "ght_internal.h"

namespace ght {

// Descriptor of one table of a batch (64 bytes, device memory).
struct BatchTable {
  uint64_t *slots;  // m * 16 pairs
  FastMod mod;      // remainder by m
  uint32_t a[4], c[4];
  uint32_t status;  // build status bits of this table
  uint32_t m;
};
static_assert(sizeof(BatchTable) == 64, "batch descriptor is 64 bytes");

struct BatchView {
  BatchTable *tables;
  const uint64_t *key_offs;    // num_tables + 1 prefix offsets into the key/value arrays
  const uint64_t *query_offs;  // num_tables + 1 prefix offsets into the query/result arrays
  Ctrl *ctrl;                  // batch-wide probe counters
  uint32_t t_lo, t_hi;         // tables this launch covers
  int32_t h;
  uint32_t max_chain, max_steps, rng_seed;
};

bool batch_shape_supported(int tile_lanes, int keys_per_lane);
// Find shapes: the above, and 4-lane tiles with 6 query sets per lane (the
// staged find: bucket parts in shared memory).
bool batch_find_shape_supported(int tile_lanes, int keys_per_lane);

// Describe a built single BCHT table (b = 16) as a batch descriptor (ght_api.cu).
// Returns false if the table is not a built 16-pair BCHT table.
bool table_descriptor(const struct ::ght_table *t, BatchTable *out);

// Copy n items from per-segment sources into one array and back
// (kern_batch.cu): dst[i] = src[s][i - offs[s]] for offs[s] <= i < offs[s+1].
cudaError_t launch_segment_gather(const uint32_t *const *src, const uint64_t *offs, uint32_t segs, uint32_t *dst,
                                  uint64_t n, cudaStream_t s);
cudaError_t launch_segment_scatter(const uint32_t *src, uint32_t *const *dst, const uint64_t *offs, uint32_t segs,
                                   uint64_t n, cudaStream_t s);
cudaError_t launch_batch_fill(const BatchView &bv, uint64_t *slots, uint64_t num_slots, cudaStream_t s);
cudaError_t launch_batch_insert(const BatchView &bv, const uint32_t *k, const uint32_t *v, uint64_t items,
                                const LaunchOpts &o, cudaStream_t s);
cudaError_t launch_batch_find(const BatchView &bv, const uint32_t *q, uint32_t *out, uint64_t items,
                              const LaunchOpts &o, cudaStream_t s);

}  // namespace ght
