// kern_probe.cu -- memory-system ceilings for the access patterns of the
// table kernels, measured on the same GPU as the tables (a measurement aid;
// the paper has no counterpart). A bulk find reads random 128-byte buckets
// (Sec. V-A: one bucket = one cache line); a bulk insert reads a random
// bucket and then updates one 8-byte slot of it with an atomic (Sec. V-B).
// The probe does exactly that to a buffer of num_lines 128-byte lines, with
// no hashing logic, so its rate bounds what the table kernels can reach.
#include "ght_internal.h"

namespace ght {

// Line of operation i: a 64-bit mixer of (seed, i), reduced mod num_lines.
__device__ __forceinline__ uint32_t probe_line(uint32_t seed, uint64_t i, const FastMod &fm) {
  uint64_t x = (i + 1) * 0x9E3779B97F4A7C15ull ^ (uint64_t)seed;
  x ^= x >> 31;
  x *= 0xD6E8FEB86659FD93ull;
  x ^= x >> 32;
  return fastmod((uint32_t)x, fm);
}

// mode 0: read the line (read-only path).
// mode 1: read the line at L2, then one 64-bit CAS into its first slot whose
//         expected value is the word just read (fire and forget).
// mode 2: as 1, and the CAS results are consumed before the next reads are
//         issued (one atomic round trip per read, like an insert that waits).
// mode 3: one 64-bit atomic add into a random line, no read.
// mode 4: read the first half of the line (its first two 32-byte sectors).
// mode 5: read the first half of the line, then one more sector of the
//         second half chosen by the data (a dependent read).
// Four lanes cover a line, lane r reading the 8-byte word at byte 32 r (one
// word of each 32-byte sector, so DRAM delivers the whole line while the
// registers hold only what is needed to keep many lines in flight); a warp
// covers 8 lines per step and keeps kProbeUnroll steps (128 lines) in flight.
constexpr int kProbeUnroll = 16;

__global__ void __launch_bounds__(256)
line_probe_kernel(unsigned long long *__restrict__ lines, uint32_t num_lines, uint64_t ops, uint32_t seed, int mode,
                  unsigned long long *__restrict__ sink) {
  const int lane = threadIdx.x & 31;
  const int grp = lane >> 2;
  const int r = lane & 3;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const FastMod fm = make_fastmod(num_lines);
  unsigned long long acc = 0;
  for (uint64_t base = warp * (8 * kProbeUnroll); base < ops; base += warps * (8 * kProbeUnroll)) {
    uint32_t ln[kProbeUnroll];
    unsigned long long x[kProbeUnroll];
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u) {
      const uint64_t i = base + 8 * u + grp;
      ln[u] = i < ops ? probe_line(seed, i, fm) : 0xFFFFFFFFu;
      x[u] = 0;
    }
    if (mode <= 2 || mode >= 4) {
#pragma unroll
      for (int u = 0; u < kProbeUnroll; ++u) {
        if (ln[u] == 0xFFFFFFFFu || (mode >= 4 && r >= 2)) continue;
        const unsigned long long *p = lines + (uint64_t)ln[u] * 16 + 4 * r;
        if (mode == 0) {
          x[u] = __ldg(p);
        } else {
          asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(x[u]) : "l"(p) : "memory");
        }
      }
    }
    if (mode == 5) {
      // the dependent sector: lane 0 of each line reads a word of sector 2 or 3
#pragma unroll
      for (int u = 0; u < kProbeUnroll; ++u) {
        if (ln[u] == 0xFFFFFFFFu || r != 0) continue;
        x[u] += __ldg(lines + (uint64_t)ln[u] * 16 + 8 + 4 * (x[u] & 1ull));
      }
    }
    if (mode >= 1 && mode <= 3) {
      unsigned long long s = 0;
#pragma unroll
      for (int u = 0; u < kProbeUnroll; ++u) {
        if (ln[u] == 0xFFFFFFFFu || r != 0) continue;
        unsigned long long *slot = lines + (uint64_t)ln[u] * 16;
        if (mode == 3) {
          atomicAdd(slot, 1ull);
        } else {
          const unsigned long long old = atomicCAS(slot, x[u], x[u] + 1ull);
          if (mode == 2) s += old;
        }
      }
      if (mode == 2) acc += __shfl_sync(kFull, s, 0);  // every CAS result before the next step's reads
    }
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u) acc += x[u];
  }
  if (acc == 0x5EEDF00DCAFEull) sink[0] = acc;  // keeps the loads; practically never taken
}

cudaError_t launch_line_probe(int mode, void *lines, uint64_t num_lines, uint64_t ops, uint32_t seed,
                              cudaStream_t s) {
  int blocks = 0;
  cudaError_t e = grid_for(line_probe_kernel, ops * 4 + kThreads, 0, &blocks);
  if (e != cudaSuccess) return e;
  line_probe_kernel<<<blocks, kThreads, 0, s>>>(static_cast<unsigned long long *>(lines), (uint32_t)num_lines, ops,
                                                seed, mode, static_cast<unsigned long long *>(lines));
  return cudaGetLastError();
}

}  // namespace ght
