// Shared device-side definitions for the gbfs library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace gbfs {

// Device error bits, OR-ed into Ctl::error by kernels and read by the host after a search.
enum : unsigned { kErrColumnRange = 1u, kErrFrontierRange = 2u, kErrCounterOverflow = 4u, kErrTimeout = 8u };

// The next frontier's size and edge total are reserved together by one 64-bit atomicAdd
// on a packed word (count << shift) | edges, so the slot order and the exclusive degree
// scan agree (the scan of Sec. 3.4, fused into Algorithm 3's frontier append).
struct Packed {
  int shift;                 // bits for the edge total
  unsigned long long mask;   // (1 << shift) - 1
  __host__ __device__ long long count(unsigned long long p) const { return (long long)(p >> shift); }
  __host__ __device__ long long edges(unsigned long long p) const { return (long long)(p & mask); }
  __host__ __device__ unsigned long long make(long long c, long long e) const {
    return ((unsigned long long)c << shift) | (unsigned long long)e;
  }
};

// Frontier in the form the expansion consumes: vertex ids, the exclusive scan of their
// degrees (cum[k] = sum of deg(v[j]) for j < k) and base[k] = off[v[k]] - cum[k], so edge
// e of the level's edge space (cum[k] <= e < cum[k + 1]) is column entry base[k] + e.
// The expansion needs v[k] only as the parent it writes, so on a degree-relabelled graph
// v holds caller ids while base is computed from the internal id.
template <typename OffT>
struct FrontierBuf {
  int32_t* v;
  OffT* cum;
  OffT* base;
};

// Tile descriptor of the chunk index: for every kChunk-th edge c * kChunk of a level's
// edge space, k = max{k : cum[k] <= c * kChunk} (the answer of Algorithm 3's binary
// search), plus what a tile that lies inside row k alone needs: the parent to write (the
// caller id u of entry k) and col = base[k] + c * kChunk, the column entry of that edge.
// Written by whoever appends entry k to the frontier.
template <typename OffT>
struct alignas(16) TileDesc {
  int32_t k;
  int32_t u;
  OffT col;
};

// Per-search control block in device memory. Two counters alternate by level parity:
// counter[cur] describes the frontier being expanded, counter[nxt] collects the next one.
struct Ctl {
  unsigned long long counter[2];
  unsigned int done[2];      // CTAs finished per parity (last-CTA detection, no spinning)
  int level;                 // level assigned to vertices claimed by the running expansion
  int depth;                 // non-empty frontiers so far (root included)
  long long reached;         // vertices reached so far (root included)
  long long edges2;          // sum of frontier degree sums = 2 m_c at the end
  unsigned int error;        // kErr* bits
  int cont;                  // 1 while the next frontier is non-empty
  int32_t* levels;           // output arrays of the running search
  int32_t* parents;
  unsigned int dropped;      // frontier-bitmap mode: the level stopped appending to the list
  int pad;
  unsigned long long bm_counter;  // packed (count, edges) of the list unpacked from the bitmap
};

// Control block of a persistent (one-launch) search: counters rotate by 3 so that level
// it reads counter[it % 3], fills counter[(it + 1) % 3] and clears counter[(it + 2) % 3].
constexpr int kMaxLevelTimes = 64;
struct PCtl {
  unsigned long long counter[3];
  unsigned int pfx[3];             // by level % 3: first bitmap word not full (visited prefix scan)
  unsigned int pad_pfx;
  unsigned int bar_count;
  unsigned int bar_gen;
  unsigned int error;
  int depth;
  long long reached;
  long long edges2;
  int steps_bottom_up;
  int unpacked_levels;                          // levels whose next frontier was unpacked from a bitmap
  unsigned long long bm_counter[3];             // by level % 3: reservations of the bitmap unpack
  unsigned int dropped[3];                      // by level % 3: the level stopped appending to the list
  int pad;
  unsigned long long start_ns;                  // device clock when the search was set up
  unsigned long long level_ns[kMaxLevelTimes];  // device clock at the end of each level
  long long level_nf[kMaxLevelTimes];           // frontier size of each level
  int level_bu[kMaxLevelTimes];                 // 1 if the level ran bottom-up
};

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Read-only, non-coherent load of a column id (the const __restrict__ read-only path the
// paper uses for the CSC arrays, Sec. 3.4.1). Column ids stream: each is read once per
// level, so they are not allocated in L1, which is left to the bitmap probes.
// (Measured on R-MAT s24: +3 % top-down.) A lane that reads several consecutive ids itself,
// as the bottom-up row scan does, uses __ldg instead so that they share one L1 fill.
__device__ __forceinline__ int32_t ld_nc(const int32_t* p) {
  int32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// Visited-bitmap pre-check load (Algorithm 3's non-atomic pre-check). Mode 0: through L1, kept there with
// priority (a stale copy is harmless: the atomicOr decides). Mode 1: L2 only
// (ld.global.cg), so words filled during the level are seen and fewer futile atomics are
// issued.
__device__ __forceinline__ uint32_t probe_load(const uint32_t* p, int mode) {
  if (mode) return __ldcg(p);
  uint32_t v;
  asm volatile("ld.global.L1::evict_last.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, d);
    if ((int)lane_id() >= d) x += y;
  }
  return x;
}

// Largest k in [lo, hi) with a[k] <= x, given a[lo] <= x (binsearch_maxle, the binary search of
// Algorithm 3). a is non-decreasing.
template <typename T, typename I>
__device__ __forceinline__ I binsearch_maxle(const T* a, I lo, I hi, T x) {
  while (hi - lo > 1) {
    I mid = lo + (hi - lo) / 2;
    if (a[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

}  // namespace gbfs
