// Device helpers shared by the single-source and multi-source kernels.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace gbfs {

// Writes chunk[c] = k for every chunk start c * kChunk inside [cum, cum + deg).
template <typename OffT>
__device__ __forceinline__ void write_chunks(int32_t* chunk, OffT cum, OffT deg, int32_t k) {
  if (deg <= 0) return;
  OffT c = (cum + kChunk - 1) / kChunk;
  const OffT end = cum + deg;
  for (; c * kChunk < end; ++c) chunk[c] = k;
}

// Tile descriptors of frontier entry k (degree deg at scan position cum, column base
// base = off[v] - cum, caller id u) for every chunk boundary inside its edge range.
template <typename OffT>
__device__ __forceinline__ void write_descs(TileDesc<OffT>* desc, OffT cum, OffT deg, int32_t k, int32_t u,
                                            OffT base) {
  if (deg <= 0) return;
  OffT c = (cum + kChunk - 1) / kChunk;
  const OffT end = cum + deg;
  for (; c * kChunk < end; ++c) desc[c] = TileDesc<OffT>{k, u, base + c * kChunk};
}

// Warp-collective version of write_chunks for one entry per lane (valid lanes only): entries
// crossing more than 32 chunk boundaries are written by the whole warp. Every lane of the
// warp must call it.
template <typename OffT>
__device__ __forceinline__ void write_chunks_warp(int32_t* chunk, bool valid, OffT cum, OffT deg, int32_t k) {
  OffT c0 = 0, c1 = 0;
  if (valid && deg > 0) {
    c0 = (cum + kChunk - 1) / kChunk;
    c1 = (cum + deg + kChunk - 1) / kChunk;
  }
  const bool big = c1 - c0 > 32;
  if (!big)
    for (OffT c = c0; c < c1; ++c) chunk[c] = k;
  const int lane = threadIdx.x & 31;
  for (unsigned bm = __ballot_sync(0xffffffffu, big); bm; bm &= bm - 1) {
    const int src = __ffs(bm) - 1;
    const OffT s0 = __shfl_sync(0xffffffffu, c0, src), s1 = __shfl_sync(0xffffffffu, c1, src);
    const int32_t sk = __shfl_sync(0xffffffffu, k, src);
    for (OffT c = s0 + lane; c < s1; c += 32) chunk[c] = sk;
  }
}

// Warp-collective version of write_descs for one entry per lane (valid lanes only): an
// entry whose edge range crosses more than 32 chunk boundaries (a hub row) has its
// descriptors written by the whole warp instead of serially by its own lane. Every lane of
// the warp must call it.
template <typename OffT>
__device__ __forceinline__ void write_descs_warp(TileDesc<OffT>* desc, bool valid, OffT cum, OffT deg, int32_t k,
                                                 int32_t u, OffT base) {
  OffT c0 = 0, c1 = 0;  // boundaries c * kChunk in [cum, cum + deg)
  if (valid && deg > 0) {
    c0 = (cum + kChunk - 1) / kChunk;
    c1 = (cum + deg + kChunk - 1) / kChunk;
  }
  const bool big = c1 - c0 > 32;
  if (!big)
    for (OffT c = c0; c < c1; ++c) desc[c] = TileDesc<OffT>{k, u, base + c * kChunk};
  const int lane = threadIdx.x & 31;
  for (unsigned bm = __ballot_sync(0xffffffffu, big); bm; bm &= bm - 1) {
    const int src = __ffs(bm) - 1;
    const OffT s0 = __shfl_sync(0xffffffffu, c0, src), s1 = __shfl_sync(0xffffffffu, c1, src);
    const OffT sb = __shfl_sync(0xffffffffu, base, src);
    const int32_t sk = __shfl_sync(0xffffffffu, k, src), su = __shfl_sync(0xffffffffu, u, src);
    for (OffT c = s0 + lane; c < s1; c += 32) desc[c] = TileDesc<OffT>{sk, su, sb + c * kChunk};
  }
}

// Frontier marks of ordered wave levels, one byte per vertex holding 0 or 1: bit j of the
// result is set when byte j of the 32-bit word x is 1 (four vertices' marks per word).
__host__ __device__ __forceinline__ unsigned mark_bits(unsigned x) {
  return (x & 1u) | ((x >> 7) & 2u) | ((x >> 14) & 4u) | ((x >> 21) & 8u);
}

// Exclusive scan of one value per thread across the block; *total receives the sum.
// s_warp needs 33 entries. Every thread of the block must call it.
template <typename OffT>
__device__ __forceinline__ OffT block_exclusive_scan(OffT x, OffT* s_warp, OffT* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  OffT inc = warp_inclusive_scan(x);
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    OffT t = lane < nw ? s_warp[lane] : 0;
    OffT ti = warp_inclusive_scan(t);
    if (lane < nw) s_warp[lane] = ti - t;
    if (lane == nw - 1) s_warp[32] = ti;
  }
  __syncthreads();
  OffT ex = s_warp[w] + inc - x;
  *total = s_warp[32];
  __syncthreads();
  return ex;
}

}  // namespace gbfs
