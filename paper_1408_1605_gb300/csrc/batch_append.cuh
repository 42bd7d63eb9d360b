// The appends of a wave's next frontier outside ordered levels: a CTA's or a warp's buffer of
// claimed vertices (vertex, degree) is reserved with one 64-bit atomic on the packed
// (count, edges) counter and written as list entries, degree-scan values, column bases and
// tile descriptors. Block- and warp-level device functions: the expansion kernels in
// bfs_batch_kernels.cu call them, and the CPU unit tests run them on an emulated block.
#pragma once

#include "batch.h"
#include "device_util.cuh"

namespace gbfs {

template <typename OffT, int BLOCK, int CLAIM>
__device__ __forceinline__ void batch_flush(const BatchArgs<OffT>& a, int nxt, int q3n, int2* s_claim, int nc,
                                            OffT* s_warp, unsigned long long* s_resv) {
  constexpr int P = (CLAIM + BLOCK - 1) / BLOCK;
  const int lo = min(nc, (int)threadIdx.x * P), hi = min(nc, lo + P);
  OffT mine = 0;
  for (int i = lo; i < hi; ++i) mine += (OffT)s_claim[i].y;
  OffT total;
  OffT run = block_exclusive_scan(mine, s_warp, &total);
  if (threadIdx.x == 0) *s_resv = atomicAdd(&a.ctl->counter[nxt], a.pk.make(nc, (long long)total));
  __syncthreads();
  const unsigned long long resv = *s_resv;
  const long long slot0 = a.pk.count(resv);
  run += (OffT)a.pk.edges(resv);
  for (int t = 0; t < P; ++t) {  // uniform trip count: the chunk writes are warp-collective
    const int i = lo + t;
    const bool valid = i < hi;
    OffT d = 0, b = 0;
    int32_t v = 0;
    const int32_t slot = (int32_t)(slot0 + i);
    if (valid) {
      v = s_claim[i].x;
      d = (OffT)s_claim[i].y;
      b = a.off[v] - run;
      a.qv[q3n][slot] = v;
      a.cum[nxt][slot] = run;
      a.base[nxt][slot] = b;
    }
    write_descs_warp(a.chunk[nxt], valid, run, d, slot, v, b);
    run += d;
  }
}

// Appends a warp's buffered claims (vertex, degree) to the wave's next frontier with one
// 64-bit atomic (the batched counterpart of the single-source warp append).
template <typename OffT, int P>
__device__ __forceinline__ void batch_warp_flush(const BatchArgs<OffT>& a, int nxt, int q3n, const int2* buf,
                                                 int nc) {
  const int lane = threadIdx.x & 31;
  const int lo = min(nc, lane * P), hi = min(nc, lo + P);
  OffT mine = 0;
  for (int i = lo; i < hi; ++i) mine += (OffT)buf[i].y;
  const OffT inc = warp_inclusive_scan(mine);
  const OffT total = __shfl_sync(0xffffffffu, inc, 31);
  unsigned long long resv = 0;
  if (lane == 0) resv = atomicAdd(&a.ctl->counter[nxt], a.pk.make(nc, (long long)total));
  resv = __shfl_sync(0xffffffffu, resv, 0);
  const long long slot0 = a.pk.count(resv);
  OffT run = (OffT)a.pk.edges(resv) + inc - mine;
  for (int t = 0; t < P; ++t) {  // uniform trip count: the chunk writes are warp-collective
    const int i = lo + t;
    const bool valid = i < hi;
    OffT d = 0, b = 0;
    int32_t v = 0;
    const int32_t slot = (int32_t)(slot0 + i);
    if (valid) {
      v = buf[i].x;
      d = (OffT)buf[i].y;
      b = a.off[v] - run;
      a.qv[q3n][slot] = v;
      a.cum[nxt][slot] = run;
      a.base[nxt][slot] = b;
    }
    write_descs_warp(a.chunk[nxt], valid, run, d, slot, v, b);
    run += d;
  }
  __syncwarp();
}

}  // namespace gbfs
