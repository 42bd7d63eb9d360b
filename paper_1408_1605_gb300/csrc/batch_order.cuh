// The two ways k_batch_order rebuilds an ordered level's next frontier (the list, its degree
// scan, column bases and tile descriptors, in vertex order within a round), as block-level
// device functions: the kernel in bfs_batch_kernels.cu calls one of them, and the CPU unit
// tests run them on an emulated block.
#pragma once

#include "batch.h"
#include "device_util.cuh"

namespace gbfs {

// k_batch_order on a degree-relabelled graph: one vertex per thread, read from the 64-bit
// masks F_{t+1}, rounds of blockDim.x consecutive vertices per CTA (the hubs, at the lowest
// ids, spread over many CTAs), a block scan of the marked vertices' counts and degrees, one
// reservation per round, then each marked vertex writes its list entry, scan value, column
// base and tile descriptors.
template <typename OffT>
__device__ __forceinline__ void order_from_masks(const BatchArgs<OffT>& a, BatchCtl* ctl, int nxt, int q3n,
                                                 OffT* s_warp, unsigned long long* s_resv_p) {
  unsigned long long& s_resv = *s_resv_p;
  const unsigned long long* Fn = a.fmask[q3n];
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x; r0 < a.n; r0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = r0 + threadIdx.x;
    const bool in = v < a.n && Fn[v] != 0ull;
    OffT o0 = 0, d = 0;
    if (in) {
      o0 = a.off[v];
      d = a.off[v + 1] - o0;
    }
    OffT tot_cnt, tot_deg;
    const OffT ex_cnt = block_exclusive_scan((OffT)(in ? 1 : 0), s_warp, &tot_cnt);
    const OffT ex_deg = block_exclusive_scan(d, s_warp, &tot_deg);
    if (tot_cnt == 0) continue;  // block-uniform
    if (threadIdx.x == 0) s_resv = atomicAdd(&ctl->counter[nxt], a.pk.make((long long)tot_cnt, (long long)tot_deg));
    __syncthreads();
    const unsigned long long resv = s_resv;
    __syncthreads();
    const int64_t slot = a.pk.count(resv) + (int64_t)ex_cnt;
    const OffT run = (OffT)a.pk.edges(resv) + ex_deg;
    const OffT b = o0 - run;
    if (in) {
      a.qv[q3n][slot] = (int32_t)v;
      a.cum[nxt][slot] = run;
      a.base[nxt][slot] = b;
    }
    write_descs_warp(a.chunk[nxt], in, run, d, (int32_t)slot, (int32_t)v, b);
  }
}

// k_batch_order on any other graph: from the byte marks the expansion left (1 / 8 of the
// bytes of the masks). Each thread takes 16 consecutive vertices with one 16-byte load of
// their marks and clears the marks it found; a block scan of the threads' marked counts and
// degree sums, one reservation per round of 16 x blockDim.x vertices, then each thread writes
// its marked vertices' list entries, scan values, column bases and tile descriptors in vertex
// order, the warp's lanes stepping through their marked vertices together.
template <typename OffT>
__device__ __forceinline__ void order_from_marks(const BatchArgs<OffT>& a, BatchCtl* ctl, int nxt, int q3n,
                                                 OffT* s_warp, unsigned long long* s_resv_p) {
  constexpr int V = 16;  // vertices per thread: one uint4 of marks
  constexpr unsigned kFull = 0xffffffffu;
  unsigned long long& s_resv = *s_resv_p;
  uint4* marks = reinterpret_cast<uint4*>(a.fmark);
  const int64_t groups = (a.n + V - 1) / V;  // the marks array holds whole 16-byte groups
  for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x; g0 < groups; g0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gi = g0 + threadIdx.x;
    const int64_t v0 = gi * V;
    unsigned sel = 0;  // bit i: vertex v0 + i is in the next frontier
    if (gi < groups) {
      const uint4 m = marks[gi];
      if (m.x | m.y | m.z | m.w) {
        sel = mark_bits(m.x) | (mark_bits(m.y) << 4) | (mark_bits(m.z) << 8) | (mark_bits(m.w) << 12);
        marks[gi] = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    OffT deg = 0;
    for (unsigned s = sel; s; s &= s - 1) {
      const int64_t v = v0 + __ffs(s) - 1;
      deg += a.off[v + 1] - a.off[v];
    }
    OffT tot_cnt, tot_deg;
    const OffT ex_cnt = block_exclusive_scan((OffT)__popc(sel), s_warp, &tot_cnt);
    const OffT ex_deg = block_exclusive_scan(deg, s_warp, &tot_deg);
    if (tot_cnt == 0) continue;  // block-uniform
    if (threadIdx.x == 0) s_resv = atomicAdd(&ctl->counter[nxt], a.pk.make((long long)tot_cnt, (long long)tot_deg));
    __syncthreads();
    const unsigned long long resv = s_resv;
    __syncthreads();
    int64_t slot = a.pk.count(resv) + (int64_t)ex_cnt;
    OffT run = (OffT)a.pk.edges(resv) + ex_deg;
    unsigned rem = sel;
    while (__any_sync(kFull, rem != 0u)) {  // warp-uniform: the descriptor writes are warp-collective
      const bool in = rem != 0u;
      int64_t v = 0;
      OffT o0 = 0, d = 0;
      if (in) {
        v = v0 + __ffs(rem) - 1;
        rem &= rem - 1u;
        o0 = a.off[v];
        d = a.off[v + 1] - o0;
      }
      const OffT b = o0 - run;
      if (in) {
        a.qv[q3n][slot] = (int32_t)v;
        a.cum[nxt][slot] = run;
        a.base[nxt][slot] = b;
      }
      write_descs_warp(a.chunk[nxt], in, run, d, (int32_t)slot, (int32_t)v, b);
      if (in) {
        ++slot;
        run += d;
      }
    }
  }
}

}  // namespace gbfs
