// The paper's 2D-partitioned search (Sec. 3.2, Algorithm 2; Sec. 3.4, Algorithm 3; Sec. 3.5,
// the frontier update), emulated on one GPU: the R x C processors P_ij are virtual, each
// with its own local CSC, level / predecessor arrays and visited bitmap in device memory,
// and the expand (vertical) and fold (horizontal) exchanges are copies between their
// buffers. It reproduces what the single-processor path leaves out: expansion into
// dst_verts blocks for other processor columns (tgt_j != j), the fold, and the update
// kernel with its sender-column predecessors.
//
// Partitioning (Sec. 3.1, after Yoo et al.): vertices are split into R C blocks of B, block
// b owned by P_ij with b = j R + i. Edge (u, v) of the adjacency matrix (column u, row v)
// belongs to P_ij with j = u / (N / C) and i = (v / B) mod R, so every edge list of a vertex
// of column block j is spread over the processors of grid column j (property i) and every
// edge's destination is owned in the sender's grid row (property ii). P_ij numbers its N / C
// columns locally from j N / C, and its N / R rows as row block m R + i -> local block m, so
// every processor of a grid row uses the same local index for a row.
#include <cuda_runtime.h>

#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <mutex>
#include <vector>

#include "capi_internal.h"
#include "gbfs.h"
#include "kernels.h"

namespace gbfs {
namespace {

// Grid geometry. n_pad = R C B >= n.
struct Geo {
  int R, C;
  int64_t n, B, NC, NR;  // block size, columns (N / C) and rows (N / R) of a local matrix
  __host__ __device__ int owner_i(int64_t v) const { return (int)((v / B) % R); }
  __host__ __device__ int owner_j(int64_t v) const { return (int)((v / B) / R); }
  __host__ __device__ int64_t local_row(int64_t v) const { return ((v / B) / R) * B + v % B; }
  // ROW2COL of Algorithm 3: local row -> local column of the same vertex at its owner P_ij
  // (row block m R + i is the owner's own block when m == j: column (j R + i) B - j N / C + off)
  __host__ __device__ int64_t row_to_col(int64_t row, int i) const { return (int64_t)i * B + row % B; }
};

// Edge counts of every (processor, local column): cnt[p][u_l], p = i C + j.
template <typename OffT>
__global__ void k_part_count(const OffT* __restrict__ off, const int32_t* __restrict__ cols, Geo geo,
                             unsigned long long* cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < geo.n; u += stride) {
    const int j = (int)(u / geo.NC);
    const int64_t ul = u - (int64_t)j * geo.NC;
    for (OffT e = off[u]; e < off[u + 1]; ++e) {
      const int32_t v = cols[e];
      if ((uint32_t)v >= (uint64_t)geo.n) continue;  // reported by the range check of the build
      const int p = geo.owner_i(v) * geo.C + j;
      atomicAdd(cnt + (size_t)p * (geo.NC + 1) + ul, 1ull);
    }
  }
}

// Rows of every local CSC column, in any order (the cursor starts at the column offset).
template <typename OffT>
__global__ void k_part_fill(const OffT* __restrict__ off, const int32_t* __restrict__ cols, Geo geo,
                            unsigned long long* cursor, int32_t* rows, unsigned* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < geo.n; u += stride) {
    const int j = (int)(u / geo.NC);
    const int64_t ul = u - (int64_t)j * geo.NC;
    for (OffT e = off[u]; e < off[u + 1]; ++e) {
      const int32_t v = cols[e];
      if ((uint32_t)v >= (uint64_t)geo.n) {
        atomicOr(err, kErrColumnRange);
        continue;
      }
      const int p = geo.owner_i(v) * geo.C + j;
      const unsigned long long at = atomicAdd(cursor + (size_t)p * (geo.NC + 1) + ul, 1ull);
      rows[at] = (int32_t)geo.local_row(v);
    }
  }
}

// Per-processor state, all processors back to back: p = i C + j.
struct Part {
  Geo geo{};
  unsigned long long* coff = nullptr;  // [RC][NC + 1] local CSC column offsets (global positions in rows)
  int32_t* rows = nullptr;             // [nnz] local row ids
  int32_t* level = nullptr;            // [RC][NR]
  int32_t* pred = nullptr;             // [RC][NR]: local column of u, or -(sender column + 2)
  uint32_t* bmap = nullptr;            // [RC][NRW]
  int64_t nrw = 0;                     // bitmap words per processor
  int32_t* front = nullptr;            // [RC][B] local columns of the processor's frontier
  int64_t* front_n = nullptr;          // [RC]
  int32_t* all_front = nullptr;        // [C][NC] gathered frontier of each grid column
  int64_t* all_n = nullptr;            // [C]
  unsigned long long* cum = nullptr;   // [RC][NC + 1] exclusive degree scan over all_front, per processor
  unsigned long long* pcum = nullptr;  // [RC + 1] edge totals of the processors, scanned
  int32_t* dst = nullptr;              // [RC][C][B] dst_verts blocks
  unsigned long long* dst_n = nullptr; // [RC][C]
  int32_t* recv = nullptr;             // [RC][C][B] (vertex, from sender column index in the block)
  int64_t* recv_n = nullptr;           // [RC][C]
  unsigned* err = nullptr;
  void* scan_tmp = nullptr;
  size_t scan_bytes = 0;
};

__global__ void k_2d_init(Part P) {
  const Geo& g = P.geo;
  const int64_t RC = (int64_t)g.R * g.C;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t x = tid; x < RC * g.NR; x += stride) {
    P.level[x] = -1;
    P.pred[x] = -1;
  }
  for (int64_t x = tid; x < RC * P.nrw; x += stride) P.bmap[x] = 0u;
  for (int64_t x = tid; x < RC; x += stride) P.front_n[x] = 0;
}

__global__ void k_2d_seed(Part P, int32_t root) {
  const Geo& g = P.geo;
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // Algorithm 2's root placement: the owner of the root
    const int i = g.owner_i(root), j = g.owner_j(root);
    const int64_t p = (int64_t)i * g.C + j, row = g.local_row(root);
    P.level[p * g.NR + row] = 0;
    P.pred[p * g.NR + row] = -1;  // the root's parent is written as the root itself at assembly
    P.bmap[p * P.nrw + row / 32] |= 1u << (row % 32);
    P.front[p * g.B] = (int32_t)g.row_to_col(row, i);
    P.front_n[p] = 1;
  }
}

// expand_comm (Algorithm 2's expand_comm step): every processor of grid column j receives the
// frontiers of all of them, concatenated in processor-row order.
__global__ void k_2d_expand_comm(Part P) {
  const Geo& g = P.geo;
  const int j = blockIdx.y;
  int64_t base = 0;
  for (int i = 0; i < g.R; ++i) {
    const int64_t p = (int64_t)i * g.C + j, k = P.front_n[p];
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < k; x += (int64_t)gridDim.x * blockDim.x)
      P.all_front[(int64_t)j * g.NC + base + x] = P.front[p * g.B + x];
    base += k;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) P.all_n[j] = base;
}

// Degrees of the gathered frontier in each processor's local CSC (input of the scans).
__global__ void k_2d_degrees(Part P) {
  const Geo& g = P.geo;
  const int p = blockIdx.y, j = p % g.C;
  const int64_t k = P.all_n[j];
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= g.NC; x += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long d = 0;
    if (x < k) {
      const int32_t ul = P.all_front[(int64_t)j * g.NC + x];
      const unsigned long long* co = P.coff + (size_t)p * (g.NC + 1);
      d = co[ul + 1] - co[ul];
    }
    P.cum[(size_t)p * (g.NC + 1) + x] = d;
  }
}

// Edge totals per processor, then their scan: the combined edge space of all processors.
__global__ void k_2d_totals(Part P) {
  const Geo& g = P.geo;
  const int64_t RC = (int64_t)g.R * g.C;
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  unsigned long long run = 0;
  for (int64_t p = 0; p < RC; ++p) {
    P.pcum[p] = run;
    run += P.cum[(size_t)p * (g.NC + 1) + g.NC];  // after the exclusive scan: the total sits at NC
  }
  P.pcum[RC] = run;
  for (int64_t x = 0; x < RC * g.C; ++x) P.dst_n[x] = 0;
}

// expand_frontier (Algorithm 3): thread -> edge of the combined edge space; binary searches
// give the processor (pcum) and the frontier entry (its scan: the binary search of
// Algorithm 3). A newly visited row v goes to the dst_verts block of its owner's processor
// column tgt = v / B (Algorithm 3's frontier append): as a row id for another column, as the
// owner's local column for this one, whose level is set here; pred[v] = u either way
// (Algorithm 3's output writes).
__global__ void k_2d_expand(Part P, int32_t lvl) {
  const Geo& g = P.geo;
  const int64_t RC = (int64_t)g.R * g.C;
  const unsigned long long total = P.pcum[RC];
  for (unsigned long long gid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; gid < total;
       gid += (unsigned long long)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = RC;  // processor: largest p with pcum[p] <= gid
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) / 2;
      if (P.pcum[mid] <= gid) lo = mid; else hi = mid;
    }
    const int64_t p = lo;
    const int i = (int)(p / g.C), j = (int)(p % g.C);
    const unsigned long long e = gid - P.pcum[p];
    const unsigned long long* cum = P.cum + (size_t)p * (g.NC + 1);
    int64_t klo = 0, khi = P.all_n[j];  // frontier entry: largest k with cum[k] <= e
    while (khi - klo > 1) {
      const int64_t mid = (klo + khi) / 2;
      if (cum[mid] <= e) klo = mid; else khi = mid;
    }
    const int32_t ul = P.all_front[(int64_t)j * g.NC + klo];
    const unsigned long long* co = P.coff + (size_t)p * (g.NC + 1);
    const int32_t v = P.rows[co[ul] + (e - cum[klo])];
    uint32_t* bmap = P.bmap + p * P.nrw;
    const uint32_t m = 1u << (v % 32);
    if (bmap[v / 32] & m) continue;
    const uint32_t q = atomicOr(bmap + v / 32, m);
    if (q & m) continue;
    const int tgt = (int)(v / g.B);
    const unsigned long long at = atomicAdd(P.dst_n + p * g.C + tgt, 1ull);
    int32_t* blk = P.dst + ((size_t)p * g.C + tgt) * g.B;
    if (tgt != j) {
      blk[at] = v;
    } else {
      blk[at] = (int32_t)g.row_to_col(v, i);
      P.level[p * g.NR + v] = lvl;
    }
    P.pred[p * g.NR + v] = ul;
  }
}

// Algorithm 3's output writes and fold_comm: the local block becomes the processor's frontier; every other
// block goes to the processor of the same grid row that owns it (receiver column tgt),
// recorded per sender column.
__global__ void k_2d_fold(Part P) {
  const Geo& g = P.geo;
  const int p = blockIdx.y, i = p / g.C, j = p % g.C;
  for (int tgt = 0; tgt < g.C; ++tgt) {
    const int64_t k = (int64_t)P.dst_n[(int64_t)p * g.C + tgt];
    const int32_t* src = P.dst + ((size_t)p * g.C + tgt) * g.B;
    const int64_t q = (int64_t)i * g.C + tgt;  // receiver
    int32_t* out = tgt == j ? P.front + (size_t)p * g.B : P.recv + ((size_t)q * g.C + j) * g.B;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < k; x += (int64_t)gridDim.x * blockDim.x)
      out[x] = src[x];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (tgt == j)
        P.front_n[p] = k;
      else
        P.recv_n[q * g.C + j] = k;
    }
  }
}

// update_frontier (Sec. 3.5): one thread per received vertex; the unvisited ones get their
// level and, as predecessor, the sender's processor column (the sender kept the parent),
// and join the processor's frontier.
__global__ void k_2d_update(Part P, int32_t lvl) {
  const Geo& g = P.geo;
  const int q = blockIdx.y, i = q / g.C, jq = q % g.C;
  for (int src = 0; src < g.C; ++src) {
    if (src == jq) continue;
    const int64_t k = P.recv_n[(int64_t)q * g.C + src];
    const int32_t* in = P.recv + ((size_t)q * g.C + src) * g.B;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < k; x += (int64_t)gridDim.x * blockDim.x) {
      const int32_t v = in[x];
      uint32_t* bmap = P.bmap + (int64_t)q * P.nrw;
      const uint32_t m = 1u << (v % 32);
      if (bmap[v / 32] & m) continue;
      const uint32_t old = atomicOr(bmap + v / 32, m);
      if (old & m) continue;
      P.level[(int64_t)q * g.NR + v] = lvl;
      P.pred[(int64_t)q * g.NR + v] = -(src + 2);
      const unsigned long long at = atomicAdd(reinterpret_cast<unsigned long long*>(P.front_n + q), 1ull);
      P.front[(int64_t)q * g.B + at] = (int32_t)g.row_to_col(v, i);
    }
  }
}

__global__ void k_2d_recv_clear(Part P) {
  const int64_t RC = (int64_t)P.geo.R * P.geo.C;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < RC * P.geo.C; x += (int64_t)gridDim.x * blockDim.x)
    P.recv_n[x] = 0;
}

__global__ void k_2d_front_total(Part P, int64_t* out) {
  const int64_t RC = (int64_t)P.geo.R * P.geo.C;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int64_t t = 0;
    for (int64_t p = 0; p < RC; ++p) t += P.front_n[p];
    *out = t;
  }
}

// Global outputs from the owners' arrays: level of v at its owner; the predecessor's global
// id from the owner's entry (a local column of the owner's grid column), or, for a vertex
// found by another column, from that sender's entry for the same local row.
__global__ void k_2d_assemble(Part P, int32_t root, int32_t* levels, int32_t* parents) {
  const Geo& g = P.geo;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += stride) {
    const int i = g.owner_i(v), j = g.owner_j(v);
    const int64_t row = g.local_row(v), p = (int64_t)i * g.C + j;
    const int32_t l = P.level[p * g.NR + row];
    int32_t par = -1;
    if (v == root) {
      par = root;
    } else if (l >= 0) {
      int32_t x = P.pred[p * g.NR + row];
      int col = j;
      if (x < 0) {  // found by the processor of column -(x + 2) in this grid row
        col = -(x + 2);
        x = P.pred[((int64_t)i * g.C + col) * g.NR + row];
      }
      par = (int32_t)((int64_t)col * g.NC + x);
    }
    levels[v] = l;
    parents[v] = par;
  }
}

template <typename T>
cudaError_t dalloc2(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
}

void free_part(Part& P) {
  cudaFree(P.coff);
  cudaFree(P.rows);
  cudaFree(P.level);
  cudaFree(P.pred);
  cudaFree(P.bmap);
  cudaFree(P.front);
  cudaFree(P.front_n);
  cudaFree(P.all_front);
  cudaFree(P.all_n);
  cudaFree(P.cum);
  cudaFree(P.pcum);
  cudaFree(P.dst);
  cudaFree(P.dst_n);
  cudaFree(P.recv);
  cudaFree(P.recv_n);
  cudaFree(P.err);
  cudaFree(P.scan_tmp);
  P = Part{};
}

// Partition build: counts, a scan of every processor's column offsets (one scan over the
// concatenated [RC][NC + 1] array gives global positions), then the fill.
template <typename OffT>
bfs_status build_part(const GraphDev& gd, int R, int C, Part& P, cudaStream_t st) {
  Geo geo;
  geo.R = R;
  geo.C = C;
  geo.n = gd.n;
  geo.B = (gd.n + (int64_t)R * C - 1) / ((int64_t)R * C);
  geo.NC = geo.B * R;
  geo.NR = geo.B * C;
  P.geo = geo;
  P.nrw = (geo.NR + 31) / 32;
  const int64_t RC = (int64_t)R * C;
  cudaError_t e = cudaSuccess;
  const size_t ncol = (size_t)RC * (geo.NC + 1);
  unsigned long long* cnt = nullptr;
  if ((e = dalloc2(&P.coff, ncol)) || (e = dalloc2(&cnt, ncol)) || (e = dalloc2(&P.rows, (size_t)gd.nnz)) ||
      (e = dalloc2(&P.level, (size_t)(RC * geo.NR))) || (e = dalloc2(&P.pred, (size_t)(RC * geo.NR))) ||
      (e = dalloc2(&P.bmap, (size_t)(RC * P.nrw))) || (e = dalloc2(&P.front, (size_t)(RC * geo.B))) ||
      (e = dalloc2(&P.front_n, (size_t)RC)) || (e = dalloc2(&P.all_front, (size_t)(C * geo.NC))) ||
      (e = dalloc2(&P.all_n, (size_t)C)) || (e = dalloc2(&P.cum, ncol)) || (e = dalloc2(&P.pcum, (size_t)RC + 1)) ||
      (e = dalloc2(&P.dst, (size_t)(RC * C * geo.B))) || (e = dalloc2(&P.dst_n, (size_t)(RC * C))) ||
      (e = dalloc2(&P.recv, (size_t)(RC * C * geo.B))) || (e = dalloc2(&P.recv_n, (size_t)(RC * C))) ||
      (e = dalloc2(&P.err, 1))) {
    cudaFree(cnt);
    free_part(P);
    return e == cudaErrorMemoryAllocation ? fail(BFS_ERR_OOM, "2D partition buffers") : cuda_fail(e, "2D partition");
  }
  size_t tb = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tb, cnt, P.coff, (int64_t)ncol, st);
  size_t tb2 = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tb2, P.cum, P.cum, (int64_t)(geo.NC + 1), st);
  P.scan_bytes = std::max(tb, tb2);
  if ((e = cudaMalloc(&P.scan_tmp, std::max<size_t>(P.scan_bytes, 16))) != cudaSuccess) {
    cudaFree(cnt);
    free_part(P);
    return fail(BFS_ERR_OOM, "2D partition scan buffer");
  }
  const int grid = std::max(1, gd.num_sms) * 8;
  const OffT* off = reinterpret_cast<const OffT*>(gd.off);
  cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * ncol, st);
  cudaMemsetAsync(P.err, 0, sizeof(unsigned), st);
  k_part_count<OffT><<<grid, 256, 0, st>>>(off, gd.cols, geo, cnt);
  tb = P.scan_bytes;
  e = cub::DeviceScan::ExclusiveSum(P.scan_tmp, tb, cnt, P.coff, (int64_t)ncol, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, P.coff, sizeof(unsigned long long) * ncol, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) {
    k_part_fill<OffT><<<grid, 256, 0, st>>>(off, gd.cols, geo, cnt, P.rows, P.err);
    e = cudaStreamSynchronize(st);
  }
  cudaFree(cnt);
  unsigned err = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&err, P.err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    free_part(P);
    return cuda_fail(e, "2D partition build");
  }
  if (err & kErrColumnRange) {
    free_part(P);
    return fail(BFS_ERR_INVALID_GRAPH, "a column id outside [0, n) was met");
  }
  return BFS_OK;
}

template <typename OffT>
bfs_status run_2d(const GraphDev& gd, int R, int C, int32_t root, int32_t* levels, int32_t* parents,
                  cudaStream_t st, int* depth) {
  Part P;
  bfs_status s = build_part<OffT>(gd, R, C, P, st);
  if (s != BFS_OK) return s;
  const Geo& g = P.geo;
  const int RC = R * C;
  const int grid = std::max(1, gd.num_sms) * 4;
  int64_t* total_dev = nullptr;
  cudaError_t e = dalloc2(&total_dev, 1);
  int64_t total = 1;
  int lvl = 1;
  if (e == cudaSuccess) {
    k_2d_init<<<grid, 256, 0, st>>>(P);
    k_2d_seed<<<1, 32, 0, st>>>(P, root);
    for (; total > 0 && lvl <= g.n + 1 && e == cudaSuccess; ++lvl) {
      k_2d_expand_comm<<<dim3(64, C), 256, 0, st>>>(P);
      k_2d_degrees<<<dim3(64, RC), 256, 0, st>>>(P);
      for (int p = 0; p < RC && e == cudaSuccess; ++p) {  // exclusive scans of the gathered degrees
        size_t tb = P.scan_bytes;
        e = cub::DeviceScan::ExclusiveSum(P.scan_tmp, tb, P.cum + (size_t)p * (g.NC + 1),
                                          P.cum + (size_t)p * (g.NC + 1), (int64_t)(g.NC + 1), st);
      }
      k_2d_totals<<<1, 32, 0, st>>>(P);
      k_2d_expand<<<grid, 256, 0, st>>>(P, lvl);
      k_2d_recv_clear<<<1, 256, 0, st>>>(P);
      k_2d_fold<<<dim3(16, RC), 256, 0, st>>>(P);
      k_2d_update<<<dim3(16, RC), 256, 0, st>>>(P, lvl);
      k_2d_front_total<<<1, 32, 0, st>>>(P, total_dev);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&total, total_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e == cudaSuccess) {
      k_2d_assemble<<<grid, 256, 0, st>>>(P, root, levels, parents);
      e = cudaStreamSynchronize(st);
    }
  }
  cudaFree(total_dev);
  free_part(P);
  if (e != cudaSuccess) return cuda_fail(e, "2D search");
  *depth = lvl - 1;
  return BFS_OK;
}

}  // namespace
}  // namespace gbfs

using namespace gbfs;

extern "C" GBFS_API bfs_status bfs_run_2d(bfs_graph_t G, int R, int C, int32_t root, int32_t* levels,
                                          int32_t* parents, void* stream) {
  clear_last_error();
  if (!G) return fail(BFS_ERR_INVALID_ARG, "graph is NULL");
  if (!levels || !parents) return fail(BFS_ERR_INVALID_ARG, "levels/parents is NULL");
  if (R < 1 || C < 1 || R > 64 || C > 64) return fail(BFS_ERR_INVALID_ARG, "R and C must be in [1, 64]");
  if (root < 0 || root >= G->g.n) return fail(BFS_ERR_INVALID_ARG, "root outside [0, n)");
  if (G->g.new_id)
    return fail(BFS_ERR_INVALID_ARG, "bfs_run_2d works in the graph's own numbering: create it without BFS_RELABEL_DEGREE");
  std::lock_guard<std::mutex> lock(G->mu);
  cudaError_t e = cudaSetDevice(G->g.device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  cudaPointerAttributes a{}, b{};
  if (cudaPointerGetAttributes(&a, levels) != cudaSuccess || cudaPointerGetAttributes(&b, parents) != cudaSuccess ||
      (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) ||
      (b.type != cudaMemoryTypeDevice && b.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return fail(BFS_ERR_INVALID_ARG, "bfs_run_2d: levels and parents must be device memory");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (G->last_done) cudaStreamWaitEvent(st, G->last_done, 0);
  int depth = 0;
  return G->g.off64 ? run_2d<int64_t>(G->g, R, C, root, levels, parents, st, &depth)
                    : run_2d<int32_t>(G->g, R, C, root, levels, parents, st, &depth);
}
