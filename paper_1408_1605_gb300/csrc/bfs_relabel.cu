// Degree relabelling of a device CSR, done once when a graph is created (graph
// construction, outside every timed search, like the generation and partitioning that the
// paper's TEPS figures leave out, Sec. 4).
//
// Vertices are renumbered by non-increasing degree (ties keep the input order), every row
// is rebuilt in the new numbering and sorted. In a skewed graph (R-MAT) a few percent of
// the vertices are the endpoints of most edges; after relabelling their visited bits share
// a few hundred KB of the bitmap that stay in each SM's L1 cache, so the per-edge bitmap
// non-atomic pre-check of Algorithm 3 mostly hits L1 instead of going to L2. Searches keep
// taking and returning the caller's vertex ids: the kernels map the root through new_id
// and write levels and parents at old_id[v].
#include <cuda_runtime.h>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cub/device/device_segmented_sort.cuh>

#include <algorithm>

#include "kernels.h"

namespace gbfs {

namespace {

template <typename OffT>
__global__ void k_degree_keys(const OffT* __restrict__ off, int64_t n, uint32_t* deg, int32_t* ids) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const OffT d = off[i + 1] - off[i];
    deg[i] = (uint32_t)min((int64_t)d, (int64_t)0xffffffff);
    ids[i] = (int32_t)i;
  }
}

// new_id[order[i]] = i, and the row lengths of the new numbering (scanned into offsets).
template <typename OffT>
__global__ void k_invert(const OffT* __restrict__ off, const int32_t* __restrict__ order, int64_t n,
                         int32_t* new_id, OffT* len) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int32_t o = order[i];
    new_id[o] = (int32_t)i;
    len[i] = off[o + 1] - off[o];
  }
}

// One warp per new row: copy the old row and map every column id. An id outside [0, n)
// is kept as it is, so that the expansion kernels still report it as a range error.
template <typename OffT>
__global__ void k_gather_rows(const OffT* __restrict__ off, const int32_t* __restrict__ cols,
                              const OffT* __restrict__ new_off, const int32_t* __restrict__ order,
                              const int32_t* __restrict__ new_id, int64_t n, int32_t* out) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
    const int32_t o = order[i];
    const OffT b = off[o], d = off[o + 1] - b, nb = new_off[i];
    for (OffT j = lane; j < d; j += 32) {
      const int32_t c = cols[b + j];
      out[nb + j] = (uint32_t)c < (uint64_t)n ? new_id[c] : c;
    }
  }
}

struct DevBufs {
  void* p[8] = {};
  int k = 0;
  template <typename T>
  cudaError_t alloc(T** out, size_t count) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(out), std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) p[k++] = *out;
    return e;
  }
  void release(void* keep0, void* keep1, void* keep2, void* keep3) {
    for (int i = 0; i < k; ++i)
      if (p[i] != keep0 && p[i] != keep1 && p[i] != keep2 && p[i] != keep3) cudaFree(p[i]);
    k = 0;
  }
};

template <typename OffT>
cudaError_t relabel_t(GraphDev& g, cudaStream_t st) {
  const int64_t n = g.n, nnz = g.nnz;
  const OffT* off = reinterpret_cast<const OffT*>(g.off);
  const int grid = std::max(1, g.num_sms) * 8;
  DevBufs b;
  uint32_t *deg = nullptr, *deg_sorted = nullptr;
  int32_t *ids = nullptr, *order = nullptr, *new_id = nullptr, *new_cols = nullptr;
  OffT *len = nullptr, *new_off = nullptr;
  void* temp = nullptr;
  cudaError_t e;
  if ((e = b.alloc(&deg, n)) != cudaSuccess || (e = b.alloc(&deg_sorted, n)) != cudaSuccess ||
      (e = b.alloc(&ids, n)) != cudaSuccess || (e = b.alloc(&order, n)) != cudaSuccess ||
      (e = b.alloc(&new_id, n)) != cudaSuccess || (e = b.alloc(&len, n)) != cudaSuccess ||
      (e = b.alloc(&new_off, n + 1)) != cudaSuccess || (e = b.alloc(&new_cols, nnz)) != cudaSuccess) {
    b.release(nullptr, nullptr, nullptr, nullptr);
    return e;
  }
  cub::DoubleBuffer<int32_t> keys(new_cols, g.cols);
  size_t t_sort = 0, t_scan = 0, t_seg = 0;
  cub::DeviceRadixSort::SortPairsDescending(nullptr, t_sort, deg, deg_sorted, ids, order, (int64_t)n, 0, 32, st);
  cub::DeviceScan::InclusiveSum(nullptr, t_scan, len, new_off + 1, (int64_t)n, st);
  if (nnz > 0) cub::DeviceSegmentedSort::SortKeys(nullptr, t_seg, keys, nnz, n, new_off, new_off + 1, st);
  const size_t t_bytes = std::max(t_sort, std::max(t_scan, t_seg));
  if ((e = cudaMalloc(&temp, std::max<size_t>(t_bytes, 16))) != cudaSuccess) {
    b.release(nullptr, nullptr, nullptr, nullptr);
    return e;
  }
  size_t tb = t_bytes;
  k_degree_keys<OffT><<<grid, 256, 0, st>>>(off, n, deg, ids);
  e = cub::DeviceRadixSort::SortPairsDescending(temp, tb, deg, deg_sorted, ids, order, (int64_t)n, 0, 32, st);
  if (e == cudaSuccess) {
    k_invert<OffT><<<grid, 256, 0, st>>>(off, order, n, new_id, len);
    e = cudaMemsetAsync(new_off, 0, sizeof(OffT), st);
  }
  tb = t_bytes;
  if (e == cudaSuccess) e = cub::DeviceScan::InclusiveSum(temp, tb, len, new_off + 1, (int64_t)n, st);
  if (e == cudaSuccess && nnz > 0) {
    k_gather_rows<OffT><<<grid, 256, 0, st>>>(off, g.cols, new_off, order, new_id, n, new_cols);
    tb = t_bytes;
    // rows sorted in the new numbering; the old column array is the sort's second buffer
    e = cub::DeviceSegmentedSort::SortKeys(temp, tb, keys, nnz, n, new_off, new_off + 1, st);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(temp);
  if (e != cudaSuccess) {
    b.release(nullptr, nullptr, nullptr, nullptr);  // the caller destroys the graph (cols may be overwritten)
    return e;
  }
  // the sorted rows end in either buffer; the other one (old columns or scratch) goes
  int32_t* sorted = nnz > 0 ? keys.Current() : g.cols;
  b.release(new_off, new_id, order, sorted);
  if (sorted != g.cols) cudaFree(g.cols);
  cudaFree(g.off);
  g.off = new_off;
  g.cols = sorted;
  g.new_id = new_id;
  g.old_id = order;
  return cudaSuccess;
}

}  // namespace

cudaError_t relabel_by_degree(GraphDev& g, cudaStream_t st) {
  if (g.new_id) return cudaSuccess;
  return g.off64 ? relabel_t<int64_t>(g, st) : relabel_t<int32_t>(g, st);
}

}  // namespace gbfs
