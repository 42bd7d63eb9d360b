// Single-source search that allocates no memory: every work buffer lives in one static
// device array of fixed size, so the call never needs cudaMalloc / cudaFree.
//
// Who needs this: code that may not allocate device memory at call time, e.g. a host
// framework whose caching allocator owns all device memory, a latency-critical loop where
// cudaMalloc / cudaFree would synchronize the device, or a service that must not be able
// to fail with out-of-memory in the middle of a request.
//
// Limits: n_vertices <= kNoAllocMaxVertices and n_entries <= kNoAllocMaxEntries, int32
// offsets. The array (about 7.4 MB) is held by every GPU that loads the library until the
// process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "capi_internal.h"
#include "gbfs.h"
#include "kernels.h"

namespace gbfs {
extern thread_local std::string t_last_error;
namespace {

constexpr int64_t kNoAllocMaxVertices = int64_t(1) << 18;  // 262,144
constexpr int64_t kNoAllocMaxEntries = int64_t(1) << 22;   // 4,194,304
constexpr int64_t kChunkCap = kNoAllocMaxEntries / kChunk + 2;

// Byte layout of the scratch array (each piece 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffBitmap = 0;
constexpr size_t kOffV0 = align256(kOffBitmap + sizeof(uint32_t) * (kNoAllocMaxVertices / 32));
constexpr size_t kVecBytes = align256(sizeof(int32_t) * kNoAllocMaxVertices);
constexpr size_t kOffV1 = kOffV0 + kVecBytes;
constexpr size_t kOffCum0 = kOffV1 + kVecBytes;
constexpr size_t kOffCum1 = kOffCum0 + kVecBytes;
constexpr size_t kOffBase0 = kOffCum1 + kVecBytes;
constexpr size_t kOffBase1 = kOffBase0 + kVecBytes;
constexpr size_t kOffChunk0 = kOffBase1 + kVecBytes;
constexpr size_t kChunkBytes = align256(sizeof(TileDesc<int32_t>) * kChunkCap);
constexpr size_t kOffChunk1 = kOffChunk0 + kChunkBytes;
constexpr size_t kOffCtl = kOffChunk1 + kChunkBytes;
constexpr size_t kOffCheck = kOffCtl + align256(sizeof(Ctl));
constexpr size_t kScratchBytes = kOffCheck + 256;

// The scratch itself. Host code must not use this name as an address (it is a host-side
// stand-in there); it takes the device address from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;                       // one call at a time in this process
unsigned char* g_scratch_dev[kMaxDevices] = {};  // device address of the array, per device

// Well-formed offsets: off[0] == 0, non-decreasing, off[n] == nnz. Any violation sets *bad.
__global__ void k_check_offsets(const int32_t* __restrict__ off, int64_t n, int64_t nnz, unsigned* bad) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = tid; v < n; v += stride)
    if (off[v + 1] < off[v]) atomicOr(bad, 1u);
  if (tid == 0 && (off[0] != 0 || (int64_t)off[n] != nnz)) atomicOr(bad, 1u);
}

// Device (or managed) memory, as the kernels read and write these arrays directly.
bool on_device(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// After a failed launch, earlier work of this call may still be running on the shared
// array: wait for it before the lock is released (its own status is not reported).
bfs_status settle(cudaStream_t cs, bfs_status s) {
  cudaStreamSynchronize(cs);
  cudaGetLastError();
  return s;
}

// Once per device, with that device current: look up the array's device address.
bfs_status scratch_for_device(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(BFS_ERR_CUDA, "device ordinal beyond the supported range");
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_scratch_dev[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_dev[dev];
  return BFS_OK;
}

}  // namespace
}  // namespace gbfs

using namespace gbfs;

extern "C" GBFS_API bfs_status bfs_run_noalloc(const int32_t* row_offsets, const int32_t* cols, int64_t n_vertices,
                                               int64_t n_entries, int32_t root, int32_t* levels, int32_t* parents,
                                               void* stream) {
  t_last_error.clear();
  if (!row_offsets || (n_entries > 0 && !cols) || !levels || !parents)
    return fail(BFS_ERR_INVALID_ARG, "NULL pointer argument");
  if (n_vertices < 1 || n_vertices > kNoAllocMaxVertices)
    return fail(BFS_ERR_INVALID_ARG, "bfs_run_noalloc: n_vertices must be in [1, " +
                                         std::to_string(kNoAllocMaxVertices) + "] (size of the static scratch)");
  if (n_entries < 0 || n_entries > kNoAllocMaxEntries)
    return fail(BFS_ERR_INVALID_ARG, "bfs_run_noalloc: n_entries must be in [0, " +
                                         std::to_string(kNoAllocMaxEntries) + "] (size of the static scratch)");
  if (root < 0 || root >= n_vertices) return fail(BFS_ERR_INVALID_ARG, "root outside [0, n)");
  if (!on_device(row_offsets) || (n_entries > 0 && !on_device(cols)) || !on_device(levels) || !on_device(parents))
    return fail(BFS_ERR_INVALID_ARG, "bfs_run_noalloc: row_offsets, cols, levels and parents must be device memory");

  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  unsigned char* s = nullptr;
  bfs_status st = scratch_for_device(dev, &s);
  if (st != BFS_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);

  GraphDev g;
  g.device = dev;
  if ((e = cudaDeviceGetAttribute(&g.num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess || g.num_sms < 1)
    return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidValue, "cudaDeviceGetAttribute(SM count)");
  g.n = n_vertices;
  g.nnz = n_entries;
  g.off64 = false;
  g.off = const_cast<int32_t*>(row_offsets);
  g.cols = const_cast<int32_t*>(cols);
  int count_bits = 0;
  for (uint64_t x = (uint64_t)n_vertices; x; x >>= 1) ++count_bits;
  g.pk.shift = 64 - count_bits;
  g.pk.mask = (1ull << g.pk.shift) - 1;

  SingleWs ws;
  ws.bitmap = reinterpret_cast<uint32_t*>(s + kOffBitmap);
  ws.v[0] = reinterpret_cast<int32_t*>(s + kOffV0);
  ws.v[1] = reinterpret_cast<int32_t*>(s + kOffV1);
  ws.cum[0] = s + kOffCum0;
  ws.cum[1] = s + kOffCum1;
  ws.base[0] = s + kOffBase0;
  ws.base[1] = s + kOffBase1;
  ws.chunk[0] = s + kOffChunk0;
  ws.chunk[1] = s + kOffChunk1;
  ws.chunk_cap = kChunkCap;
  ws.ctl = reinterpret_cast<Ctl*>(s + kOffCtl);
  unsigned* check = reinterpret_cast<unsigned*>(s + kOffCheck);

  // The array keeps the previous call's contents: clear the check word here; the init
  // kernel below resets the bitmap, the control block and the first frontier.
  if ((e = cudaMemsetAsync(check, 0, sizeof(unsigned), cs)) != cudaSuccess) return cuda_fail(e, "memset");
  k_check_offsets<<<g.num_sms * 4, 256, 0, cs>>>(row_offsets, n_vertices, n_entries, check);
  unsigned bad = 0;
  if ((e = cudaMemcpyAsync(&bad, check, sizeof(unsigned), cudaMemcpyDeviceToHost, cs)) != cudaSuccess ||
      (e = cudaStreamSynchronize(cs)) != cudaSuccess)
    return settle(cs, cuda_fail(e, "offsets check"));
  if (bad) return fail(BFS_ERR_INVALID_GRAPH, "row_offsets is not a well-formed CSR offsets array");

  launch_init_single<int32_t>(g, root, levels, parents, ws, cs);
  if ((e = cudaGetLastError()) != cudaSuccess) return settle(cs, cuda_fail(e, "init kernel"));
  ExpandArgs<int32_t> a{};
  a.off = row_offsets;
  a.cols = cols;
  a.bitmap = ws.bitmap;
  a.n = n_vertices;
  a.fr[0] = ws.fr<int32_t>(0);
  a.fr[1] = ws.fr<int32_t>(1);
  a.chunk[0] = ws.desc<int32_t>(0);
  a.chunk[1] = ws.desc<int32_t>(1);
  a.ctl = ws.ctl;
  a.pk = g.pk;
  a.use_cond = 0;
  a.probe_mode = 1;
  const int grid = expand_grid<int32_t>(kDefaultShape, g.num_sms);
  Ctl c{};
  for (int64_t it = 0; it <= n_vertices; ++it) {
    if ((e = launch_expand<int32_t>(kDefaultShape, a, grid, cs)) != cudaSuccess)
      return settle(cs, cuda_fail(e, "expand kernel"));
    if ((e = cudaMemcpyAsync(&c, ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, cs)) != cudaSuccess ||
        (e = cudaStreamSynchronize(cs)) != cudaSuccess)
      return settle(cs, cuda_fail(e, "level flag"));
    if (c.error & kErrColumnRange) return fail(BFS_ERR_INVALID_GRAPH, "a column id outside [0, n) was met");
    if (!c.cont) break;
  }
  return BFS_OK;
}
