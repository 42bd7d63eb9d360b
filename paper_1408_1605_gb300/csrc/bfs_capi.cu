// C ABI of the gbfs library: graph upload and checks, single-source search, one-level
// expansion. The level loop of a search stays on the device: one CUDA graph per graph
// handle holds a conditional WHILE node whose body is the expansion kernel; the kernel's
// last CTA sets the condition to "next frontier non-empty" (the termination test of Algorithm 2,
// without the per-level host round trip of the original design, Sec. 3.4).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "batch.h"
#include "capi_internal.h"
#include "gbfs.h"
#include "kernels.h"

namespace gbfs {

thread_local std::string t_last_error;

bfs_status fail(bfs_status s, const std::string& msg) {
  t_last_error = msg;
  return s;
}

void clear_last_error() { t_last_error.clear(); }

bfs_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky-free error so later calls are not affected
  return fail(e == cudaErrorMemoryAllocation ? BFS_ERR_OOM : BFS_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

static int bits_for(uint64_t x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

template <typename T>
static bfs_status device_alloc(T** p, size_t count, const char* what) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, what);
  *p = static_cast<T*>(q);
  return BFS_OK;
}

static void free_single_ws(SingleWs& ws) {
  cudaFree(ws.bitmap);
  for (int i = 0; i < 2; ++i) {
    cudaFree(ws.v[i]);
    cudaFree(ws.cum[i]);
    cudaFree(ws.base[i]);
    cudaFree(ws.chunk[i]);
  }
  cudaFree(ws.ctl);
  cudaFree(ws.scan_partial);
  cudaFree(ws.host_levels);
  cudaFree(ws.host_parents);
  for (int i = 0; i < 3; ++i) cudaFree(ws.fbm[i]);
  cudaFree(ws.pctl);
  if (ws.pctl_host) cudaFreeHost(ws.pctl_host);
  if (ws.ctl_host) cudaFreeHost(ws.ctl_host);
  if (ws.ev0) cudaEventDestroy(ws.ev0);
  if (ws.ev1) cudaEventDestroy(ws.ev1);
  if (ws.ev_mid) cudaEventDestroy(ws.ev_mid);
  ws = SingleWs{};
}

bfs_status ensure_single_ws(bfs_graph_s* G) {
  SingleWs& ws = G->ws;
  if (ws.ready) return BFS_OK;
  const GraphDev& g = G->g;
  const size_t osz = g.off64 ? 8 : 4;
  bfs_status s;
  if ((s = device_alloc(&ws.bitmap, (size_t)(g.n + 31) / 32, "bitmap"))) goto bad;
  ws.chunk_cap = g.nnz / kChunk + 2;
  for (int i = 0; i < 2; ++i) {
    if ((s = device_alloc(&ws.v[i], (size_t)g.n, "frontier"))) goto bad;
    if ((s = device_alloc(reinterpret_cast<char**>(&ws.cum[i]), (size_t)g.n * osz, "frontier scan"))) goto bad;
    if ((s = device_alloc(reinterpret_cast<char**>(&ws.base[i]), (size_t)g.n * osz, "frontier base"))) goto bad;
    // tile descriptors: 16 bytes for either offset width
    static_assert(sizeof(TileDesc<int32_t>) == 16 && sizeof(TileDesc<int64_t>) == 16, "descriptor size");
    if ((s = device_alloc(reinterpret_cast<char**>(&ws.chunk[i]), (size_t)ws.chunk_cap * 16, "chunk index"))) goto bad;
  }
  if ((s = device_alloc(&ws.ctl, 1, "control block"))) goto bad;
  if ((s = device_alloc(&ws.pctl, 1, "control block"))) goto bad;
  for (int i = 0; i < 3; ++i)
    if ((s = device_alloc(&ws.fbm[i], (size_t)(g.n + 31) / 32, "frontier bitmap"))) goto bad;
  ws.scan_parts = g.num_sms * 4;
  if ((s = device_alloc(reinterpret_cast<char**>(&ws.scan_partial), (size_t)ws.scan_parts * 8, "scan partials")))
    goto bad;
  {
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&ws.ctl_host), sizeof(Ctl), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&ws.pctl_host), sizeof(PCtl), cudaHostAllocDefault);
    if (e != cudaSuccess) {
      s = cuda_fail(e, "pinned control mirror");
      goto bad;
    }
    if ((e = cudaEventCreate(&ws.ev0)) != cudaSuccess || (e = cudaEventCreate(&ws.ev1)) != cudaSuccess ||
        (e = cudaEventCreate(&ws.ev_mid)) != cudaSuccess) {
      s = cuda_fail(e, "events");
      goto bad;
    }
    if ((e = cudaMemset(ws.ctl, 0, sizeof(Ctl))) != cudaSuccess) {
      s = cuda_fail(e, "control init");
      goto bad;
    }
  }
  ws.ready = true;
  return BFS_OK;
bad:
  free_single_ws(ws);
  return s;
}

template <typename OffT>
ExpandArgs<OffT> make_args(const bfs_graph_s* G, uint32_t* bitmap) {
  const GraphDev& g = G->g;
  const SingleWs& ws = G->ws;
  ExpandArgs<OffT> a{};
  a.off = reinterpret_cast<const OffT*>(g.off);
  a.cols = g.cols;
  a.bitmap = bitmap;
  a.n = g.n;
  a.fr[0] = ws.fr<OffT>(0);
  a.fr[1] = ws.fr<OffT>(1);
  a.chunk[0] = ws.desc<OffT>(0);
  a.chunk[1] = ws.desc<OffT>(1);
  a.ctl = ws.ctl;
  a.pk = g.pk;
  a.cond = 0;
  a.use_cond = 0;
  a.probe_mode = G->probe_mode;
  a.old_id = g.old_id;
  a.fbm[0] = a.fbm[1] = nullptr;
  a.list_cap = -1;
  if (G->frontier_mode != BFS_FRONTIER_LIST) {  // next-frontier bitmaps by level parity
    a.fbm[0] = ws.fbm[0];
    a.fbm[1] = ws.fbm[1];
    a.list_cap = frontier_list_cap(G->frontier_mode, g.n);
  }
  return a;
}

// Builds the device-resident level loop: graph = WHILE(cond) { expand }.
template <typename OffT>
static bfs_status build_loop_graph(bfs_graph_s* G, cudaStream_t st) {
  cudaError_t e;
  cudaGraph_t graph = nullptr;
  if ((e = cudaGraphCreate(&graph, 0)) != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
  cudaGraphConditionalHandle handle;
  if ((e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault)) != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(e, "cudaGraphConditionalHandleCreate");
  }
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp)) != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(e, "cudaGraphAddNode(conditional)");
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  ExpandArgs<OffT> a = make_args<OffT>(G, G->ws.bitmap);
  a.cond = handle;
  a.use_cond = 1;
  // Capture the expansion launch into the body graph, on a private stream: the caller's
  // stream may be the legacy default stream, which cannot capture.
  (void)st;
  cudaStream_t cs = nullptr;
  if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(e, "cudaStreamCreate");
  }
  if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess) {
    cudaStreamDestroy(cs);
    cudaGraphDestroy(graph);
    return cuda_fail(e, "cudaStreamBeginCaptureToGraph");
  }
  cudaError_t le = launch_expand<OffT>(G->shape, a, G->grid, cs);
  if (a.fbm[0]) launch_unpack_level<OffT>(G->g, a, cs);  // frontier-bitmap mode
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(cs, &captured);
  cudaStreamDestroy(cs);
  if (le != cudaSuccess || e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(le != cudaSuccess ? le : e, "capture of the expansion kernel");
  }
  cudaGraphExec_t exec = nullptr;
  if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  G->loop_graph = graph;
  G->loop_exec = exec;
  return BFS_OK;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename OffT>
static bfs_status run_single(bfs_graph_s* G, int32_t root, int32_t* levels, int32_t* parents, cudaStream_t st,
                             bfs_stats* stats) {
  SingleWs& ws = G->ws;
  cudaError_t e;
  const bool host_out = !is_device_ptr(levels) || !is_device_ptr(parents);
  int32_t* dl = levels;
  int32_t* dp = parents;
  if (host_out) {
    if (!ws.host_levels) {
      bfs_status s;
      if ((s = device_alloc(&ws.host_levels, (size_t)G->g.n, "levels staging"))) return s;
      if ((s = device_alloc(&ws.host_parents, (size_t)G->g.n, "parents staging"))) return s;
    }
    dl = ws.host_levels;
    dp = ws.host_parents;
  }
  if (G->last_done) cudaStreamWaitEvent(st, G->last_done, 0);  // workspace reuse across streams
  if ((e = cudaEventRecord(ws.ev0, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  const bool persistent = G->loop_mode == BFS_LOOP_PERSISTENT;
  if (persistent)
    launch_init_persist<OffT>(G->g, root, dl, dp, ws, st);
  else
    launch_init_single<OffT>(G->g, root, dl, dp, ws, st, G->frontier_mode != BFS_FRONTIER_LIST);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "init kernel");
  if ((e = cudaEventRecord(ws.ev_mid, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  if (persistent) {
    PersistArgs<OffT> pa{};
    pa.off = reinterpret_cast<const OffT*>(G->g.off);
    pa.cols = G->g.cols;
    pa.bitmap = ws.bitmap;
    for (int i = 0; i < 3; ++i) pa.fbm[i] = ws.fbm[i];
    pa.n = G->g.n;
    pa.nnz = G->g.nnz;
    pa.fr[0] = ws.fr<OffT>(0);
    pa.fr[1] = ws.fr<OffT>(1);
    pa.chunk[0] = ws.desc<OffT>(0);
    pa.chunk[1] = ws.desc<OffT>(1);
    pa.ctl = ws.pctl;
    pa.pk = G->g.pk;
    pa.levels = dl;
    pa.parents = dp;
    pa.alpha = G->alpha;
    pa.beta = G->beta;
    pa.allow_bottom_up = G->bottom_up;
    pa.probe_mode = G->probe_mode;
    pa.spin_limit = G->wait_limit;
    pa.old_id = G->g.old_id;
    pa.bitmap_mode = G->frontier_mode != BFS_FRONTIER_LIST;
    pa.list_cap = frontier_list_cap(G->frontier_mode, G->g.n);
    int& pg = G->pgrid[G->bottom_up ? 1 : 0];
    if (!pg) {
      pg = persistent_grid<OffT>(G->shape, G->g.num_sms, G->bottom_up != 0);
      if (G->persist_ctas > 0) pg = std::min(pg, G->persist_ctas * G->g.num_sms);
    }
    if ((e = launch_persistent<OffT>(G->shape, pa, pg, st)) != cudaSuccess)
      return cuda_fail(e, "persistent search kernel");
  } else if (G->host_loop) {
    ExpandArgs<OffT> a = make_args<OffT>(G, ws.bitmap);
    for (int64_t it = 0; it <= G->g.n; ++it) {
      if ((e = launch_expand<OffT>(G->shape, a, G->grid, st)) != cudaSuccess) return cuda_fail(e, "expand kernel");
      if (a.fbm[0]) launch_unpack_level<OffT>(G->g, a, st);  // frontier-bitmap mode
      if ((e = cudaMemcpyAsync(&ws.ctl_host->cont, &ws.ctl->cont, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess)
        return cuda_fail(e, "level flag copy");
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "level sync");
      if (!ws.ctl_host->cont) break;
    }
  } else {
    if (!G->loop_exec) {
      bfs_status s = build_loop_graph<OffT>(G, st);
      if (s != BFS_OK) return s;
    }
    if ((e = cudaGraphLaunch(G->loop_exec, st)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  }
  if ((e = cudaEventRecord(ws.ev1, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  if (host_out) {
    const size_t bytes = (size_t)G->g.n * sizeof(int32_t);
    if ((e = cudaMemcpyAsync(levels, dl, bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "levels copy");
    if ((e = cudaMemcpyAsync(parents, dp, bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "parents copy");
  }
  if (persistent) {
    if ((e = cudaMemcpyAsync(ws.pctl_host, ws.pctl, sizeof(PCtl), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "control copy");
  } else if ((e = cudaMemcpyAsync(ws.ctl_host, ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st)) != cudaSuccess) {
    return cuda_fail(e, "control copy");
  }
  if (!G->last_done && (e = cudaEventCreateWithFlags(&G->last_done, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "cudaEventCreate");
  cudaEventRecord(G->last_done, st);
  if (stats || host_out) {
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "search");
    const unsigned error = persistent ? ws.pctl_host->error : ws.ctl_host->error;
    if (error & kErrColumnRange) return fail(BFS_ERR_INVALID_GRAPH, "a column id outside [0, n) was met");
    if (error & kErrTimeout) return fail(BFS_ERR_TIMEOUT, "a grid barrier wait expired");
    if (stats) {
      float ms = 0.f, loop_ms = 0.f;
      cudaEventElapsedTime(&ms, ws.ev0, ws.ev1);
      cudaEventElapsedTime(&loop_ms, ws.ev_mid, ws.ev1);
      const int depth = persistent ? ws.pctl_host->depth : ws.ctl_host->depth;
      const long long reached = persistent ? ws.pctl_host->reached : ws.ctl_host->reached;
      const long long edges2 = persistent ? ws.pctl_host->edges2 : ws.ctl_host->edges2;
      stats->depth = depth;
      stats->bottom_up_levels = persistent ? ws.pctl_host->steps_bottom_up : 0;
      G->last_unpacked = persistent ? ws.pctl_host->unpacked_levels : -1;
      stats->vertices_reached = reached;
      stats->edges_traversed = edges2 / 2;
      stats->device_ms = ms;
      stats->expand_ms = loop_ms;
    }
  }
  return BFS_OK;
}

template <typename OffT>
static bfs_status expand_one(bfs_graph_s* G, const int32_t* front, int64_t nf, int32_t level, uint32_t* bitmap,
                             int32_t* levels, int32_t* parents, int32_t* next, int64_t* next_count,
                             cudaStream_t st) {
  SingleWs& ws = G->ws;
  cudaError_t e;
  if (G->last_done) cudaStreamWaitEvent(st, G->last_done, 0);
  launch_scan_frontier<OffT>(G->g, front, nf, level, levels, parents, ws, st);
  ExpandArgs<OffT> a = make_args<OffT>(G, bitmap);
  a.fr[level & 1].v = next;  // the next frontier of `level` is written at parity level & 1
  if ((e = launch_expand<OffT>(G->shape, a, G->grid, st)) != cudaSuccess) return cuda_fail(e, "expand kernel");
  launch_write_count(ws.ctl, G->g.pk, next_count, st);
  if ((e = cudaMemcpyAsync(ws.ctl_host, ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "control copy");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "expand");
  const Ctl& c = *ws.ctl_host;
  if (c.error & kErrFrontierRange) return fail(BFS_ERR_INVALID_ARG, "a frontier vertex is outside [0, n)");
  if (c.error & kErrCounterOverflow) return fail(BFS_ERR_INVALID_ARG, "frontier edge total exceeds capacity");
  if (c.error & kErrColumnRange) return fail(BFS_ERR_INVALID_GRAPH, "a column id outside [0, n) was met");
  return BFS_OK;
}

// One level producing its next frontier as a bitmap only (the list cap is -1: no appends),
// then, if `next` is given, the warp-centric unpack of that bitmap into a list.
template <typename OffT>
static bfs_status expand_bitmap_one(bfs_graph_s* G, const int32_t* front, int64_t nf, int32_t level, uint32_t* bitmap,
                                    int32_t* levels, int32_t* parents, uint32_t* next_bitmap, int32_t* next,
                                    int64_t* next_count, cudaStream_t st) {
  SingleWs& ws = G->ws;
  cudaError_t e;
  if (G->last_done) cudaStreamWaitEvent(st, G->last_done, 0);
  const size_t words = (size_t)(G->g.n + 31) / 32;
  if ((e = cudaMemsetAsync(next_bitmap, 0, words * sizeof(uint32_t), st)) != cudaSuccess)
    return cuda_fail(e, "memset");
  if (nf > 0) {
    launch_scan_frontier<OffT>(G->g, front, nf, level, levels, parents, ws, st);
    ExpandArgs<OffT> a = make_args<OffT>(G, bitmap);
    const int nxt = level & 1;  // the expansion of `level` writes parity level & 1
    a.fbm[0] = a.fbm[1] = nullptr;
    a.fbm[nxt] = next_bitmap;
    a.list_cap = -1;  // bitmap only
    if ((e = cudaMemsetAsync(&ws.ctl->dropped, 0, sizeof(unsigned), st)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = launch_expand<OffT>(G->shape, a, G->grid, st)) != cudaSuccess) return cuda_fail(e, "expand kernel");
  }
  launch_write_count(ws.ctl, G->g.pk, next_count, st);
  if (nf == 0 && (e = cudaMemsetAsync(next_count, 0, sizeof(int64_t), st)) != cudaSuccess) return cuda_fail(e, "memset");
  if ((e = cudaMemcpyAsync(ws.ctl_host, ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "control copy");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "expand");
  const Ctl& c = *ws.ctl_host;
  if (nf > 0) {
    if (c.error & kErrFrontierRange) return fail(BFS_ERR_INVALID_ARG, "a frontier vertex is outside [0, n)");
    if (c.error & kErrCounterOverflow) return fail(BFS_ERR_INVALID_ARG, "frontier edge total exceeds capacity");
    if (c.error & kErrColumnRange) return fail(BFS_ERR_INVALID_GRAPH, "a column id outside [0, n) was met");
  }
  if (next && (e = unpack_bitmap_to_list<OffT>(G->g, ws, level & 1, next_bitmap, next, next_count, st)) != cudaSuccess)
    return cuda_fail(e, "bitmap unpack");
  if (!G->last_done && (e = cudaEventCreateWithFlags(&G->last_done, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "cudaEventCreate");
  cudaEventRecord(G->last_done, st);
  return BFS_OK;
}

// Switches the single-source expansion shape; the level-loop graph is rebuilt on next use.
void set_single_shape(bfs_graph_s* G, int shape) {
  G->shape = shape;
  G->pgrid[0] = G->pgrid[1] = 0;
  G->grid = G->g.off64 ? expand_grid<int64_t>(shape, G->g.num_sms) : expand_grid<int32_t>(shape, G->g.num_sms);
  if (G->loop_exec) cudaGraphExecDestroy(G->loop_exec);
  if (G->loop_graph) cudaGraphDestroy(G->loop_graph);
  G->loop_exec = nullptr;
  G->loop_graph = nullptr;
}

}  // namespace gbfs

using namespace gbfs;

// ------------------------------------------------------------------------------------------
// Graph creation and checks

template <typename InT>
static bfs_status check_offsets(const InT* off, int64_t n, int64_t nnz, int64_t* max_deg) {
  if (off[0] != 0) return fail(BFS_ERR_INVALID_GRAPH, "row_offsets[0] != 0");
  int64_t md = 0;
  for (int64_t v = 0; v < n; ++v) {
    const int64_t d = (int64_t)off[v + 1] - (int64_t)off[v];
    if (d < 0) return fail(BFS_ERR_INVALID_GRAPH, "row_offsets decreases at vertex " + std::to_string(v));
    md = std::max(md, d);
  }
  if ((int64_t)off[n] != nnz) return fail(BFS_ERR_INVALID_GRAPH, "row_offsets[n] != n_entries");
  *max_deg = md;
  return BFS_OK;
}

template <typename InT>
static bfs_status validate_full(const InT* off, const int32_t* cols, int64_t n, int64_t nnz) {
  for (int64_t i = 0; i < nnz; ++i)
    if (cols[i] < 0 || cols[i] >= n)
      return fail(BFS_ERR_INVALID_GRAPH, "column id out of range at entry " + std::to_string(i));
  // symmetry: the multiset of (u, v) equals that of (v, u)
  std::vector<uint64_t> a((size_t)nnz), b((size_t)nnz);
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = (int64_t)off[u]; e < (int64_t)off[u + 1]; ++e) {
      a[(size_t)e] = (uint64_t)u * (uint64_t)n + (uint64_t)cols[e];
      b[(size_t)e] = (uint64_t)cols[e] * (uint64_t)n + (uint64_t)u;
    }
  std::sort(a.begin(), a.end());
  std::sort(b.begin(), b.end());
  if (a != b) return fail(BFS_ERR_INVALID_GRAPH, "the CSR is not symmetric");
  return BFS_OK;
}

template <typename InT, typename OffT>
static void convert_offsets(const InT* in, OffT* out, int64_t n) {
  for (int64_t i = 0; i <= n; ++i) out[i] = (OffT)in[i];
}

extern "C" {

GBFS_API const char* bfs_last_error(void) { return t_last_error.c_str(); }

GBFS_API const char* bfs_version(void) { return "gbfs 0.1 (sm_103a)"; }

GBFS_API bfs_status bfs_graph_create(const void* row_offsets, const int32_t* cols, int64_t n_vertices,
                                     int64_t n_entries, uint32_t flags, void* stream, bfs_graph_t* out) {
  t_last_error.clear();
  if (!out) return fail(BFS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!row_offsets) return fail(BFS_ERR_INVALID_ARG, "row_offsets is NULL");
  if (n_entries > 0 && !cols) return fail(BFS_ERR_INVALID_ARG, "cols is NULL");
  if (n_vertices < 1 || n_vertices > INT32_MAX) return fail(BFS_ERR_INVALID_ARG, "n_vertices outside [1, 2^31-1]");
  if (n_entries < 0) return fail(BFS_ERR_INVALID_ARG, "n_entries < 0");
  const uint32_t known =
      BFS_HOST_PTRS | BFS_DEVICE_PTRS | BFS_OFFSETS_INT32 | BFS_OFFSETS_INT64 | BFS_VALIDATE | BFS_RELABEL_DEGREE |
                         BFS_KEEP_INT64;
  if (flags & ~known) return fail(BFS_ERR_INVALID_ARG, "unknown flag bits");
  if ((flags & BFS_HOST_PTRS) && (flags & BFS_DEVICE_PTRS))
    return fail(BFS_ERR_INVALID_ARG, "BFS_HOST_PTRS and BFS_DEVICE_PTRS both set");
  if ((flags & BFS_OFFSETS_INT32) && (flags & BFS_OFFSETS_INT64))
    return fail(BFS_ERR_INVALID_ARG, "BFS_OFFSETS_INT32 and BFS_OFFSETS_INT64 both set");
  const bool in64 = flags & BFS_OFFSETS_INT64;
  const bool dev_in = flags & BFS_DEVICE_PTRS;
  if (!in64 && n_entries > INT32_MAX) return fail(BFS_ERR_INVALID_ARG, "int32 offsets cannot hold n_entries");
  const int64_t n = n_vertices, nnz = n_entries;
  const size_t isz = in64 ? 8 : 4;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;

  // Host view of the offsets (copied back when they live on the device).
  std::vector<unsigned char> off_host_copy;
  const void* off_h = row_offsets;
  if (dev_in) {
    off_host_copy.resize((size_t)(n + 1) * isz);
    if ((e = cudaMemcpy(off_host_copy.data(), row_offsets, off_host_copy.size(), cudaMemcpyDeviceToHost)) !=
        cudaSuccess)
      return cuda_fail(e, "offsets read-back");
    off_h = off_host_copy.data();
  }
  int64_t max_deg = 0;
  bfs_status s = in64 ? check_offsets(static_cast<const int64_t*>(off_h), n, nnz, &max_deg)
                      : check_offsets(static_cast<const int32_t*>(off_h), n, nnz, &max_deg);
  if (s != BFS_OK) return s;
  if (max_deg > INT32_MAX) return fail(BFS_ERR_INVALID_GRAPH, "a vertex has 2^31 or more entries");
  if (flags & BFS_VALIDATE) {
    std::vector<int32_t> cols_copy;
    const int32_t* cols_h = cols;
    if (dev_in && nnz > 0) {
      cols_copy.resize((size_t)nnz);
      if ((e = cudaMemcpy(cols_copy.data(), cols, (size_t)nnz * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "cols read-back");
      cols_h = cols_copy.data();
    }
    s = in64 ? validate_full(static_cast<const int64_t*>(off_h), cols_h, n, nnz)
             : validate_full(static_cast<const int32_t*>(off_h), cols_h, n, nnz);
    if (s != BFS_OK) return s;
  }

  auto* G = new (std::nothrow) bfs_graph_s();
  if (!G) return fail(BFS_ERR_OOM, "host allocation");
  GraphDev& g = G->g;
  if ((e = cudaGetDevice(&g.device)) != cudaSuccess) {
    delete G;
    return cuda_fail(e, "cudaGetDevice");
  }
  cudaDeviceGetAttribute(&g.num_sms, cudaDevAttrMultiProcessorCount, g.device);
  g.n = n;
  g.nnz = nnz;
  g.off64 = nnz > INT32_MAX || (flags & BFS_KEEP_INT64) != 0;
  const int count_bits = bits_for((uint64_t)n);
  g.pk.shift = 64 - count_bits;
  g.pk.mask = (g.pk.shift >= 64) ? ~0ull : ((1ull << g.pk.shift) - 1);
  if ((uint64_t)nnz > g.pk.mask) {
    delete G;
    return fail(BFS_ERR_INVALID_GRAPH, "graph too large for the packed frontier counter");
  }
  const size_t osz = g.off64 ? 8 : 4;
  if ((e = cudaMalloc(&g.off, (size_t)(n + 1) * osz)) != cudaSuccess ||
      (e = cudaMalloc(reinterpret_cast<void**>(&g.cols), (size_t)std::max<int64_t>(nnz, 1) * 4)) != cudaSuccess) {
    cudaFree(g.off);
    delete G;
    return cuda_fail(e, "graph allocation");
  }
  // offsets: direct copy when the width matches, else a host-side conversion
  if ((osz == isz)) {
    e = cudaMemcpyAsync(g.off, row_offsets, (size_t)(n + 1) * osz,
                        dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
  } else {
    std::vector<unsigned char> conv((size_t)(n + 1) * osz);
    if (g.off64)
      convert_offsets(static_cast<const int32_t*>(off_h), reinterpret_cast<int64_t*>(conv.data()), n);
    else
      convert_offsets(static_cast<const int64_t*>(off_h), reinterpret_cast<int32_t*>(conv.data()), n);
    e = cudaMemcpyAsync(g.off, conv.data(), conv.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e == cudaSuccess && nnz > 0)
    e = cudaMemcpyAsync(g.cols, cols, (size_t)nnz * 4, dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(g.off);
    cudaFree(g.cols);
    delete G;
    return cuda_fail(e, "graph upload");
  }
  const bool relabel = (flags & BFS_RELABEL_DEGREE) != 0;
  if (relabel && (e = relabel_by_degree(g, st)) != cudaSuccess) {
    cudaFree(g.off);
    cudaFree(g.cols);
    delete G;
    return e == cudaErrorMemoryAllocation ? fail(BFS_ERR_OOM, "relabelling: device allocation")
                                          : cuda_fail(e, "relabelling");
  }
  // Bitmap pre-check: relabelled graphs concentrate the probes on the hub words, which L1
  // serves best; otherwise the L2-only load sees claims made during the level sooner.
  G->probe_mode = g.new_id ? 0 : 1;
  G->loop_mode = BFS_LOOP_GRAPH;
  G->host_loop = false;
  G->bottom_up = 0;
  G->shape = kDefaultShape;
  G->grid = g.off64 ? expand_grid<int64_t>(G->shape, g.num_sms) : expand_grid<int32_t>(G->shape, g.num_sms);
  G->batch_shape = kDefaultBatchShape;
  *out = G;
  return BFS_OK;
}

GBFS_API bfs_status bfs_graph_destroy(bfs_graph_t G) {
  if (!G) return BFS_OK;
  {
    std::lock_guard<std::mutex> lock(G->mu);
    cudaSetDevice(G->g.device);
    if (G->last_done) cudaEventSynchronize(G->last_done);
    destroy_batch_state(G);
    if (G->loop_exec) cudaGraphExecDestroy(G->loop_exec);
    if (G->loop_graph) cudaGraphDestroy(G->loop_graph);
    if (G->last_done) cudaEventDestroy(G->last_done);
    free_single_ws(G->ws);
    cudaFree(G->g.off);
    cudaFree(G->g.cols);
    cudaFree(G->g.new_id);
    cudaFree(G->g.old_id);
  }
  delete G;
  return BFS_OK;
}

GBFS_API bfs_status bfs_graph_set_option(bfs_graph_t G, int option, int64_t value) {
  clear_last_error();
  if (!G) return fail(BFS_ERR_INVALID_ARG, "graph is NULL");
  std::lock_guard<std::mutex> lock(G->mu);
  switch (option) {
    case BFS_OPT_LOOP:
      if (value < BFS_LOOP_PERSISTENT || value > BFS_LOOP_HOST) return fail(BFS_ERR_INVALID_ARG, "unknown loop mode");
      G->loop_mode = (int)value;
      G->host_loop = value == BFS_LOOP_HOST;
      return BFS_OK;
    case BFS_OPT_BOTTOM_UP:
      G->bottom_up = value != 0;
      set_batch_shape(G, G->batch_shape);  // the captured wave loop holds the policy
      return BFS_OK;
    case BFS_OPT_ALPHA:
    case BFS_OPT_BETA:
      if (value < 1 || value > (1 << 20)) return fail(BFS_ERR_INVALID_ARG, "alpha/beta outside [1, 2^20]");
      (option == BFS_OPT_ALPHA ? G->alpha : G->beta) = (int)value;
      set_batch_shape(G, G->batch_shape);
      return BFS_OK;
    case BFS_OPT_WAIT_LIMIT:
      if (value < 0 || value > (1ll << 40)) return fail(BFS_ERR_INVALID_ARG, "wait limit outside [0, 2^40]");
      G->wait_limit = value;
      return BFS_OK;
    case BFS_OPT_PERSIST_CTAS:
      if (value < 0 || value > 64) return fail(BFS_ERR_INVALID_ARG, "CTAs per SM outside [0, 64]");
      if (G->persist_ctas != (int)value) {
        if (G->last_done) cudaEventSynchronize(G->last_done);
        G->persist_ctas = (int)value;
        G->pgrid[0] = G->pgrid[1] = 0;
      }
      return BFS_OK;
    case BFS_OPT_WAVE_DENSE_ROWS:
      if (value < -1 || value > (1ll << 40)) return fail(BFS_ERR_INVALID_ARG, "dense rows outside [-1, 2^40]");
      if (G->dense_rows != value) {
        if (G->last_done) cudaEventSynchronize(G->last_done);
        G->dense_rows = value;
        destroy_batch_state(G);  // the pool is sized when the wave state is next allocated
      }
      return BFS_OK;
    case BFS_OPT_FRONTIER:
      if (value < BFS_FRONTIER_LIST || value > BFS_FRONTIER_BITMAP) return fail(BFS_ERR_INVALID_ARG, "unknown frontier mode");
      if (G->frontier_mode != (int)value) {
        if (G->last_done) cudaEventSynchronize(G->last_done);
        G->frontier_mode = (int)value;
        set_single_shape(G, G->shape);  // the captured level loop holds the old mode
      }
      return BFS_OK;
    case BFS_OPT_PROBE:
      if (value < 0 || value > 1) return fail(BFS_ERR_INVALID_ARG, "probe mode outside [0, 1]");
      if (G->probe_mode != (int)value) {
        if (G->last_done) cudaEventSynchronize(G->last_done);
        G->probe_mode = (int)value;
        set_single_shape(G, G->shape);  // the captured level loop holds the old mode
      }
      return BFS_OK;
  }
  return fail(BFS_ERR_INVALID_ARG, "unknown option");
}

GBFS_API bfs_status bfs_graph_get_option(bfs_graph_t G, int option, int64_t* value) {
  clear_last_error();
  if (!G || !value) return fail(BFS_ERR_INVALID_ARG, "NULL argument");
  switch (option) {
    case BFS_OPT_LOOP: *value = G->loop_mode; return BFS_OK;
    case BFS_OPT_BOTTOM_UP: *value = G->bottom_up; return BFS_OK;
    case BFS_OPT_ALPHA: *value = G->alpha; return BFS_OK;
    case BFS_OPT_BETA: *value = G->beta; return BFS_OK;
    case BFS_OPT_WAIT_LIMIT: *value = G->wait_limit; return BFS_OK;
    case BFS_OPT_PROBE: *value = G->probe_mode; return BFS_OK;
    case BFS_OPT_PERSIST_CTAS: *value = G->persist_ctas; return BFS_OK;
    case BFS_OPT_RELABELED: *value = G->g.new_id != nullptr; return BFS_OK;
    case BFS_OPT_FRONTIER: *value = G->frontier_mode; return BFS_OK;
    case BFS_OPT_WAVE_DENSE_ROWS: *value = G->dense_rows; return BFS_OK;
    case BFS_OPT_UNPACKED_LEVELS: *value = G->last_unpacked; return BFS_OK;
    case BFS_OPT_WAVE_LEVELS: *value = batch_last_levels(G); return BFS_OK;
    case BFS_OPT_WAVE_OVERFLOW: *value = batch_last_overflow(G); return BFS_OK;
  }
  return fail(BFS_ERR_INVALID_ARG, "unknown option");
}

GBFS_API bfs_status bfs_level_profile(bfs_graph_t G, int cap, double* level_ms, int64_t* frontier,
                                      int32_t* bottom_up, int* n_levels) {
  clear_last_error();
  if (!G || !n_levels || cap < 0) return fail(BFS_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lock(G->mu);
  if (!G->ws.ready || !G->ws.pctl_host) return fail(BFS_ERR_NOT_FOUND, "no persistent search has run on this graph");
  if (G->last_done) cudaEventSynchronize(G->last_done);
  const PCtl& c = *G->ws.pctl_host;
  const int levels = std::min(std::max(c.depth, 0), kMaxLevelTimes);
  unsigned long long prev = c.start_ns;
  for (int i = 0; i < levels && i < cap; ++i) {
    if (level_ms) level_ms[i] = (double)(c.level_ns[i] - prev) * 1e-6;
    if (frontier) frontier[i] = c.level_nf[i];
    if (bottom_up) bottom_up[i] = c.level_bu[i];
    prev = c.level_ns[i];
  }
  *n_levels = levels;
  return BFS_OK;
}

GBFS_API bfs_status bfs_graph_info(bfs_graph_t G, int64_t* n_vertices, int64_t* n_entries) {
  if (!G) return fail(BFS_ERR_INVALID_ARG, "graph is NULL");
  if (n_vertices) *n_vertices = G->g.n;
  if (n_entries) *n_entries = G->g.nnz;
  return BFS_OK;
}

GBFS_API bfs_status bfs_run(bfs_graph_t G, int32_t root, int32_t* levels, int32_t* parents, void* stream,
                            bfs_stats* stats) {
  t_last_error.clear();
  if (!G) return fail(BFS_ERR_INVALID_ARG, "graph is NULL");
  if (!levels || !parents) return fail(BFS_ERR_INVALID_ARG, "levels/parents is NULL");
  if (root < 0 || root >= G->g.n) return fail(BFS_ERR_INVALID_ARG, "root outside [0, n)");
  std::lock_guard<std::mutex> lock(G->mu);
  cudaError_t e = cudaSetDevice(G->g.device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  bfs_status s = ensure_single_ws(G);
  if (s != BFS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return G->g.off64 ? run_single<int64_t>(G, root, levels, parents, st, stats)
                    : run_single<int32_t>(G, root, levels, parents, st, stats);
}

GBFS_API bfs_status bfs_expand_bitmap(bfs_graph_t G, const int32_t* frontier, int64_t n_frontier, int32_t level,
                                      uint32_t* bitmap, int32_t* levels, int32_t* parents, uint32_t* next_bitmap,
                                      int32_t* next, int64_t* next_count, void* stream) {
  t_last_error.clear();
  if (!G) return fail(BFS_ERR_INVALID_ARG, "graph is NULL");
  if (n_frontier < 0 || n_frontier > G->g.n) return fail(BFS_ERR_INVALID_ARG, "n_frontier outside [0, n]");
  if (n_frontier > 0 && !frontier) return fail(BFS_ERR_INVALID_ARG, "frontier is NULL");
  if (!bitmap || !levels || !parents || !next_bitmap || !next_count) return fail(BFS_ERR_INVALID_ARG, "NULL output");
  if (level < 1) return fail(BFS_ERR_INVALID_ARG, "level must be >= 1");
  if (G->g.new_id)
    return fail(BFS_ERR_INVALID_ARG,
                "bfs_expand_bitmap works in the graph's own numbering: create it without BFS_RELABEL_DEGREE");
  std::lock_guard<std::mutex> lock(G->mu);
  cudaError_t e = cudaSetDevice(G->g.device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  bfs_status s = ensure_single_ws(G);
  if (s != BFS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return G->g.off64 ? expand_bitmap_one<int64_t>(G, frontier, n_frontier, level, bitmap, levels, parents, next_bitmap,
                                                 next, next_count, st)
                    : expand_bitmap_one<int32_t>(G, frontier, n_frontier, level, bitmap, levels, parents, next_bitmap,
                                                 next, next_count, st);
}

GBFS_API bfs_status bfs_expand(bfs_graph_t G, const int32_t* frontier, int64_t n_frontier, int32_t level,
                               uint32_t* bitmap, int32_t* levels, int32_t* parents, int32_t* next,
                               int64_t* next_count, void* stream) {
  t_last_error.clear();
  if (!G) return fail(BFS_ERR_INVALID_ARG, "graph is NULL");
  if (n_frontier < 0 || n_frontier > G->g.n) return fail(BFS_ERR_INVALID_ARG, "n_frontier outside [0, n]");
  if (n_frontier > 0 && !frontier) return fail(BFS_ERR_INVALID_ARG, "frontier is NULL");
  if (!bitmap || !levels || !parents || !next || !next_count) return fail(BFS_ERR_INVALID_ARG, "NULL output");
  if (level < 1) return fail(BFS_ERR_INVALID_ARG, "level must be >= 1");
  if (G->g.new_id)
    return fail(BFS_ERR_INVALID_ARG, "bfs_expand works in the graph's own numbering: create it without BFS_RELABEL_DEGREE");
  std::lock_guard<std::mutex> lock(G->mu);
  cudaError_t e = cudaSetDevice(G->g.device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  bfs_status s = ensure_single_ws(G);
  if (s != BFS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n_frontier == 0) {
    if ((e = cudaMemsetAsync(next_count, 0, sizeof(int64_t), st)) != cudaSuccess) return cuda_fail(e, "memset");
    return BFS_OK;
  }
  return G->g.off64 ? expand_one<int64_t>(G, frontier, n_frontier, level, bitmap, levels, parents, next, next_count,
                                          st)
                    : expand_one<int32_t>(G, frontier, n_frontier, level, bitmap, levels, parents, next, next_count,
                                          st);
}

}  // extern "C"
