// Kernel-shape selection: the expansion kernels are compiled for a few (BLOCK, E, CLAIM)
// shapes: threads per CTA, edges per thread (the paper's edges-per-thread parameter,
// Sec. 3.4.1, whose best value it found by a sweep) and the claim-buffer size. bfs_tune
// times every compiled shape on caller-given roots of the caller's graph and keeps the
// fastest; bfs_graph_set_shape applies a stored choice.
#include <cuda_runtime.h>

#include <limits>
#include <mutex>
#include <vector>

#include "batch.h"
#include "capi_internal.h"
#include "gbfs.h"

using namespace gbfs;

extern "C" {

GBFS_API int bfs_shape_count(int kind) {
  return kind == BFS_KERNEL_SINGLE ? kNumExpandShapes : kind == BFS_KERNEL_BATCH ? kNumBatchShapes : 0;
}

GBFS_API bfs_status bfs_shape_info(int kind, int shape, int* block, int* edges_per_thread, int* claim_buffer,
                                   int* warp_tiles) {
  clear_last_error();
  const ExpandShape* t = kind == BFS_KERNEL_SINGLE ? kExpandShapes : kind == BFS_KERNEL_BATCH ? kBatchShapes : nullptr;
  if (!t || shape < 0 || shape >= bfs_shape_count(kind)) return fail(BFS_ERR_INVALID_ARG, "unknown kernel kind or shape");
  if (block) *block = t[shape].block;
  if (edges_per_thread) *edges_per_thread = t[shape].e;
  if (claim_buffer) *claim_buffer = t[shape].claim;
  if (warp_tiles) *warp_tiles = t[shape].warp_tiles;
  return BFS_OK;
}

GBFS_API bfs_status bfs_graph_set_shape(bfs_graph_t G, int kind, int shape) {
  clear_last_error();
  if (!G) return fail(BFS_ERR_INVALID_ARG, "graph is NULL");
  if (shape < 0 || shape >= bfs_shape_count(kind)) return fail(BFS_ERR_INVALID_ARG, "unknown kernel kind or shape");
  std::lock_guard<std::mutex> lock(G->mu);
  cudaError_t e = cudaSetDevice(G->g.device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  if (G->last_done) cudaEventSynchronize(G->last_done);  // no level-loop graph may be in flight
  if (kind == BFS_KERNEL_SINGLE)
    set_single_shape(G, shape);
  else
    set_batch_shape(G, shape);
  return BFS_OK;
}

GBFS_API bfs_status bfs_graph_get_shape(bfs_graph_t G, int kind, int* shape) {
  clear_last_error();
  if (!G || !shape) return fail(BFS_ERR_INVALID_ARG, "NULL argument");
  if (kind != BFS_KERNEL_SINGLE && kind != BFS_KERNEL_BATCH) return fail(BFS_ERR_INVALID_ARG, "unknown kernel kind");
  *shape = kind == BFS_KERNEL_SINGLE ? G->shape : G->batch_shape;
  return BFS_OK;
}

GBFS_API bfs_status bfs_tune(bfs_graph_t G, int kind, const int32_t* roots, int n_roots, int32_t* levels,
                             int32_t* parents, void* stream, double* ms_per_shape, int* best_shape) {
  clear_last_error();
  if (!G || !roots || !levels || !parents || n_roots < 1) return fail(BFS_ERR_INVALID_ARG, "NULL argument or no roots");
  if (kind != BFS_KERNEL_SINGLE && kind != BFS_KERNEL_BATCH) return fail(BFS_ERR_INVALID_ARG, "unknown kernel kind");
  if (kind == BFS_KERNEL_BATCH && n_roots > kMaxWave) return fail(BFS_ERR_INVALID_ARG, "n_roots outside [1, 64]");
  const int count = bfs_shape_count(kind);
  // Single-source candidates: every shape under the CUDA-graph loop, then every shape under
  // the persistent loop with as many CTAs as fit, then with 2 CTAs per SM, then with 1 (only
  // the persistent ones when bottom-up levels are enabled). Fewer CTAs make the grid barrier
  // cheaper, which pays on graphs of hundreds of small levels.
  const int n_cand = kind == BFS_KERNEL_SINGLE ? 4 * count : count;
  auto persist_ctas = [count](int c) { return c >= 3 * count ? 1 : c >= 2 * count ? 2 : 0; };
  const bool bu = G->bottom_up != 0;
  int best = -1;
  double best_ms = std::numeric_limits<double>::infinity();
  std::vector<bfs_stats> st((size_t)n_roots);
  for (int c = 0; c < n_cand; ++c) {
    const int s = c % count;
    double ms = 0;
    bfs_status r;
    if (kind == BFS_KERNEL_SINGLE) {
      const int loop = c < count ? BFS_LOOP_GRAPH : BFS_LOOP_PERSISTENT;
      if (bu && loop == BFS_LOOP_GRAPH) {
        if (ms_per_shape) ms_per_shape[c] = -1.0;  // not a candidate
        continue;
      }
      if ((r = bfs_graph_set_option(G, BFS_OPT_LOOP, loop)) != BFS_OK) return r;
      if ((r = bfs_graph_set_option(G, BFS_OPT_PERSIST_CTAS, persist_ctas(c))) != BFS_OK) return r;
      if ((r = bfs_graph_set_shape(G, kind, s)) != BFS_OK) return r;
      if ((r = bfs_run(G, roots[0], levels, parents, stream, st.data())) != BFS_OK) return r;  // warm-up
      for (int i = 0; i < n_roots; ++i) {
        if ((r = bfs_run(G, roots[i], levels, parents, stream, st.data())) != BFS_OK) return r;
        ms += st[0].device_ms;
      }
      ms /= n_roots;
    } else {
      if ((r = bfs_graph_set_shape(G, kind, s)) != BFS_OK) return r;
      if ((r = bfs_run_batch(G, roots, n_roots, levels, parents, stream, st.data())) != BFS_OK) return r;
      if ((r = bfs_run_batch(G, roots, n_roots, levels, parents, stream, st.data())) != BFS_OK) return r;
      ms = st[0].device_ms;
    }
    if (ms_per_shape) ms_per_shape[c] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  bfs_status r;
  if (kind == BFS_KERNEL_SINGLE) {
    if ((r = bfs_graph_set_option(G, BFS_OPT_LOOP, best < count ? BFS_LOOP_GRAPH : BFS_LOOP_PERSISTENT)) != BFS_OK)
      return r;
    if ((r = bfs_graph_set_option(G, BFS_OPT_PERSIST_CTAS, persist_ctas(best))) != BFS_OK) return r;
  }
  if ((r = bfs_graph_set_shape(G, kind, best % count)) != BFS_OK) return r;
  if (best_shape) *best_shape = best;
  return BFS_OK;
}

}  // extern "C"
