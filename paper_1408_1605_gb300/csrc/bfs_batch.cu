// C ABI of the multi-source search: bfs_run_batch runs up to 64 roots as one wave (one
// bit per root in 64-bit visited / frontier masks). The level loop is a CUDA graph with a
// conditional WHILE node, as for single-source searches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "batch.h"
#include "capi_internal.h"
#include "gbfs.h"

namespace gbfs {

struct BatchState {
  BatchBufs b;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int grid = 0;
  cudaEvent_t ev0 = nullptr, ev_mid = nullptr, ev1 = nullptr;
  BatchCtl* ctl_host = nullptr;      // pinned
  long long* stats_host = nullptr;   // pinned, 3 * kMaxWave
  long long last_levels = 0;         // levels and overflow records of the last wave
  long long last_overflow = 0;
  int32_t* stage_lvl = nullptr;      // device staging when outputs are host memory
  int32_t* stage_par = nullptr;
  int stage_roots = 0;
};

template <typename T>
static cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
}

void free_batch_bufs(BatchBufs& b);

static void free_batch(BatchState* S) {
  free_batch_bufs(S->b);
  cudaFree(S->stage_lvl);
  cudaFree(S->stage_par);
  if (S->exec) cudaGraphExecDestroy(S->exec);
  if (S->graph) cudaGraphDestroy(S->graph);
  if (S->ev0) cudaEventDestroy(S->ev0);
  if (S->ev_mid) cudaEventDestroy(S->ev_mid);
  if (S->ev1) cudaEventDestroy(S->ev1);
  if (S->ctl_host) cudaFreeHost(S->ctl_host);
  if (S->stats_host) cudaFreeHost(S->stats_host);
}

long long batch_last_levels(const bfs_graph_s* G) { return G->batch ? G->batch->last_levels : 0; }
long long batch_last_overflow(const bfs_graph_s* G) { return G->batch ? G->batch->last_overflow : 0; }

void destroy_batch_state(bfs_graph_s* G) {
  if (G->batch) {
    free_batch(G->batch);
    delete G->batch;
    G->batch = nullptr;
  }
}


void free_batch_bufs(BatchBufs& b) {
  cudaFree(b.visited);
  for (int i = 0; i < 3; ++i) {
    cudaFree(b.fmask[i]);
    cudaFree(b.qv[i]);
  }
  for (int i = 0; i < 2; ++i) {
    cudaFree(b.cum[i]);
    cudaFree(b.base[i]);
    cudaFree(b.chunk[i]);
  }
  cudaFree(b.ctl);
  cudaFree(b.slots);
  cudaFree(b.stats);
  cudaFree(b.roots_dev);
  cudaFree(b.evc);
  cudaFree(b.ev);
  cudaFree(b.ovf);
  cudaFree(b.dense_idx);
  cudaFree(b.done);
  cudaFree(b.fmark);
  cudaFree(b.dense_par);
  cudaFree(b.dense_lvl);
  cudaFree(b.dense_mask);
  b = BatchBufs{};
}

// Room for claim records beyond the per-vertex slots; past it a claim writes its outputs at
// once. (A list of n records, enough for every spilled record of an R-MAT s26 wave, was
// measured slower than this one: replaying tens of millions of records after the last level
// cost more than writing them during the levels.)
static long long overflow_cap(const GraphDev& g, int ev_slots) {
  (void)ev_slots;
  return g.n / 4 + 65536;
}

// Dense rows of the waves that keep their claim records to the end: `rows` if given (at
// most one per vertex), else one per 16 vertices.
static long long dense_rows_cap(const GraphDev& g, int ev_slots, long long rows) {
  if (ev_slots != kEventSlotsWave) return 0;
  return rows >= 0 ? std::min<long long>(rows, g.n) : g.n / 16 + 1024;
}

// The default pool: a row per vertex (row v is v's: no allocation on the claim path, measured
// 4-17 % faster waves on R-MAT s22 / s26 and uniform s26 than one row per 16 vertices) when
// those 520 bytes per vertex take at most a quarter of the free device memory.
static long long default_dense_rows(const GraphDev& g) {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  const size_t per_row = sizeof(int32_t) * 2 * kMaxWave + sizeof(unsigned long long);
  return (size_t)g.n * per_row <= free_b / 4 ? g.n : -1;
}

size_t batch_bufs_bytes(const GraphDev& g, int ev_slots, long long dense_rows) {
  const size_t osz = g.off64 ? 8 : 4;
  const size_t ovf_cap = (size_t)overflow_cap(g, ev_slots);
  const size_t dense = (size_t)dense_rows_cap(g, ev_slots, dense_rows);
  return (size_t)g.n * (8 * 4 + 4 * 3 + 2 * 2 * osz + 4 + sizeof(ClaimEvent) * ev_slots + (dense ? 4 : 0)) +
         (ev_slots == kEventSlotsWave ? (size_t)(g.n + 31) / 32 * 4 : 0) + (size_t)(g.n + 15) / 16 * 16 +
         ovf_cap * sizeof(OvfEvent) + 2 * 16 * (size_t)(g.nnz / kChunk + 2) + dense * (8 * kMaxWave + 8) +
         64 * 1024;
}

cudaError_t alloc_batch_bufs(const GraphDev& g, BatchBufs& b, int ev_slots, long long dense_rows) {
  const size_t osz = g.off64 ? 8 : 4;
  b.chunk_cap = g.nnz / kChunk + 2;
  cudaError_t e = dalloc(&b.visited, (size_t)g.n);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    e = dalloc(&b.fmask[i], (size_t)g.n);
    if (e == cudaSuccess) e = dalloc(&b.qv[i], (size_t)g.n);
  }
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = dalloc(reinterpret_cast<char**>(&b.cum[i]), (size_t)g.n * osz);
    if (e == cudaSuccess) e = dalloc(reinterpret_cast<char**>(&b.base[i]), (size_t)g.n * osz);
    if (e == cudaSuccess) e = dalloc(reinterpret_cast<char**>(&b.chunk[i]), (size_t)b.chunk_cap * 16);
  }
  if (e == cudaSuccess) e = dalloc(&b.ctl, 1);
  if (e == cudaSuccess) e = dalloc(&b.slots, 1);
  if (e == cudaSuccess) e = dalloc(&b.stats, 3 * kMaxWave);
  if (e == cudaSuccess) e = dalloc(&b.roots_dev, 4 * kMaxWave);
  b.ovf_cap = overflow_cap(g, ev_slots);
  if (e == cudaSuccess) e = dalloc(&b.evc, (size_t)g.n);
  b.ev_slots = ev_slots;
  if (e == cudaSuccess) e = dalloc(&b.ev, (size_t)g.n * ev_slots);
  if (e == cudaSuccess) e = dalloc(&b.ovf, (size_t)b.ovf_cap);
  b.dense_cap = dense_rows_cap(g, ev_slots, dense_rows);
  b.dense_ident = b.dense_cap > 0 && b.dense_cap >= g.n;  // row v is vertex v's: no index
  if (b.dense_cap > 0) {
    if (e == cudaSuccess && !b.dense_ident) e = dalloc(&b.dense_idx, (size_t)g.n);
    if (e == cudaSuccess) e = dalloc(&b.dense_par, (size_t)b.dense_cap * kMaxWave);
    if (e == cudaSuccess) e = dalloc(&b.dense_lvl, (size_t)b.dense_cap * kMaxWave);
    if (e == cudaSuccess) e = dalloc(&b.dense_mask, (size_t)b.dense_cap);
  }
  if (ev_slots == kEventSlotsWave && e == cudaSuccess) e = dalloc(&b.done, (size_t)(g.n + 31) / 32);
  const size_t fmark_bytes = (size_t)(g.n + 15) / 16 * 16;  // whole 16-byte words: the padding stays 0
  if (e == cudaSuccess) e = dalloc(&b.fmark, fmark_bytes);
  if (e == cudaSuccess) e = cudaMemset(b.fmark, 0, fmark_bytes);
  if (e == cudaSuccess) e = cudaMemset(b.evc, 0, sizeof(int32_t) * (size_t)g.n);
  if (e == cudaSuccess) e = cudaMemset(b.ctl, 0, sizeof(BatchCtl));
  if (e != cudaSuccess) {
    free_batch_bufs(b);
    return e;
  }
  b.ready = true;
  return cudaSuccess;
}

bfs_status ensure_batch_state(bfs_graph_s* G) {
  if (G->batch && G->batch->b.ready) return BFS_OK;
  auto* S = new (std::nothrow) BatchState();
  if (!S) return fail(BFS_ERR_OOM, "host allocation");
  const GraphDev& g = G->g;
  cudaError_t e =
      alloc_batch_bufs(g, S->b, kEventSlotsWave, G->dense_rows >= 0 ? G->dense_rows : default_dense_rows(g));
  if (e == cudaSuccess) e = cudaEventCreate(&S->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&S->ev_mid);
  if (e == cudaSuccess) e = cudaEventCreate(&S->ev1);
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&S->ctl_host), sizeof(BatchCtl), 0);
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&S->stats_host), sizeof(long long) * 3 * kMaxWave, 0);
  if (e != cudaSuccess) {
    free_batch(S);
    delete S;
    return cuda_fail(e, "batch work buffers");
  }
  S->grid = g.off64 ? batch_expand_grid<int64_t>(G->batch_shape, g.num_sms)
                    : batch_expand_grid<int32_t>(G->batch_shape, g.num_sms);
  G->batch = S;
  return BFS_OK;
}

template <typename OffT>
BatchArgs<OffT> batch_args(const bfs_graph_s* G) {
  BatchArgs<OffT> a = make_batch_args<OffT>(G->g, G->batch->b);
  a.allow_bu = G->bottom_up;  // BFS_OPT_BOTTOM_UP also lets waves run bottom-up levels
  a.alpha = G->alpha;
  a.beta = G->beta;
  a.defer = 1;  // every event kept until the wave ends; the outputs are written once, after it
  // Done marks only for graphs in input order: there a vertex's 64-bit visited mask is a
  // DRAM-random read that a mark spares (uniform s26 waves 415 vs 469 ms). On graphs
  // relabelled by degree the masks most edges read are the hubs', few and L2-resident, and
  // the extra mark read cost more than it saved (R-MAT s26 waves 80 vs 71 ms, s22 6.9 vs
  // 4.0 ms).
  if (G->g.old_id) a.done = nullptr;
  if (a.dense_cap <= 0) {  // no dense rows: overflow list, then direct writes
    a.dense_idx = nullptr;
    a.dense_ident = 0;
  }
  return a;
}

template BatchArgs<int32_t> batch_args<int32_t>(const bfs_graph_s*);
template BatchArgs<int64_t> batch_args<int64_t>(const bfs_graph_s*);

template <typename OffT>
static bfs_status build_batch_graph(bfs_graph_s* G) {
  BatchState* S = G->batch;
  cudaError_t e;
  cudaGraph_t graph = nullptr;
  if ((e = cudaGraphCreate(&graph, 0)) != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
  cudaGraphConditionalHandle handle;
  cudaGraphNodeParams cp{};
  cudaGraphNode_t node;
  cudaStream_t cs = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t captured = nullptr;
  BatchArgs<OffT> a = batch_args<OffT>(G);
  if ((e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault)) != cudaSuccess) goto bad;
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if ((e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp)) != cudaSuccess) goto bad;
  a.cond = handle;
  a.use_cond = 1;
  if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) goto bad;
  if ((e = cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
    cudaStreamDestroy(cs);
    goto bad;
  }
  {
    cudaError_t le = launch_batch_expand<OffT>(G->batch_shape, a, S->grid, cs);
    if (a.allow_bu) launch_batch_count<OffT>(a, G->g.num_sms, cs);
    launch_batch_order<OffT>(a, G->g.num_sms, cs);
    e = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    if (le != cudaSuccess) e = le;
  }
  if (e != cudaSuccess) goto bad;
  if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) goto bad;
  S->graph = graph;
  S->exec = exec;
  return BFS_OK;
bad:
  cudaGraphDestroy(graph);
  return cuda_fail(e, "batch level-loop graph");
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
static bfs_status run_batch(bfs_graph_s* G, const int32_t* roots, int n_roots, int32_t* levels, int32_t* parents,
                            cudaStream_t st, bfs_stats* stats) {
  BatchState* S = G->batch;
  const GraphDev& g = G->g;
  cudaError_t e;
  const bool host_out = !is_device_ptr(levels) || !is_device_ptr(parents);
  int32_t* dl = levels;
  int32_t* dp = parents;
  const size_t per = (size_t)g.n;
  if (host_out) {
    if (S->stage_roots < n_roots) {
      cudaFree(S->stage_lvl);
      cudaFree(S->stage_par);
      S->stage_lvl = S->stage_par = nullptr;
      S->stage_roots = 0;
      if ((e = dalloc(&S->stage_lvl, per * n_roots)) != cudaSuccess ||
          (e = dalloc(&S->stage_par, per * n_roots)) != cudaSuccess)
        return cuda_fail(e, "batch output staging");
      S->stage_roots = n_roots;
    }
    dl = S->stage_lvl;
    dp = S->stage_par;
  }
  // slot table: root b writes row b of the outputs
  WaveSlots slots{};
  for (int b = 0; b < kMaxWave; ++b) {
    const int bb = b < n_roots ? b : 0;
    slots.lvl[b] = dl + per * bb;
    slots.par[b] = dp + per * bb;
    slots.start[b] = 0;
  }
  // distinct roots, each with the mask of the slots it seeds
  std::map<int32_t, unsigned long long> masks;
  for (int b = 0; b < n_roots; ++b) masks[roots[b]] |= 1ull << b;
  std::vector<RootSeed> seeds;
  for (auto& kv : masks) seeds.push_back(RootSeed{kv.first, kv.second});
  if (G->last_done) cudaStreamWaitEvent(st, G->last_done, 0);
  if ((e = cudaEventRecord(S->ev0, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  if ((e = cudaMemcpyAsync(S->b.slots, &slots, sizeof(WaveSlots), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(S->b.roots_dev, seeds.data(), sizeof(RootSeed) * seeds.size(), cudaMemcpyHostToDevice,
                           st)) != cudaSuccess)
    return cuda_fail(e, "batch inputs");
  BatchArgs<OffT> a = batch_args<OffT>(G);
  a.n_slots = n_roots;
  // no fill of the outputs: the final pass writes every entry the roots' seeds do not
  launch_batch_clear<OffT>(a, g.num_sms, st);
  launch_batch_seed<OffT>(a, reinterpret_cast<const RootSeed*>(S->b.roots_dev), (int)seeds.size(), 0, true, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch init");
  if ((e = cudaEventRecord(S->ev_mid, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  if (G->host_loop) {
    for (int64_t it = 0; it <= g.n; ++it) {
      if ((e = launch_batch_expand<OffT>(G->batch_shape, a, S->grid, st)) != cudaSuccess)
        return cuda_fail(e, "batch expand");
      if (a.allow_bu) launch_batch_count<OffT>(a, g.num_sms, st);
      launch_batch_order<OffT>(a, g.num_sms, st);
      if ((e = cudaMemcpyAsync(S->ctl_host, S->b.ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "batch level sync");
      if (!S->ctl_host->cont) break;
    }
  } else {
    if (!S->exec) {
      bfs_status s = build_batch_graph<OffT>(G);
      if (s != BFS_OK) return s;
    }
    if ((e = cudaGraphLaunch(S->exec, st)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  }
  launch_batch_final<OffT>(a, g.num_sms, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch outputs");
  if ((e = cudaEventRecord(S->ev1, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  if (stats)
    launch_batch_stats<OffT>(reinterpret_cast<const OffT*>(g.off), g.new_id, g.n, S->b.slots, n_roots, S->b.stats, g.num_sms,
                             st);
  if (host_out) {
    if ((e = cudaMemcpyAsync(levels, dl, per * n_roots * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(parents, dp, per * n_roots * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "batch output copy");
  }
  if ((e = cudaMemcpyAsync(S->ctl_host, S->b.ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "batch control copy");
  if (stats && (e = cudaMemcpyAsync(S->stats_host, S->b.stats, sizeof(long long) * 3 * n_roots,
                                    cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "batch stats copy");
  if (!G->last_done && (e = cudaEventCreateWithFlags(&G->last_done, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "cudaEventCreate");
  cudaEventRecord(G->last_done, st);
  if (stats || host_out) {
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "batch search");
    if (S->ctl_host->error & kErrColumnRange) return fail(BFS_ERR_INVALID_GRAPH, "a column id outside [0, n) was met");
    S->last_levels = S->ctl_host->level - 1;
    S->last_overflow = (long long)S->ctl_host->ovf_count;
    if (stats) {
      float ms = 0.f, loop_ms = 0.f;
      cudaEventElapsedTime(&ms, S->ev0, S->ev1);
      cudaEventElapsedTime(&loop_ms, S->ev_mid, S->ev1);
      for (int b = 0; b < n_roots; ++b) {
        stats[b].depth = (int32_t)S->stats_host[3 * b + 2];
        stats[b].bottom_up_levels = S->ctl_host->bu_levels;  // levels the wave ran bottom-up
        stats[b].vertices_reached = S->stats_host[3 * b + 1];
        stats[b].edges_traversed = S->stats_host[3 * b + 0] / 2;
        stats[b].device_ms = ms;
        stats[b].expand_ms = loop_ms;
      }
    }
  }
  return BFS_OK;
}

// Switches the multi-source expansion shape; the level-loop graph is rebuilt on next use.
void set_batch_shape(bfs_graph_s* G, int shape) {
  G->batch_shape = shape;
  if (G->batch) {
    BatchState* S = G->batch;
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->graph) cudaGraphDestroy(S->graph);
    S->exec = nullptr;
    S->graph = nullptr;
    S->grid = G->g.off64 ? batch_expand_grid<int64_t>(shape, G->g.num_sms)
                         : batch_expand_grid<int32_t>(shape, G->g.num_sms);
  }
}

}  // namespace gbfs

using namespace gbfs;

extern "C" GBFS_API bfs_status bfs_run_batch(bfs_graph_t G, const int32_t* roots, int n_roots, int32_t* levels,
                                             int32_t* parents, void* stream, bfs_stats* per_root_stats) {
  clear_last_error();
  if (!G) return fail(BFS_ERR_INVALID_ARG, "graph is NULL");
  if (!roots || !levels || !parents) return fail(BFS_ERR_INVALID_ARG, "NULL argument");
  if (n_roots < 1 || n_roots > kMaxWave) return fail(BFS_ERR_INVALID_ARG, "n_roots outside [1, 64]");
  for (int b = 0; b < n_roots; ++b)
    if (roots[b] < 0 || roots[b] >= G->g.n) return fail(BFS_ERR_INVALID_ARG, "root outside [0, n)");
  std::lock_guard<std::mutex> lock(G->mu);
  cudaError_t e = cudaSetDevice(G->g.device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  bfs_status s = ensure_batch_state(G);
  if (s != BFS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return G->g.off64 ? run_batch<int64_t>(G, roots, n_roots, levels, parents, st, per_root_stats)
                    : run_batch<int32_t>(G, roots, n_roots, levels, parents, st, per_root_stats);
}
