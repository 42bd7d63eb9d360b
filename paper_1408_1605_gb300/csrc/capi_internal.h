// Host-side state behind the opaque C-ABI handles (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "gbfs.h"
#include "kernels.h"

namespace gbfs {

struct BatchState;  // multi-source work buffers, see bfs_batch.cu

// Expansion shape used unless the autotuner or bfs_graph_set_shape picks another.
constexpr int kDefaultShape = 7;  // warp tiles of 128 edges, 48 registers (fastest on R-MAT)

bfs_status fail(bfs_status s, const std::string& msg);
void clear_last_error();
bfs_status cuda_fail(cudaError_t e, const char* what);

void launch_write_count(Ctl* ctl, Packed pk, int64_t* out, cudaStream_t st);

}  // namespace gbfs

struct bfs_graph_s {
  gbfs::GraphDev g;
  gbfs::SingleWs ws;
  std::mutex mu;
  int shape = gbfs::kDefaultShape;        // single-source expansion shape (kExpandShapes)
  int grid = 0;
  int batch_shape = 0;                     // multi-source expansion shape (kBatchShapes)
  bool host_loop = false;
  int loop_mode = 1;        // BFS_LOOP_PERSISTENT / BFS_LOOP_GRAPH / BFS_LOOP_HOST
  int bottom_up = 0;        // allow bottom-up levels (persistent loop only)
  int alpha = 8, beta = 24;
  int probe_mode = 1;       // bitmap pre-check through L2 (1) or default caching (0)
  long long wait_limit = 1ll << 27;  // grid-barrier polls before a wait gives up
  int persist_ctas = 0;     // CTAs per SM of a persistent search (0: as many as fit)
  int frontier_mode = 0;    // BFS_FRONTIER_LIST / _AUTO / _BITMAP
  long long last_unpacked = -1;  // levels unpacked from a bitmap by the last persistent search
  long long dense_rows = -1;     // BFS_OPT_WAVE_DENSE_ROWS (-1: the allocated pool)
  int pgrid[2] = {0, 0};    // CTAs of the persistent kernel (top-down only, with bottom-up)
  cudaGraph_t loop_graph = nullptr;
  cudaGraphExec_t loop_exec = nullptr;
  cudaEvent_t last_done = nullptr;  // completion of the last call that used the work buffers
  gbfs::BatchState* batch = nullptr;
};

namespace gbfs {
bfs_status ensure_single_ws(bfs_graph_s* G);
void set_batch_shape(bfs_graph_s* G, int shape);
void set_single_shape(bfs_graph_s* G, int shape);
void destroy_batch_state(bfs_graph_s* G);
long long batch_last_levels(const bfs_graph_s* G);    // levels of the last wave (0: none yet)
long long batch_last_overflow(const bfs_graph_s* G);  // its claim records beyond the per-vertex slots
}  // namespace gbfs
