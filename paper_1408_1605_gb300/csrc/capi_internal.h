// Host-side state behind the opaque C-ABI handles (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "gbfs.h"
#include "kernels.h"

namespace gbfs {

struct BatchState;  // multi-source work buffers, see bfs_batch.cu

// Expansion shape used unless the autotuner or GBFS_SHAPE picks another.
constexpr int kDefaultShape = 0;

bfs_status fail(bfs_status s, const std::string& msg);
void clear_last_error();
bfs_status cuda_fail(cudaError_t e, const char* what);

void launch_write_count(Ctl* ctl, Packed pk, int64_t* out, cudaStream_t st);

}  // namespace gbfs

struct bfs_graph_s {
  gbfs::GraphDev g;
  gbfs::SingleWs ws;
  std::mutex mu;
  int shape = gbfs::kDefaultShape;
  int grid = 0;
  bool host_loop = false;
  cudaGraph_t loop_graph = nullptr;
  cudaGraphExec_t loop_exec = nullptr;
  cudaEvent_t last_done = nullptr;  // completion of the last call that used the work buffers
  gbfs::BatchState* batch = nullptr;
};

namespace gbfs {
bfs_status ensure_single_ws(bfs_graph_s* G);
void destroy_batch_state(bfs_graph_s* G);
}  // namespace gbfs
