// Multi-source (batched) BFS: filled in below.
#include "capi_internal.h"

namespace gbfs {
struct BatchState {};
void destroy_batch_state(bfs_graph_s* G) {
  delete G->batch;
  G->batch = nullptr;
}
}  // namespace gbfs
