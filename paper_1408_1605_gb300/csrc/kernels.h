// Internal declarations shared by the gbfs translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gbfs {

// Granularity of the precomputed per-tile binary-search answers (chunk index). Every
// expansion tile size is a multiple of it.
constexpr int kChunk = 128;

// Device copy of a graph: offsets are int32 when the entry count allows, else int64.
struct GraphDev {
  int device = 0;
  int num_sms = 0;
  int64_t n = 0;
  int64_t nnz = 0;
  bool off64 = false;
  void* off = nullptr;      // OffT[n + 1]
  int32_t* cols = nullptr;  // int32[nnz]
  Packed pk{};
  // Degree relabelling (BFS_RELABEL_DEGREE): off / cols hold the renumbered graph, new_id
  // maps a caller id to the internal one and old_id back. Both NULL when not relabelled.
  int32_t* new_id = nullptr;
  int32_t* old_id = nullptr;
};

// Renumbers g by non-increasing degree on the device (replaces off / cols, sets new_id /
// old_id). Synchronous on st.
cudaError_t relabel_by_degree(GraphDev& g, cudaStream_t st);

// Work buffers of single-source searches on one graph (reused across calls).
struct SingleWs {
  bool ready = false;
  uint32_t* bitmap = nullptr;  // ceil(n / 32) words
  int32_t* v[2] = {nullptr, nullptr};
  void* cum[2] = {nullptr, nullptr};
  void* base[2] = {nullptr, nullptr};
  void* chunk[2] = {nullptr, nullptr};  // TileDesc<OffT>[chunk_cap] (the chunk index)
  int64_t chunk_cap = 0;       // entries per chunk array
  Ctl* ctl = nullptr;
  void* scan_partial = nullptr;
  int scan_parts = 0;
  int32_t* host_levels = nullptr;   // device staging when the caller passes host outputs
  int32_t* host_parents = nullptr;
  Ctl* ctl_host = nullptr;          // pinned mirror of ctl
  uint32_t* fbm[3] = {nullptr, nullptr, nullptr};  // frontier bitmaps (persistent search)
  PCtl* pctl = nullptr;
  PCtl* pctl_host = nullptr;        // pinned mirror
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_mid = nullptr;

  template <typename OffT>
  FrontierBuf<OffT> fr(int i) const {
    return FrontierBuf<OffT>{v[i], reinterpret_cast<OffT*>(cum[i]), reinterpret_cast<OffT*>(base[i])};
  }
  template <typename OffT>
  TileDesc<OffT>* desc(int i) const {
    return reinterpret_cast<TileDesc<OffT>*>(chunk[i]);
  }
};

template <typename OffT>
struct ExpandArgs {
  const OffT* off;
  const int32_t* cols;
  uint32_t* bitmap;
  int64_t n;
  FrontierBuf<OffT> fr[2];
  TileDesc<OffT>* chunk[2];
  Ctl* ctl;
  Packed pk;
  cudaGraphConditionalHandle cond;
  int use_cond;
  int probe_mode;   // bitmap pre-check: 0 default caching, 1 L2 only
  const int32_t* old_id;  // internal -> caller vertex id (NULL: identity)
  uint32_t* fbm[2];       // next-frontier bitmaps by level parity (frontier-bitmap mode), else NULL
  long long list_cap;     // frontier-bitmap mode: most list entries a level appends (-1: none)
};

template <typename OffT>
struct PersistArgs {
  const OffT* off;
  const int32_t* cols;
  uint32_t* bitmap;
  uint32_t* fbm[3];
  int64_t n;
  int64_t nnz;
  FrontierBuf<OffT> fr[2];
  TileDesc<OffT>* chunk[2];
  PCtl* ctl;
  Packed pk;
  int32_t* levels;
  int32_t* parents;
  int alpha;            // switch to bottom-up when frontier edges * alpha > unexplored edges
  int beta;             // back to top-down when frontier vertices * beta < n (and shrinking)
  int allow_bottom_up;
  int probe_mode;
  long long spin_limit;  // polls of a grid-barrier wait before it gives up (kErrTimeout)
  const int32_t* old_id;  // internal -> caller vertex id (NULL: identity)
  int bitmap_mode;        // frontier-bitmap mode: top-down levels also record claims in fbm
  long long list_cap;     // most list entries a top-down level appends (-1: none) in that mode
};

struct ExpandShape {
  int id, block, e, claim;
  int warp_tiles;  // 1: each warp expands its own tiles of 32 x e edges (claim = per warp)
};
extern const ExpandShape kExpandShapes[];
extern const int kNumExpandShapes;

// Frontier-bitmap mode (the paper's list-or-bitmap switch, Sec. 5): a top-down level
// appends to the next-frontier list only while it holds at most list_cap entries, the
// point past which a list of 32-bit ids is larger than an n-bit bitmap; every claim is also
// set in the next-frontier bitmap, and a level that stopped appending has its list rebuilt
// from the bitmap afterwards.
inline long long frontier_list_cap(int mode, int64_t n) {
  return mode == 2 ? -1 : (n + 31) / 32;  // 1: auto (list bits > n switches), 2: bitmap always
}

// After an expansion of a level-loop launch (graph or host loop): when the level dropped
// its list, rebuild the next frontier from the bitmap (vertex order, warp-centric unpack);
// in every case leave the bitmap cleared for reuse.
template <typename OffT>
void launch_unpack_level(const GraphDev& g, const ExpandArgs<OffT>& a, cudaStream_t st);
// The same unpack on caller state (bfs_expand_bitmap): the vertices of `bitmap` as a list
// (next[0 .. *count)), plus the scan and tile descriptors in the workspace buffers of parity
// `par`. Synchronous.
template <typename OffT>
cudaError_t unpack_bitmap_to_list(const GraphDev& g, SingleWs& ws, int par, const uint32_t* bitmap, int32_t* next,
                                  int64_t* count_dev, cudaStream_t st);

template <typename OffT>
void launch_init_single(const GraphDev& g, int32_t root, int32_t* levels, int32_t* parents, SingleWs& ws,
                        cudaStream_t st, bool clear_fbm = false);
template <typename OffT>
void launch_scan_frontier(const GraphDev& g, const int32_t* front, int64_t nf, int32_t level, int32_t* levels,
                          int32_t* parents, SingleWs& ws, cudaStream_t st);
template <typename OffT>
cudaError_t launch_expand(int shape, const ExpandArgs<OffT>& a, int grid, cudaStream_t st);
template <typename OffT>
int expand_grid(int shape, int num_sms);
template <typename OffT>
void launch_init_persist(const GraphDev& g, int32_t root, int32_t* levels, int32_t* parents, SingleWs& ws,
                         cudaStream_t st);
template <typename OffT>
cudaError_t launch_persistent(int shape, const PersistArgs<OffT>& a, int grid, cudaStream_t st);
template <typename OffT>
int persistent_grid(int shape, int num_sms, bool with_bu);

}  // namespace gbfs
