// Multi-source (batched) BFS state shared by the batch and serving translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace gbfs {

constexpr int kMaxWave = 64;  // roots per wave: one bit each in a 64-bit mask

// Where the outputs of each bit (slot) of a wave go, and the wave level at which each
// slot's root entered (so level[v] for that root = wave level - start).
struct WaveSlots {
  int32_t* lvl[kMaxWave];
  int32_t* par[kMaxWave];
  int32_t start[kMaxWave];
};

// Device control block of a wave. Queue buffers rotate by 3 (the expansion of frontier t
// clears the masks of frontier t - 1), scan buffers and counters by 2.
struct BatchCtl {
  unsigned long long counter[2];
  unsigned int done[2];
  int level;                      // wave level assigned by the running expansion (t + 1)
  int cont;                       // next frontier non-empty
  long long prev_count;           // size of frontier t - 1
  unsigned int error;
  unsigned int emit_done;         // CTAs finished in the emit kernel (last-CTA detection)
  unsigned long long alive[2];    // OR of the masks claimed by the running expansion (next parity)
  unsigned long long ovf_count;   // parent events that did not fit the per-vertex slots
  int bu;                         // the running level goes bottom-up (set by the previous level)
  int bu_strict;                  // the choice if some root's next frontier is small
  int bu_levels;                  // bottom-up levels so far
  long long seen;                 // degree sum of the frontiers expanded so far
  unsigned long long bitcnt[kMaxWave];  // per-root size of the new frontier (bottom-up choice)
  unsigned long long dense_count; // dense rows handed out in this wave
  unsigned int recorded;          // the running expansion wrote claim records (per-level outputs)
  unsigned int pad;
};

// Parent event of a claim: at wave level `level`, vertex u's edge claimed the bits `mask`
// of the claimed vertex (u in caller ids, ready to be written out; the event array itself is
// indexed internally).
struct ClaimEvent {
  int32_t u;
  int32_t level;
  unsigned long long mask;
};
struct OvfEvent {  // an event that did not fit the vertex's slots; v and u in caller ids
  int32_t v;
  int32_t u;
  unsigned long long mask;
  int32_t level;
  int32_t pad;
};
// Per-vertex event slots. Serving waves write their outputs after every level and reuse the
// slots level by level; bfs_run_batch keeps every event of the wave and writes the outputs
// once, after the last level, so a vertex needs room for the events of all its levels.
constexpr int kEventSlots = 4;
constexpr int kEventSlotsWave = 8;

template <typename OffT>
struct BatchArgs {
  const OffT* off;
  const int32_t* cols;
  int64_t n;
  unsigned long long* visited;    // V[v]: bit b set once root b reached v
  unsigned long long* fmask[3];   // F_t[v]: bits of roots that have v in frontier t
  int32_t* qv[3];                 // frontier vertex lists
  OffT* cum[2];
  OffT* base[2];
  TileDesc<OffT>* chunk[2];       // tile descriptors every kChunk edges (k, internal id of entry k, column)
  BatchCtl* ctl;
  const WaveSlots* slots;
  int32_t* evc;                   // events recorded per vertex this level (this wave, with defer)
  ClaimEvent* ev;                 // [n][ev_slots]
  OvfEvent* ovf;                  // events beyond the slots
  long long ovf_cap;
  Packed pk;
  cudaGraphConditionalHandle cond;
  int use_cond;
  const int32_t* new_id;          // caller -> internal vertex id (NULL: identity)
  const int32_t* old_id;          // internal -> caller vertex id (NULL: identity)
  int64_t nnz;
  int allow_bu;                   // bottom-up levels allowed (Beamer's switching, per wave)
  int alpha, beta;                // switching thresholds (as for single-source searches)
  int ev_slots;                   // event slots per vertex (kEventSlots or kEventSlotsWave)
  int defer;                      // 1: events kept for the whole wave, outputs written once at its end
  int n_slots;                    // slots (roots) of the wave whose outputs the final pass writes
  int allow_ordered;              // large frontiers may be rebuilt in vertex order (no bottom-up levels)
  // Waves with deferred outputs: a vertex whose claims outgrow its event slots gets a dense
  // row (parent and wave level per root bit, and the mask of bits set there) from a pool.
  int32_t* dense_idx;             // [n]: the vertex's row, -1 if none (NULL: no dense rows)
  int32_t* dense_par;             // [dense_cap][64]
  int32_t* dense_lvl;             // [dense_cap][64]
  unsigned long long* dense_mask; // [dense_cap]
  long long dense_cap;
  int dense_ident;                // the pool holds a row per vertex: row v is v's (no dense_idx)
  // Waves whose roots all start at level 0 (bfs_run_batch): bit v set once V[v] holds every
  // root still searching, so no edge into v can claim again (NULL: not kept).
  uint32_t* done;
  // [n rounded up to 16]: byte v is 1 once an ordered expansion put v into the next frontier
  // (the claim whose OR found F_{t+1}[v] empty stores it); k_batch_order reads and clears it.
  uint8_t* fmark;
  int order_marks;                // ordered levels keep byte marks (graphs not relabelled by degree)
};

// Work buffers of multi-source searches on one graph.
struct BatchBufs {
  bool ready = false;
  unsigned long long* visited = nullptr;
  unsigned long long* fmask[3] = {nullptr, nullptr, nullptr};
  int32_t* qv[3] = {nullptr, nullptr, nullptr};
  void* cum[2] = {nullptr, nullptr};
  void* base[2] = {nullptr, nullptr};
  void* chunk[2] = {nullptr, nullptr};  // TileDesc<OffT>[chunk_cap]
  int64_t chunk_cap = 0;
  BatchCtl* ctl = nullptr;
  WaveSlots* slots = nullptr;       // device
  long long* stats = nullptr;       // device: per slot [edges2, reached, depth]
  int32_t* roots_dev = nullptr;     // device: (vertex, mask lo, mask hi) per distinct root
  int32_t* evc = nullptr;
  ClaimEvent* ev = nullptr;
  OvfEvent* ovf = nullptr;
  long long ovf_cap = 0;
  int ev_slots = kEventSlots;
  int32_t* dense_idx = nullptr;   // dense rows (waves with deferred outputs only)
  int32_t* dense_par = nullptr;
  int32_t* dense_lvl = nullptr;
  unsigned long long* dense_mask = nullptr;
  long long dense_cap = 0;
  bool dense_ident = false;
  uint32_t* done = nullptr;         // [n / 32] (waves with deferred outputs only)
  uint8_t* fmark = nullptr;         // [n rounded up to 16], zero between ordered levels
};

struct RootSeed {
  int32_t v;
  unsigned long long mask;
};

template <typename OffT>
BatchArgs<OffT> make_batch_args(const GraphDev& g, const BatchBufs& b) {
  BatchArgs<OffT> a{};
  a.off = reinterpret_cast<const OffT*>(g.off);
  a.cols = g.cols;
  a.n = g.n;
  a.visited = b.visited;
  for (int i = 0; i < 3; ++i) {
    a.fmask[i] = b.fmask[i];
    a.qv[i] = b.qv[i];
  }
  for (int i = 0; i < 2; ++i) {
    a.cum[i] = reinterpret_cast<OffT*>(b.cum[i]);
    a.base[i] = reinterpret_cast<OffT*>(b.base[i]);
    a.chunk[i] = reinterpret_cast<TileDesc<OffT>*>(b.chunk[i]);
  }
  a.ctl = b.ctl;
  a.slots = b.slots;
  a.evc = b.evc;
  a.ev = b.ev;
  a.ovf = b.ovf;
  a.ovf_cap = b.ovf_cap;
  a.pk = g.pk;
  a.use_cond = 0;
  a.new_id = g.new_id;
  a.old_id = g.old_id;
  a.nnz = g.nnz;
  a.ev_slots = b.ev_slots;
  a.defer = 0;
  a.n_slots = kMaxWave;
  a.allow_ordered = 1;
  a.dense_idx = b.dense_idx;
  a.dense_par = b.dense_par;
  a.dense_lvl = b.dense_lvl;
  a.dense_mask = b.dense_mask;
  a.dense_cap = b.dense_cap;
  a.dense_ident = b.dense_ident ? 1 : 0;
  a.done = b.done;
  a.fmark = b.fmark;
  a.order_marks = g.old_id ? 0 : 1;
  return a;
}

// The dense row of vertex v: row v when the pool holds one per vertex, else handed out on
// first use (-1 when there are none or the pool is spent). Two claimers racing for a new row
// both take one; the loser's stays unused.
template <typename OffT>
__device__ __forceinline__ int32_t dense_row(const BatchArgs<OffT>& a, int32_t v) {
  if (a.dense_ident) return v;
  if (!a.dense_idx) return -1;
  const int32_t row = *(volatile int32_t*)(a.dense_idx + v);
  if (row >= 0) return row;
  // a spent pool is seen by a plain read: no atomic on the shared count once it is full
  if ((long long)*(volatile unsigned long long*)&a.ctl->dense_count >= a.dense_cap) return -1;
  const unsigned long long t = atomicAdd(&a.ctl->dense_count, 1ull);
  if ((long long)t >= a.dense_cap) return -1;
  const int32_t prev = atomicCAS(a.dense_idx + v, -1, (int32_t)t);
  return prev < 0 ? (int32_t)t : prev;
}

// A record slot in the overflow list, or -1 once the list is full. The count is read before
// the atomic, so that claims past a full list (a deep graph's wave claims every vertex once
// per root, at different levels) write their outputs at once instead of serialising on
// the one counter.
__device__ __forceinline__ long long ovf_slot(BatchCtl* ctl, long long cap) {
  if ((long long)*(volatile unsigned long long*)&ctl->ovf_count >= cap) return -1;
  const unsigned long long o = atomicAdd(&ctl->ovf_count, 1ull);
  return (long long)o < cap ? (long long)o : -1;
}

// Claim bits of vertex v with parent u at wave level L, written into its dense row.
template <typename OffT>
__device__ __forceinline__ void dense_write(const BatchArgs<OffT>& a, int32_t row, unsigned long long bits,
                                            int32_t u, int32_t L) {
  for (unsigned long long m = bits; m; m &= m - 1) {
    const int b = __ffsll((long long)m) - 1;
    a.dense_par[(size_t)row * kMaxWave + b] = u;
    a.dense_lvl[(size_t)row * kMaxWave + b] = L;
  }
  atomicOr(a.dense_mask + row, bits);
}

// Vertex-ordered frontiers: when the frontier being expanded holds at least n / kOrderedDiv
// vertices, the expansion only marks the next frontier's masks (no appends; on graphs not
// relabelled by degree also a byte mark per vertex, BatchArgs::fmark) and k_batch_order
// rebuilds the list from them in vertex order, so that the next expansion reads its
// frontier's masks, rows and neighbours' masks in address order. Decided from the current
// frontier's size, which every kernel of the level reads alike.
constexpr long long kOrderedDiv = 16;
template <typename OffT>
__device__ __forceinline__ bool wave_ordered(const BatchArgs<OffT>& a, long long nf) {
  return a.allow_ordered && !a.allow_bu && nf * kOrderedDiv >= a.n;
}

// True when a claim carries a single root bit: it is written out at once (that root's level
// and parent, two stores) instead of becoming a record. On graphs whose roots' frontiers
// rarely meet (grids: one bit per claim) this takes the record atomics and the later output
// pass off the claim path; claims of many bits at once (R-MAT) keep their records, whose
// outputs are written in whole lines.
__device__ __forceinline__ bool single_bit(unsigned long long bits) { return bits && !(bits & (bits - 1)); }

// Writes the level (wave level L minus the slot's start) and the parent u of every bit of
// `bits` of caller vertex vc.
__device__ __forceinline__ void write_claim_now(unsigned long long bits, int32_t vc, int32_t u, int L,
                                                int32_t* const* s_par, int32_t* const* s_lvl,
                                                const int32_t* s_start) {
  for (unsigned long long m = bits; m; m &= m - 1) {
    const int b = __ffsll((long long)m) - 1;
    s_par[b][vc] = u;
    s_lvl[b][vc] = L - s_start[b];
  }
}

// Where the claim of `bits` of vertex v (internal id) by u (caller id) at wave level L
// goes: written at once if it carries one bit; else a record in the vertex's slot `slot`
// (taken by the caller from its record count), past the slots its dense row, then the
// overflow list, then written at once. Returns whether a record was written.
template <typename OffT>
__device__ __forceinline__ bool record_claim(const BatchArgs<OffT>& a, int32_t v, unsigned long long bits, int32_t u,
                                             int L, int slot, int32_t* const* s_par, int32_t* const* s_lvl,
                                             const int32_t* s_start) {
  int32_t drow = -1;
  if (single_bit(bits)) {
    write_claim_now(bits, a.old_id ? __ldg(a.old_id + v) : v, u, L, s_par, s_lvl, s_start);
    return false;
  }
  if (slot < a.ev_slots) {
    ClaimEvent ce;
    ce.u = u;
    ce.level = L;
    ce.mask = bits;
    a.ev[(size_t)v * a.ev_slots + slot] = ce;
    return true;
  }
  if ((drow = dense_row(a, v)) >= 0) {
    dense_write(a, drow, bits, u, L);
    return true;
  }
  const long long o = ovf_slot(a.ctl, a.ovf_cap);
  const int32_t vc = a.old_id ? __ldg(a.old_id + v) : v;  // outputs use caller ids
  if (o >= 0) {
    a.ovf[o] = OvfEvent{vc, u, bits, L, 0};
    return true;
  }
  write_claim_now(bits, vc, u, L, s_par, s_lvl, s_start);  // no room
  return false;
}

// Statistics of one output array: out[0] = degree sum of reached vertices (2 m_c),
// out[1] = reached count, out[2] = max level + 1.
template <typename OffT>
void launch_level_stats(const OffT* off, const int32_t* new_id, int64_t n, const int32_t* levels, long long* out,
                        int num_sms, cudaStream_t st);

// dense_rows: rows of the dense-row pool of waves with ev_slots = kEventSlotsWave (-1: the
// default, one per 16 vertices).
cudaError_t alloc_batch_bufs(const GraphDev& g, BatchBufs& b, int ev_slots = kEventSlots, long long dense_rows = -1);
void free_batch_bufs(BatchBufs& b);
size_t batch_bufs_bytes(const GraphDev& g, int ev_slots = kEventSlots, long long dense_rows = -1);

template <typename OffT>
void launch_batch_clear(const BatchArgs<OffT>& a, int num_sms, cudaStream_t st);
template <typename OffT>
void launch_batch_seed(const BatchArgs<OffT>& a, const RootSeed* seeds_dev, int n_seeds, int wave_level,
                       bool fresh, cudaStream_t st);
extern const ExpandShape kBatchShapes[];
extern const int kNumBatchShapes;
constexpr int kDefaultBatchShape = 4;  // warp tiles of 128 edges, 256 threads
template <typename OffT>
cudaError_t launch_batch_expand(int shape, const BatchArgs<OffT>& a, int grid, cudaStream_t st);
template <typename OffT>
int batch_expand_grid(int shape, int num_sms);
void launch_fill(int32_t* p, int64_t count, int32_t value, int num_sms, cudaStream_t st);
// Writes the levels and parents of the roots' vertices claimed by the last expansion.
template <typename OffT>
void launch_batch_emit(const BatchArgs<OffT>& a, int num_sms, cudaStream_t st);
// Waves with deferred outputs (a.defer): after each level, only the per-root sizes of the
// new frontier (for the bottom-up choice; launched only when bottom-up levels are allowed);
// after the last level, every output entry of the wave's slots, written once.
template <typename OffT>
void launch_batch_count(const BatchArgs<OffT>& a, int num_sms, cudaStream_t st);
template <typename OffT>
void launch_batch_final(const BatchArgs<OffT>& a, int num_sms, cudaStream_t st);
// After every expansion: rebuilds the next frontier in vertex order if the expansion was an
// ordered one (wave_ordered), else returns at once.
template <typename OffT>
void launch_batch_order(const BatchArgs<OffT>& a, int num_sms, cudaStream_t st);
template <typename OffT>
void launch_batch_stats(const OffT* off, const int32_t* new_id, int64_t n, const WaveSlots* slots, int n_slots,
                        long long* stats, int num_sms, cudaStream_t st);
void launch_clear_bits(unsigned long long* visited, int64_t n, unsigned long long mask, int num_sms,
                       cudaStream_t st);

}  // namespace gbfs
