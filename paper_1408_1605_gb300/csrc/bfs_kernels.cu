// Single-source BFS kernels for sm_103a: output init, the standalone degree scan, and
// the fused frontier-expansion kernels (Sec. 3.4, Algorithm 3, with the optimizations of
// Sec. 3.4.1), per level or all levels in one persistent launch with bottom-up levels.
//
// Level structure (Algorithm 2 with R = C = 1). The frontier of a level is held as
// (v[k], cum[k], base[k]) plus a chunk index of tile descriptors: descriptor c holds
// k = max{k : cum[k] <= c * kChunk}, the answer of Algorithm 3's binary search for
// every kChunk-th edge, with that entry's parent id and the column entry of edge
// c * kChunk; it is written when the frontier is built. One expansion processes the
// level's edge space [0, r) in tiles, of BLOCK * E edges per CTA (CTA tiles) or of 32 * E
// edges per warp (warp tiles):
//   1. tile bounds from the chunk index (the per-tile binary search, precomputed);
//   2. the edge -> entry map: a warp tile inside one row takes it from its descriptor; a
//      warp tile over at most 32 entries holds them one per lane and searches them with
//      shuffles; a CTA tile stages its entries in shared memory, searches once, then walks
//      (Sec. 3.4.1: advance k while e >= cum[k + 1]);
//   3. lane l takes edges l, l + 32, ... of its warp's 32 * E (coalesced column reads), and
//      all E column loads are issued before any is used (the interleaving of Sec. 3.4.1);
//   4. bitmap pre-check, then atomicOr claim (Algorithm 3's visited test and claim); the winner writes
//      level and parent (Algorithm 3's output writes) and reads the claimed vertex's degree;
//   5. claimed vertices are appended to a warp (or CTA) buffer with one shared atomic or
//      ballot per warp; the buffer is flushed with ONE global 64-bit atomicAdd that reserves
//      both the queue slots and the edge range (the exclusive scan of the next frontier's
//      degrees, Sec. 3.4, fused into Algorithm 3's frontier append).
// The last CTA to finish closes the level (no spin-waits in the per-level kernels; the
// persistent kernel's grid barrier waits are bounded).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "device_util.cuh"
#include "kernels.h"

namespace gbfs {

// ---------------------------------------------------------------------------------------
// Frontier construction helpers

template <typename OffT>
__global__ void k_init_single(const OffT* __restrict__ off, int64_t n, int32_t root, const int32_t* new_id,
                              int32_t* levels, int32_t* parents, uint32_t* bitmap, FrontierBuf<OffT> f0,
                              TileDesc<OffT>* chunk0, Ctl* ctl, Packed pk, uint32_t* fbm0, uint32_t* fbm1) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += stride) {  // outputs are indexed by caller ids
    const bool is_root = i == root;
    levels[i] = is_root ? 0 : -1;
    parents[i] = is_root ? root : -1;
  }
  const int32_t rn = new_id ? new_id[root] : root;  // the root's internal id
  const int64_t nw = (n + 31) / 32;
  for (int64_t w = tid; w < nw; w += stride) {
    bitmap[w] = (w == (rn >> 5)) ? (1u << (rn & 31)) : 0u;
    if (fbm0) {  // frontier-bitmap mode: next-frontier bitmaps start cleared
      fbm0[w] = 0u;
      fbm1[w] = 0u;
    }
  }
  const OffT o0 = off[rn], deg = off[rn + 1] - o0;
  // chunk starts of the root's row, spread over the grid (a hub root spans many chunks)
  const int64_t nchunks = ((int64_t)deg + kChunk - 1) / kChunk;
  for (int64_t c = tid; c < nchunks; c += stride) chunk0[c] = TileDesc<OffT>{0, root, o0 + (OffT)(c * kChunk)};
  if (tid == 0) {
    f0.v[0] = root;  // the queue holds caller ids
    f0.cum[0] = 0;
    f0.base[0] = o0;
    ctl->counter[0] = pk.make(1, (long long)deg);
    ctl->counter[1] = 0;
    ctl->done[0] = ctl->done[1] = 0;
    ctl->level = 1;
    ctl->depth = 1;
    ctl->reached = 1;
    ctl->edges2 = 0;
    ctl->error = 0;
    ctl->cont = deg > 0;
    ctl->levels = levels;
    ctl->parents = parents;
    ctl->dropped = 0;
    ctl->bm_counter = 0;
  }
}

// Degree gather + exclusive scan of a caller-given frontier list (Sec. 3.4: the degrees
// of the frontier vertices are scanned into the cumulative degree array). Reduce-then-scan
// over a fixed grid: per-CTA partial sums, a one-CTA scan of the partials, then a
// per-CTA rescan that writes (v, cum, base) and the chunk index.
template <typename OffT>
__device__ __forceinline__ OffT frontier_degree(const OffT* off, int64_t n, int32_t v, Ctl* ctl) {
  if ((uint32_t)v >= (uint64_t)n) {
    atomicOr(&ctl->error, kErrFrontierRange);
    return 0;
  }
  return off[v + 1] - off[v];
}

template <typename OffT>
__global__ void k_scan_partials(const OffT* __restrict__ off, int64_t n, const int32_t* __restrict__ front,
                                int64_t nf, OffT* partial, Ctl* ctl) {
  __shared__ OffT s_warp[33];
  const int64_t per = (nf + gridDim.x - 1) / gridDim.x;
  const int64_t lo = min(nf, per * blockIdx.x), hi = min(nf, lo + per);
  OffT sum = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) sum += frontier_degree(off, n, front[i], ctl);
  OffT total;
  block_exclusive_scan(sum, s_warp, &total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

template <typename OffT>
__global__ void k_scan_top(OffT* partial, int nparts, int64_t nf, Ctl* ctl, Packed pk, int32_t level,
                           int32_t* levels, int32_t* parents, long long max_edges) {
  __shared__ OffT s_warp[33];
  __shared__ OffT s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < nparts; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const OffT x = i < nparts ? partial[i] : 0;
    OffT total;
    const OffT ex = block_exclusive_scan(x, s_warp, &total);
    if (i < nparts) partial[i] = s_carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // A caller frontier with repeated hubs can exceed the chunk index / counter capacity:
    // report it and expand nothing.
    const bool over = (long long)s_carry > max_edges;
    if (over) atomicOr(&ctl->error, kErrCounterOverflow);
    const int cur = (level - 1) & 1;
    ctl->counter[cur] = over ? 0ull : pk.make(nf, (long long)s_carry);
    ctl->counter[cur ^ 1] = 0;
    ctl->done[0] = ctl->done[1] = 0;
    ctl->level = level;
    ctl->depth = 0;
    ctl->reached = 0;
    ctl->edges2 = 0;
    ctl->cont = 1;
    ctl->levels = levels;
    ctl->parents = parents;
  }
}

template <typename OffT>
__global__ void k_scan_final(const OffT* __restrict__ off, int64_t n, const int32_t* __restrict__ front,
                             int64_t nf, const OffT* partial, FrontierBuf<OffT> f, TileDesc<OffT>* chunk,
                             const Ctl* ctl) {
  __shared__ OffT s_warp[33];
  if (ctl->error & kErrCounterOverflow) return;  // reported by k_scan_top; nothing to expand
  const int64_t per = (nf + gridDim.x - 1) / gridDim.x;
  const int64_t lo = min(nf, per * blockIdx.x), hi = min(nf, lo + per);
  OffT carry = partial[blockIdx.x];
  for (int64_t b = lo; b < hi; b += blockDim.x) {
    const int64_t i = b + threadIdx.x;
    int32_t v = 0;
    OffT d = 0, o = 0;
    if (i < hi) {
      v = front[i];
      if ((uint32_t)v < (uint64_t)n) {
        o = off[v];
        d = off[v + 1] - o;
      }
    }
    OffT total;
    const OffT ex = block_exclusive_scan(d, s_warp, &total);
    if (i < hi) {
      const OffT c = carry + ex;
      f.v[i] = v;
      f.cum[i] = c;
      f.base[i] = o - c;
      write_descs(chunk, c, d, (int32_t)i, v, o - c);
    }
    carry += total;
  }
}

// ---------------------------------------------------------------------------------------
// Frontier expansion (top-down step, shared by the per-level kernel and the persistent one)

template <typename OffT, int BLOCK, int E, int CLAIM>
struct ExpandSmem {
  static constexpr int T = BLOCK * E;
  static constexpr int CAP = T + 1;  // staged frontier entries per tile (fast path)
  // layout: base[CAP] (OffT) | rel[CAP + 1] (int32) | u[CAP] (int32) | claim[CLAIM] (int2)
  static constexpr size_t off_base = 0;
  static constexpr size_t off_rel = off_base + sizeof(OffT) * CAP;
  static constexpr size_t off_u = off_rel + sizeof(int32_t) * (CAP + 1);
  static constexpr size_t off_claim = ((off_u + sizeof(int32_t) * CAP) + 15) & ~size_t(15);
  static constexpr size_t bytes = off_claim + sizeof(int2) * CLAIM;
};

// Static shared state of one CTA.
template <typename OffT>
struct ExpandShared {
  OffT warp[33];
  unsigned long long resv;
  int nclaim, klo, kend;
};

// Where one level reads its frontier and writes the next one.
template <typename OffT>
struct LevelIO {
  FrontierBuf<OffT> in, out;
  const TileDesc<OffT>* chunk_in;
  TileDesc<OffT>* chunk_out;
  unsigned long long* counter_out;  // packed (count, edges) of the next frontier
  int32_t* levels;
  int32_t* parents;
  uint32_t* fbm_out;                // next frontier as a bitmap (nullptr: not kept)
  int L;                            // level assigned to claimed vertices
  int probe_mode;                   // bitmap pre-check: 0 default caching, 1 L2 only
  const int32_t* old_id;            // internal -> caller id for the outputs (NULL: identity)
  int64_t nf;                       // current frontier size
  OffT r;                           // current frontier's degree sum
  long long list_cap;               // frontier-bitmap mode: most list entries (kNoListCap: list only)
  uint32_t vis_below;               // every vertex below it is visited: no pre-check for those
  unsigned* dropped;                // set when a claim was left out of the list (bitmap only)
};

constexpr long long kNoListCap = 0x7fffffffffffffffll;

// Frontier-bitmap mode, per warp, decided where a full claim buffer would be appended: keep
// appending while the list stays within the cap; past it the level drops its list (flagged
// once) and the warp only counts its claims, which are all in the next-frontier bitmap.
template <typename OffT>
__device__ __forceinline__ bool keep_listing(const LevelIO<OffT>& io, Packed pk, int pending) {
  if (io.list_cap == kNoListCap) return true;
  unsigned long long c = 0;
  if ((threadIdx.x & 31) == 0) c = *(volatile unsigned long long*)io.counter_out;
  c = __shfl_sync(0xffffffffu, c, 0);
  const bool keep = pk.count(c) + pending <= io.list_cap;
  if (!keep && (threadIdx.x & 31) == 0) *(volatile unsigned*)io.dropped = 1u;
  return keep;
}

// The claims a warp counted without appending them, added to the list's count once, at the
// end of the warp's share of the level (one atomic per warp, not per tile).
template <typename OffT>
__device__ __forceinline__ void add_counted(const LevelIO<OffT>& io, Packed pk, long long counted) {
  if ((threadIdx.x & 31) == 0 && counted > 0) atomicAdd(io.counter_out, pk.make(counted, 0));
}

// Appends the CTA's buffered claims to the next frontier: one 64-bit atomic reserves the
// slots and the exclusive-scan range of their degrees (Sec. 3.4 scan, fused).
template <typename OffT, int BLOCK, int CLAIM>
__device__ __forceinline__ void flush_claims(const OffT* off, Packed pk, const LevelIO<OffT>& io, int2* s_claim,
                                             int nc, ExpandShared<OffT>& sh) {
  // Thread t owns the consecutive buffer items [t * P, t * P + P).
  constexpr int P = (CLAIM + BLOCK - 1) / BLOCK;
  const int lo = min(nc, (int)threadIdx.x * P), hi = min(nc, lo + P);
  OffT mine = 0;
  for (int i = lo; i < hi; ++i) mine += (OffT)s_claim[i].y;
  OffT total;
  OffT run = block_exclusive_scan(mine, sh.warp, &total);
  if (threadIdx.x == 0) sh.resv = atomicAdd(io.counter_out, pk.make(nc, (long long)total));
  __syncthreads();
  const unsigned long long resv = sh.resv;
  const long long slot0 = pk.count(resv);
  run += (OffT)pk.edges(resv);
  for (int t = 0; t < P; ++t) {  // uniform trip count: the descriptor writes are warp-collective
    const int i = lo + t;
    const bool valid = i < hi;
    OffT d = 0, b = 0;
    int32_t vc = 0;
    const int32_t slot = (int32_t)(slot0 + i);
    if (valid) {
      const int32_t v = s_claim[i].x;
      d = (OffT)s_claim[i].y;
      vc = io.old_id ? __ldg(io.old_id + v) : v;  // caller id (only ever written out as a parent)
      b = off[v] - run;
      io.out.v[slot] = vc;
      io.out.cum[slot] = run;
      io.out.base[slot] = b;
    }
    write_descs_warp(io.chunk_out, valid, run, d, slot, vc, b);
    run += d;
  }
}

// The CTA's buffered claims: appended (flush_claims) while the list stays within the cap of
// the frontier-bitmap mode, else only counted. Every thread of the CTA calls it.
template <typename OffT, int BLOCK, int CLAIM>
__device__ __forceinline__ void cta_flush_or_count(const OffT* off, Packed pk, const LevelIO<OffT>& io,
                                                   int2* s_claim, int nc, ExpandShared<OffT>& sh) {
  if (io.list_cap != kNoListCap) {
    if (threadIdx.x == 0) {
      const unsigned long long c = *(volatile unsigned long long*)io.counter_out;
      sh.klo = pk.count(c) + nc <= io.list_cap;
      if (!sh.klo) {
        *(volatile unsigned*)io.dropped = 1u;
        atomicAdd(io.counter_out, pk.make(nc, 0));
      }
    }
    __syncthreads();
    const bool listing = sh.klo != 0;
    __syncthreads();
    if (!listing) return;
  }
  flush_claims<OffT, BLOCK, CLAIM>(off, pk, io, s_claim, nc, sh);
}

// A claim buffered by a warp: everything the append needs, so that it reads nothing more
// from the graph: the vertex's caller id, its degree and its row offset off[v].
template <typename OffT>
struct ClaimRec {
  int32_t vc;
  int32_t deg;
  OffT o0;
};

// Appends a warp's buffered claims (buf[0..nc), nc <= 32 * P) to the next frontier with
// one 64-bit atomic for the warp: lane i owns items [i P, i P + P); a warp scan of the
// degrees gives each item its place in the next level's edge space.
template <typename OffT, int P>
__device__ __forceinline__ void warp_flush(Packed pk, const LevelIO<OffT>& io, const ClaimRec<OffT>* buf, int nc) {
  const int lane = threadIdx.x & 31;
  const int lo = min(nc, lane * P), hi = min(nc, lo + P);
  OffT mine = 0;
  for (int i = lo; i < hi; ++i) mine += (OffT)buf[i].deg;
  const OffT inc = warp_inclusive_scan(mine);
  const OffT total = __shfl_sync(0xffffffffu, inc, 31);
  unsigned long long resv = 0;
  if (lane == 0) resv = atomicAdd(io.counter_out, pk.make(nc, (long long)total));
  resv = __shfl_sync(0xffffffffu, resv, 0);
  const long long slot0 = pk.count(resv);
  OffT run = (OffT)pk.edges(resv) + inc - mine;
  for (int t = 0; t < P; ++t) {  // uniform trip count: the descriptor writes are warp-collective
    const int i = lo + t;
    const bool valid = i < hi;
    ClaimRec<OffT> c{0, 0, 0};
    if (valid) c = buf[i];
    const OffT d = (OffT)c.deg;
    const int32_t slot = (int32_t)(slot0 + i);
    const OffT b = c.o0 - run;
    if (valid) {
      io.out.v[slot] = c.vc;  // caller id (only ever written out as a parent)
      io.out.cum[slot] = run;
      io.out.base[slot] = b;
    }
    write_descs_warp(io.chunk_out, valid, run, d, slot, c.vc, b);
    run += d;
  }
  __syncwarp();
}

// Warp-aggregated push of this thread's claim (if any) into the CTA buffer.
__device__ __forceinline__ void push_claim(bool claimed, int32_t v, int32_t deg, int2* s_claim, int* nclaim) {
  const unsigned ball = __ballot_sync(0xffffffffu, claimed);
  if (ball) {
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(ball) - 1;
    int pos = 0;
    if (lane == leader) pos = atomicAdd(nclaim, __popc(ball));
    pos = __shfl_sync(0xffffffffu, pos, leader);
    if (claimed) s_claim[pos + __popc(ball & lanemask_lt())] = make_int2(v, deg);
  }
}

// One top-down level over tiles tile0, tile0 + tstride, ... of the level's edge space,
// followed by the final flush of the CTA's claims. Every thread of the CTA calls it.
template <typename OffT, int BLOCK, int E, int CLAIM>
__device__ void td_level(const OffT* __restrict__ off, const int32_t* __restrict__ cols, uint32_t* bitmap,
                         int64_t n, Packed pk, unsigned* err, const LevelIO<OffT>& io, unsigned char* dsmem,
                         ExpandShared<OffT>& sh, int64_t tile0, int64_t tstride) {
  using S = ExpandSmem<OffT, BLOCK, E, CLAIM>;
  constexpr int T = S::T;
  constexpr int CAP = S::CAP;
  static_assert(CLAIM >= T, "claim buffer must hold one full tile");
  OffT* s_base = reinterpret_cast<OffT*>(dsmem + S::off_base);
  int32_t* s_rel = reinterpret_cast<int32_t*>(dsmem + S::off_rel);
  int32_t* s_u = reinterpret_cast<int32_t*>(dsmem + S::off_u);
  int2* s_claim = reinterpret_cast<int2*>(dsmem + S::off_claim);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const OffT r = io.r;
  const int64_t nf = io.nf;
  const int64_t ntiles = ((int64_t)r + T - 1) / T;
  const int L = io.L;
  const int probe_mode = io.probe_mode;

  if (threadIdx.x == 0) sh.nclaim = 0;
  for (int64_t tile = tile0; tile < ntiles; tile += tstride) {
    const OffT e0 = (OffT)(tile * T);
    const int cnt = (int)min((OffT)T, r - e0);
    __syncthreads();  // the previous tile's shared-memory reads are done
    if (threadIdx.x == 0) {
      sh.klo = io.chunk_in[e0 / kChunk].k;
      sh.kend = (e0 + cnt < r) ? io.chunk_in[(e0 + cnt) / kChunk].k : (int32_t)(nf - 1);
    }
    __syncthreads();
    const int klo = sh.klo;
    const int kend = sh.kend;
    const int s = kend - klo + 1;
    const bool fast = s <= CAP;
    if (fast) {
      for (int i = threadIdx.x; i < s; i += BLOCK) {
        const OffT c = io.in.cum[klo + i];
        s_rel[i] = (int32_t)max(c - e0, (OffT)0);
        s_base[i] = io.in.base[klo + i];
        s_u[i] = io.in.v[klo + i];
      }
      if (threadIdx.x == 0) s_rel[s] = 0x7fffffff;  // sentinel
      __syncthreads();
    }

    // Thread -> edge mapping. Warp w owns tile edges [w * 32E, (w + 1) * 32E).
    int32_t vv[E], uu[E];
    OffT col[E];
    bool ok[E];
    {
      const int er0 = warp * 32 * E + lane;
      int k = 0;
      if (fast && er0 < cnt) k = binsearch_maxle(s_rel, 0, s, er0);
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int er = er0 + 32 * j;
        ok[j] = er < cnt;
        uu[j] = 0;
        col[j] = 0;
        if (ok[j]) {
          if (fast) {
            // linear walk (Sec. 3.4.1), with a bounded number of steps before a search
            int steps = 0;
            while (s_rel[k + 1] <= er && steps < 4) { ++k; ++steps; }
            if (s_rel[k + 1] <= er) k = binsearch_maxle(s_rel, k, s, er);
            col[j] = s_base[k] + e0 + er;
            uu[j] = s_u[k];
          } else {
            // many zero-degree frontier entries: search the global scan directly
            const OffT e = e0 + er;
            const int32_t kk = binsearch_maxle(io.in.cum, (int64_t)klo, (int64_t)kend + 1, e);
            col[j] = io.in.base[kk] + e;
            uu[j] = io.in.v[kk];
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < E; ++j) vv[j] = ok[j] ? ld_nc(cols + col[j]) : 0;
    uint32_t bits[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      if (ok[j] && (uint32_t)vv[j] >= (uint64_t)n) {
        atomicOr(err, kErrColumnRange);
        ok[j] = false;
      }
      bits[j] = ok[j] ? probe_load(bitmap + (vv[j] >> 5), probe_mode) : 0xffffffffu;
    }
    // Claims in phases so that the E atomics, then the E degree reads, are in flight
    // together instead of one round trip after another.
    bool claimed[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const uint32_t m = 1u << (vv[j] & 31);
      claimed[j] = !(bits[j] & m);
      if (claimed[j]) bits[j] = atomicOr(bitmap + (vv[j] >> 5), m);
    }
    OffT o0[E], o1[E];
    int32_t ov[E];  // caller id of the claimed vertex
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const uint32_t m = 1u << (vv[j] & 31);
      claimed[j] = claimed[j] && !(bits[j] & m);
      o0[j] = 0;
      o1[j] = 0;
      ov[j] = vv[j];
      if (claimed[j]) {
        o0[j] = off[vv[j]];
        o1[j] = off[vv[j] + 1];
        if (io.old_id) ov[j] = __ldg(io.old_id + vv[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < E; ++j) {
      if (claimed[j]) {
        io.levels[ov[j]] = L;
        io.parents[ov[j]] = uu[j];
        if (io.fbm_out) atomicOr(io.fbm_out + (vv[j] >> 5), 1u << (vv[j] & 31));
      }
    }
#pragma unroll
    for (int j = 0; j < E; ++j) push_claim(claimed[j], vv[j], (int32_t)(o1[j] - o0[j]), s_claim, &sh.nclaim);
    __syncthreads();
    const int nc = sh.nclaim;
    if (nc > CLAIM - T) {
      cta_flush_or_count<OffT, BLOCK, CLAIM>(off, pk, io, s_claim, nc, sh);
      __syncthreads();
      if (threadIdx.x == 0) sh.nclaim = 0;
    }
  }
  __syncthreads();
  const int nc = sh.nclaim;
  if (nc > 0) cta_flush_or_count<OffT, BLOCK, CLAIM>(off, pk, io, s_claim, nc, sh);
  __syncthreads();
}

// Shared state of one warp in the warp-tile variant of the top-down step.
template <typename OffT, int E, int WCAP>
struct WarpTileSmem {
  static constexpr int TW = 32 * E;  // edges per warp tile
  ClaimRec<OffT> claim[WCAP];        // claims, appended by the warp alone
};

// The top-down step with warp-sized tiles: warp w expands tiles w, w + W, ... of 32 E
// edges on its own, so no CTA-wide barrier is needed inside a level. The mapping of edge e
// to the frontier entry k = max{k : cum[k] <= e} (the binary search of Algorithm 3): a tile inside one row
// takes it from its descriptor; a tile over at most 32 entries holds them one per lane and
// finds k with a five-step binary search over the lanes (shuffles, no shared memory); a tile
// over more entries searches the global scan. The rest (column reads, pre-check, atomicOr
// claim, level / parent writes, fused append and degree scan) is the CTA-tile step's, with
// the claims appended through the warp's own buffer. Shared memory holds only that buffer,
// which leaves the most L1 to the bitmap probes.
template <typename OffT, int E, int WCAP>
__device__ void td_level_warp(const OffT* __restrict__ off, const int32_t* __restrict__ cols, uint32_t* bitmap,
                              int64_t n, Packed pk, unsigned* err, const LevelIO<OffT>& io,
                              WarpTileSmem<OffT, E, WCAP>& sm, int64_t tile0, int64_t tstride) {
  constexpr int TW = WarpTileSmem<OffT, E, WCAP>::TW;
  static_assert(TW % kChunk == 0, "warp tiles must start on chunk-index boundaries");
  static_assert(WCAP >= TW && WCAP % 32 == 0, "claim buffer must hold one full tile");
  constexpr int P = WCAP / 32;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const OffT r = io.r;
  const int64_t nf = io.nf;
  const int64_t ntiles = ((int64_t)r + TW - 1) / TW;
  const int L = io.L;
  const int probe_mode = io.probe_mode;
  int nc = 0;  // claims buffered (warp-uniform)
  // frontier-bitmap mode: appending until the list would pass the cap, then counting only
  bool listing = io.list_cap >= 0;
  long long counted = 0;
  // (Loading the next tile's entry range and staged entries one tile ahead was measured:
  // no faster, and slower once it made the kernel spill.)
  for (int64_t tile = tile0; tile < ntiles; tile += tstride) {
    const OffT e0 = (OffT)(tile * TW);
    const int cnt = (int)min((OffT)TW, r - e0);
    const TileDesc<OffT> d0 = io.chunk_in[e0 / kChunk];
    const int32_t klo = d0.k;
    const int32_t kend = (e0 + cnt < r) ? io.chunk_in[(e0 + cnt) / kChunk].k : (int32_t)(nf - 1);
    // A tile inside one row (the entry of its first edge also holds the edge after it)
    // needs no staging: its descriptor gives the column entry and the parent.
    const bool one_row = klo == kend;
    const int s = kend - klo + 1;
    // Up to 32 entries: lane i holds entry klo + i in registers (where its row starts in the
    // tile, its column base and caller id); no shared memory is used for staging.
    const bool fast = s <= 32;
    int32_t e_rel = 0x7fffffff, e_u = 0;
    OffT e_base = 0;
    if (fast && !one_row && lane < s) {
      const OffT c = io.in.cum[klo + lane];
      e_rel = (int32_t)max(c - e0, (OffT)0);  // entry klo starts at or before the tile
      e_base = io.in.base[klo + lane];
      e_u = io.in.v[klo + lane];
    }
    int32_t vv[E], uu[E];
    OffT col[E];
    bool ok[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int er = lane + 32 * j;
      ok[j] = er < cnt;
      uu[j] = 0;
      col[j] = 0;
      if (!one_row && fast) {
        // k = max{i : rel_i <= er} by a binary search over the lanes (rel_0 = 0 <= er)
        int k = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          const int rc = __shfl_sync(full, e_rel, k + step);
          if (rc <= er) k += step;
        }
        const OffT b = __shfl_sync(full, e_base, k);
        const int32_t u = __shfl_sync(full, e_u, k);
        col[j] = b + e0 + er;
        uu[j] = u;
      }
      if (ok[j]) {
        if (one_row) {
          col[j] = d0.col + er;
          uu[j] = d0.u;
        } else if (!fast) {
          // more than 32 entries (short rows): search the global scan directly
          const OffT e = e0 + er;
          const int32_t k = binsearch_maxle(io.in.cum, (int64_t)klo, (int64_t)kend + 1, e);
          col[j] = io.in.base[k] + e;
          uu[j] = io.in.v[k];
        }
      }
    }
    uint32_t bits[E];
    if constexpr (E <= 4) {
      // The loads of a tile take no branch: a lane past the tile's end reads column entry 0
      // and bitmap word 0 and drops what it read; the range check of the column ids is one
      // branch per tile. (Measured with 4 edges per thread: +1.7 % on R-MAT s26, +2 % on
      // uniform s26; with 8, 3 % slower than the per-edge branches below.)
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int32_t c = ld_nc(cols + (ok[j] ? col[j] : (OffT)0));
        vv[j] = ok[j] ? c : 0;
      }
      bool bad = false;
#pragma unroll
      for (int j = 0; j < E; ++j) bad |= (uint32_t)vv[j] >= (uint64_t)n;
      if (bad) {
        atomicOr(err, kErrColumnRange);
#pragma unroll
        for (int j = 0; j < E; ++j)
          if ((uint32_t)vv[j] >= (uint64_t)n) {
            ok[j] = false;
            vv[j] = 0;
          }
      }
      // Edges into the visited prefix [0, vis_below) need no pre-check: their lanes read the
      // (hot) bitmap word 0 instead and take the word as full.
      const uint32_t vb = io.vis_below;
#pragma unroll
      for (int j = 0; j < E; ++j) ok[j] = ok[j] && (uint32_t)vv[j] >= vb;
      if (probe_mode == 0) {
#pragma unroll
        for (int j = 0; j < E; ++j) bits[j] = probe_load(bitmap + (ok[j] ? (uint32_t)vv[j] >> 5 : 0u), 0);
      } else {
#pragma unroll
        for (int j = 0; j < E; ++j) bits[j] = probe_load(bitmap + (ok[j] ? (uint32_t)vv[j] >> 5 : 0u), 1);
      }
#pragma unroll
      for (int j = 0; j < E; ++j)
        if (!ok[j]) bits[j] = 0xffffffffu;
    } else {
#pragma unroll
      for (int j = 0; j < E; ++j) vv[j] = ok[j] ? ld_nc(cols + col[j]) : 0;
#pragma unroll
      for (int j = 0; j < E; ++j) {
        if (ok[j] && (uint32_t)vv[j] >= (uint64_t)n) {
          atomicOr(err, kErrColumnRange);
          ok[j] = false;
        }
        bits[j] = ok[j] ? probe_load(bitmap + (vv[j] >> 5), probe_mode) : 0xffffffffu;
      }
    }
    bool claimed[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const uint32_t m = 1u << (vv[j] & 31);
      claimed[j] = !(bits[j] & m);
      if (claimed[j]) bits[j] = atomicOr(bitmap + (vv[j] >> 5), m);
    }
    OffT o0[E], o1[E];
    int32_t ov[E];
    unsigned wc = 0;  // bit j: some lane of the warp claimed with edge j (warp-uniform)
    int tot = 0;      // claims of the warp in this tile
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const uint32_t m = 1u << (vv[j] & 31);
      claimed[j] = claimed[j] && !(bits[j] & m);
      const unsigned b = __ballot_sync(full, claimed[j]);
      if (b) wc |= 1u << j;
      tot += __popc(b);
    }
    // Room for this tile's claims first, while few registers are live. In frontier-bitmap
    // mode a full buffer past the list cap is counted instead of appended.
    if (listing && nc + tot > WCAP) {
      __syncwarp();
      if (keep_listing(io, pk, nc)) {
        warp_flush<OffT, P>(pk, io, sm.claim, nc);
      } else {
        listing = false;
        counted += nc;
      }
      nc = 0;
    }
    if (!listing) counted += tot;
    // Most edges of a large level find their vertex visited: the claim work below is
    // skipped by a warp-uniform branch wherever no lane of the warp claimed.
#pragma unroll
    for (int j = 0; j < E; ++j) {
      o0[j] = 0;
      o1[j] = 0;
      ov[j] = vv[j];
      if ((wc >> j) & 1u) {
        if (claimed[j]) {
          if (listing) {
            o0[j] = off[vv[j]];
            o1[j] = off[vv[j] + 1];
          }
          if (io.old_id) ov[j] = __ldg(io.old_id + vv[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < E; ++j) {
      if ((wc >> j) & 1u) {
        if (claimed[j]) {
          io.levels[ov[j]] = L;
          io.parents[ov[j]] = uu[j];
          if (io.fbm_out) atomicOr(io.fbm_out + (vv[j] >> 5), 1u << (vv[j] & 31));
        }
        if (listing) {
          const unsigned b = __ballot_sync(full, claimed[j]);
          if (claimed[j])
            sm.claim[nc + __popc(b & lanemask_lt())] = ClaimRec<OffT>{ov[j], (int32_t)(o1[j] - o0[j]), o0[j]};
          nc += __popc(b);
        }
      }
    }
  }
  __syncwarp();
  if (nc > 0) {
    if (keep_listing(io, pk, nc))
      warp_flush<OffT, P>(pk, io, sm.claim, nc);
    else
      counted += nc;
  }
  if (io.list_cap != kNoListCap) {
    if (io.list_cap < 0 && counted > 0 && (threadIdx.x & 31) == 0) *(volatile unsigned*)io.dropped = 1u;
    add_counted(io, pk, counted);
  }
}

// Frontier-bitmap unpack (the paper's warp-centric unpacking of a vertex bitmap into a
// list, Sec. 5): rounds of blockDim.x bitmap words per CTA, thread t taking word t of its
// round. A block scan of the words' vertex counts and degree sums gives each thread its
// place; one 64-bit atomicAdd per round on `counter` reserves the CTA's list slots and edge
// range (the same packed (count, edges) word as the expansion's appends), and the entries
// of a round are written in vertex order: id (caller numbering), scan value, column base and
// the tile descriptors of every kChunk-th edge, a warp-wide loop over the set bits. With
// `clear`, the words are zeroed as they are read. Every thread of the CTA calls it.
template <typename OffT>
__device__ void unpack_bitmap(const OffT* __restrict__ off, const int32_t* old_id, uint32_t* fbm, int64_t n,
                              Packed pk, FrontierBuf<OffT> out, TileDesc<OffT>* chunk_out,
                              unsigned long long* counter, bool clear, ExpandShared<OffT>& sh, int64_t round0,
                              int64_t rstride) {
  const int64_t nwords = (n + 31) / 32;
  const unsigned full = 0xffffffffu;
  for (int64_t round = round0; round * blockDim.x < nwords; round += rstride) {
    const int64_t w = round * blockDim.x + threadIdx.x;
    uint32_t word = 0;
    if (w < nwords) {
      word = fbm[w];
      if (clear && word) fbm[w] = 0u;
    }
    OffT cnt = (OffT)__popc(word), dsum = 0;
    for (uint32_t rem = word; rem; rem &= rem - 1) {
      const int64_t v = w * 32 + __ffs(rem) - 1;
      dsum += off[v + 1] - off[v];
    }
    OffT tot_cnt, tot_deg;
    const OffT ex_cnt = block_exclusive_scan(cnt, sh.warp, &tot_cnt);
    const OffT ex_deg = block_exclusive_scan(dsum, sh.warp, &tot_deg);
    if (tot_cnt == 0) continue;  // block-uniform
    if (threadIdx.x == 0) sh.resv = atomicAdd(counter, pk.make((long long)tot_cnt, (long long)tot_deg));
    __syncthreads();
    const unsigned long long resv = sh.resv;
    __syncthreads();
    int64_t slot = pk.count(resv) + (int64_t)ex_cnt;
    OffT run = (OffT)pk.edges(resv) + ex_deg;
    // uniform trip count per warp: the descriptor writes are warp-collective
    const int qmax = __reduce_max_sync(full, (unsigned)cnt);
    uint32_t rem = word;
    for (int q = 0; q < qmax; ++q) {
      const bool valid = rem != 0;
      int32_t v = 0, vc = 0;
      OffT d = 0, b = 0;
      if (valid) {
        v = (int32_t)(w * 32 + __ffs(rem) - 1);
        rem &= rem - 1;
        const OffT o0 = off[v];
        d = off[v + 1] - o0;
        vc = old_id ? __ldg(old_id + v) : v;
        b = o0 - run;
        out.v[slot] = vc;
        out.cum[slot] = run;
        out.base[slot] = b;
      }
      write_descs_warp(chunk_out, valid, run, d, (int32_t)slot, vc, b);
      if (valid) {
        ++slot;
        run += d;
      }
    }
  }
}

// Dynamic shared memory of an expansion shape: CTA tiles (staging + CTA claim buffer) or
// warp tiles (one WarpTileSmem per warp, CLAIM = claim entries per warp).
template <typename OffT, int BLOCK, int E, int CLAIM, bool WT>
struct ShapeSmem {
  static constexpr size_t bytes =
      WT ? (BLOCK / 32) * sizeof(WarpTileSmem<OffT, E, CLAIM>) : ExpandSmem<OffT, BLOCK, E, CLAIM>::bytes;
};

// TPS: resident threads per SM the registers are sized for (the launch bound).
template <typename OffT, int BLOCK, int E, int CLAIM, bool WT, int TPS>
__global__ void __launch_bounds__(BLOCK, TPS / BLOCK) k_expand(ExpandArgs<OffT> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ExpandShared<OffT> sh;
  Ctl* ctl = a.ctl;
  const int L = *(volatile int*)&ctl->level;
  const int cur = (L - 1) & 1, nxt = cur ^ 1;
  const unsigned long long pc = *(volatile unsigned long long*)&ctl->counter[cur];
  LevelIO<OffT> io;
  io.in = a.fr[cur];
  io.out = a.fr[nxt];
  io.chunk_in = a.chunk[cur];
  io.chunk_out = a.chunk[nxt];
  io.counter_out = &ctl->counter[nxt];
  io.levels = *(int32_t* volatile*)&ctl->levels;
  io.parents = *(int32_t* volatile*)&ctl->parents;
  io.fbm_out = a.fbm[nxt];  // NULL unless in frontier-bitmap mode
  io.L = L;
  io.probe_mode = a.probe_mode;
  io.old_id = a.old_id;
  io.nf = a.pk.count(pc);
  io.r = (OffT)a.pk.edges(pc);
  io.list_cap = a.fbm[nxt] ? a.list_cap : kNoListCap;
  io.dropped = &ctl->dropped;
  io.vis_below = 0;
  if constexpr (WT) {
    auto* wsm = reinterpret_cast<WarpTileSmem<OffT, E, CLAIM>*>(smem) + (threadIdx.x >> 5);
    td_level_warp<OffT, E, CLAIM>(a.off, a.cols, a.bitmap, a.n, a.pk, &ctl->error, io, *wsm,
                                  (int64_t)blockIdx.x * (BLOCK / 32) + (threadIdx.x >> 5),
                                  (int64_t)gridDim.x * (BLOCK / 32));
    __syncthreads();
  } else {
    td_level<OffT, BLOCK, E, CLAIM>(a.off, a.cols, a.bitmap, a.n, a.pk, &ctl->error, io, smem, sh, blockIdx.x,
                                    gridDim.x);
  }

  // Level epilogue by the last CTA to finish: close the level and prepare the next.
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(&ctl->done[cur], 1u);
    if (t == gridDim.x - 1) {
      __threadfence();
      const unsigned long long pn = atomicAdd(&ctl->counter[nxt], 0ull);
      const long long nn = a.pk.count(pn);
      ctl->edges2 += (long long)io.r;
      if (nn > 0) {
        ctl->depth += 1;
        ctl->reached += nn;
      }
      ctl->counter[cur] = 0;
      ctl->done[cur] = 0;
      ctl->level = L + 1;
      ctl->cont = nn > 0;
      ctl->bm_counter = 0;  // the unpack after this level, if the level dropped its list
      if (a.use_cond) cudaGraphSetConditional(a.cond, nn > 0 ? 1u : 0u);
    }
  }
}

// After an expansion in frontier-bitmap mode (graph or host loop): if the level dropped its
// list, rebuild the next frontier (list, scan, descriptors) from its bitmap, which is cleared
// on the way; else just clear the bitmap. The last CTA installs the rebuilt counter.
template <typename OffT>
__global__ void __launch_bounds__(256) k_unpack_level(ExpandArgs<OffT> a) {
  __shared__ ExpandShared<OffT> sh;
  Ctl* ctl = a.ctl;
  const int par = (*(volatile int*)&ctl->level - 1) & 1;  // parity of the next expansion's input
  uint32_t* fbm = a.fbm[par];
  const bool dropped = *(volatile unsigned*)&ctl->dropped != 0;
  if (dropped) {
    unpack_bitmap<OffT>(a.off, a.old_id, fbm, a.n, a.pk, a.fr[par], a.chunk[par], &ctl->bm_counter, true, sh,
                        blockIdx.x, gridDim.x);
  } else {
    const int64_t nwords = (a.n + 31) / 32;
    uint4* p = reinterpret_cast<uint4*>(fbm);
    const int64_t nv = nwords / 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x)
      p[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t i = nv * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
         i += (int64_t)gridDim.x * blockDim.x)
      fbm[i] = 0u;
    return;  // grid-uniform: no counter to install
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ctl->done[par], 1u) == gridDim.x - 1) {
      __threadfence();
      ctl->counter[par] = *(volatile unsigned long long*)&ctl->bm_counter;
      ctl->done[par] = 0;
      ctl->dropped = 0;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Persistent search: every level in one cooperative launch, with a grid barrier between
// levels and a per-level choice between the top-down step above and a bottom-up step.

// Grid barrier (sense reversal) with a bounded wait: after spin_limit polls the CTA records
// kErrTimeout and leaves; every CTA then stops at the next level boundary (all later waits
// are bounded too). A limit of 0 makes every arrival but the last give up at once. (A
// two-level arrival, CTAs counting in by groups of 32 on their own cache lines, was measured
// slower on 3D grids: 10 vs 9 us per level; the last arriver's extra dependent atomic costs
// more than the contention it removes.)
__device__ __forceinline__ void grid_barrier(PCtl* c, unsigned nblocks, long long spin_limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &c->bar_gen;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&c->bar_count, 1u);
    if (arrived == nblocks - 1) {
      c->bar_count = 0;
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      long long spins = 0;
      while (*gen == g) {
        if (++spins > spin_limit) {
          atomicOr(&c->error, kErrTimeout);
          break;
        }
        if (spins > 64) __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// One bottom-up level (Beamer et al.'s step, the paper's related work, Sec. 6): every
// unvisited vertex scans its row for a neighbour in the current frontier (a bitmap) and
// stops at the first. Warp w takes visited word w (32 vertices), so no atomics are needed
// on the visited and next-frontier bitmaps, and every warp appends its claimed vertices
// through its own slice of the claim buffer with a warp-level flush: warps never wait for
// one another inside the level. Claimed vertices enter the next frontier queue exactly as
// in the top-down step.
template <typename OffT, int WCAP>
__device__ void bu_level(const OffT* __restrict__ off, const int32_t* __restrict__ cols, uint32_t* bitmap,
                         const uint32_t* __restrict__ fbm_in, int64_t n, Packed pk, const LevelIO<OffT>& io,
                         ClaimRec<OffT>* wbuf, int64_t warp0, int64_t wstride) {
  static_assert(WCAP >= 64, "per-warp claim buffer too small");
  constexpr int P = (WCAP + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int64_t nwords = (n + 31) / 32;
  const int L = io.L;
  int nc = 0;  // warp-uniform
  for (int64_t w = warp0; w < nwords; w += wstride) {
    bool found = false;
    int32_t parent = 0, deg = 0;
    OffT b = 0;
    const uint32_t vis = bitmap[w];
    const int32_t v = (int32_t)(w * 32 + lane);
    if (v < n && !((vis >> lane) & 1u)) {
      b = off[v];
      const OffT e = off[v + 1];
      deg = (int32_t)(e - b);
      OffT i = b;
      for (; i + 4 <= e && !found; i += 4) {
        int32_t u4[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) u4[j] = __ldg(cols + i + j);  // one L1 fill for the four
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t u = (uint32_t)u4[j];
          if (!found && u < (uint64_t)n && ((fbm_in[u >> 5] >> (u & 31)) & 1u)) {
            found = true;
            parent = (int32_t)u;
          }
        }
      }
      for (; i < e && !found; ++i) {
        const uint32_t u = (uint32_t)__ldg(cols + i);
        if (u < (uint64_t)n && ((fbm_in[u >> 5] >> (u & 31)) & 1u)) {
          found = true;
          parent = (int32_t)u;
        }
      }
    }
    const unsigned claimed = __ballot_sync(0xffffffffu, found);
    if (claimed) {
      if (found) {
        const int32_t ov = io.old_id ? __ldg(io.old_id + v) : v;
        io.levels[ov] = L;
        io.parents[ov] = io.old_id ? __ldg(io.old_id + parent) : parent;
        wbuf[nc + __popc(claimed & lanemask_lt())] = ClaimRec<OffT>{ov, deg, b};
      }
      if (lane == 0) {
        bitmap[w] = vis | claimed;
        io.fbm_out[w] = claimed;
      }
      nc += __popc(claimed);
      __syncwarp();
      if (nc > WCAP - 32) {
        warp_flush<OffT, P>(pk, io, wbuf, nc);
        nc = 0;
      }
    }
  }
  if (nc > 0) warp_flush<OffT, P>(pk, io, wbuf, nc);
  __syncthreads();
}

// WITH_BU = false compiles the top-down-only variant (fewer registers, more resident CTAs).
template <typename OffT, int BLOCK, int E, int CLAIM, bool WITH_BU, bool WT, int TPS>
__global__ void __launch_bounds__(BLOCK, (WITH_BU && TPS > 1024 ? 1024 : TPS) / BLOCK)
    k_bfs_persistent(PersistArgs<OffT> a) {
  using S = ExpandSmem<OffT, BLOCK, E, CLAIM>;
  using W = WarpTileSmem<OffT, E, CLAIM>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ExpandShared<OffT> sh;
  PCtl* c = a.ctl;
  const int warp = threadIdx.x >> 5;
  W* wsm = reinterpret_cast<W*>(smem) + warp;
  // bottom-up claim buffer of this warp: its warp-tile buffer, or its slice of the CTA's
  constexpr int BU_WCAP = WT ? CLAIM : (int)(CLAIM * sizeof(int2) / sizeof(ClaimRec<OffT>)) / (BLOCK / 32);
  ClaimRec<OffT>* bu_buf =
      WT ? wsm->claim : reinterpret_cast<ClaimRec<OffT>*>(smem + S::off_claim) + warp * BU_WCAP;
  const int64_t nwords = (a.n + 31) / 32;
  const int64_t gtid = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * BLOCK;
  long long seen_deg = 0;          // degree sum of every frontier so far (same on all CTAs)
  long long prev_nf = 0;
  bool bottom_up = false;
  __shared__ long long s_nf, s_r;
  __shared__ int s_stop;
  __shared__ unsigned s_pfx;
  int64_t pfx_w = 0;  // bitmap words [0, pfx_w) are full (same on all CTAs)
  for (int it = 0;; ++it) {
    const int cur3 = it % 3, nxt3 = (it + 1) % 3, old3 = (it + 2) % 3;
    // Loop control is read once per CTA and broadcast, so that every thread of the CTA takes
    // the same path even when a barrier wait has expired and other CTAs are still writing.
    if (threadIdx.x == 0) {
      const unsigned long long pc = *(volatile unsigned long long*)&c->counter[cur3];
      s_nf = a.pk.count(pc);
      s_r = a.pk.edges(pc);
      s_stop = s_nf == 0 || (*(volatile unsigned*)&c->error & kErrTimeout) != 0;
    }
    __syncthreads();
    const long long nf = s_nf;
    const long long r = s_r;
    if (s_stop) break;
    seen_deg += r;
    // direction choice (Beamer's heuristic): bottom-up while the frontier's edges are a
    // large share of the unexplored ones, back to top-down once the frontier shrinks
    const long long unexplored = a.nnz - seen_deg + r;
    if (WITH_BU && a.allow_bottom_up) {
      if (!bottom_up)
        bottom_up = r * (long long)a.alpha > unexplored && nf > prev_nf;
      else
        bottom_up = !(nf * (long long)a.beta < a.n && nf < prev_nf);
    }
    prev_nf = nf;
    const bool keep_fbm = WITH_BU || a.bitmap_mode;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      c->counter[old3] = 0;
      c->steps_bottom_up += bottom_up ? 1 : 0;
      c->dropped[nxt3] = 0;     // for level it + 1 (last read before level it - 1 ended)
      c->bm_counter[nxt3] = 0;
      c->pfx[nxt3] = 0xffffffffu;
    }
    // Visited prefix of a relabelled graph: its vertices are numbered by falling degree, and
    // by the large levels the highest-degree ones are all visited (R-MAT s22: the first
    // 110 K-300 K of 4.2 M at the dominant level, which sends 73-87 % of its edges there).
    // On a level of at least n edges every thread checks one bitmap word past the last
    // prefix, each CTA a block of consecutive words; the first word not full, over all CTAs,
    // ends the prefix. Costs one grid barrier on the few large levels.
    if (a.old_id && !(WITH_BU && bottom_up) && r >= a.n) {  // grid-uniform
      if (threadIdx.x == 0) s_pfx = 0xffffffffu;
      __syncthreads();
      for (int64_t w0 = pfx_w + (int64_t)blockIdx.x * BLOCK; w0 < nwords; w0 += gstride) {
        const int64_t w = w0 + threadIdx.x;
        const bool open = w < nwords && __ldcg(a.bitmap + w) != 0xffffffffu;
        if (open) atomicMin(&s_pfx, (unsigned)w);
        if (__syncthreads_or(open)) break;  // block-uniform
      }
      if (threadIdx.x == 0 && s_pfx != 0xffffffffu) atomicMin(&c->pfx[cur3], s_pfx);
      grid_barrier(c, gridDim.x, a.spin_limit);
      if (threadIdx.x == 0) s_pfx = *(volatile unsigned*)&c->pfx[cur3];
      __syncthreads();
      pfx_w = s_pfx == 0xffffffffu ? nwords : (int64_t)s_pfx;
    }
    if (keep_fbm)
      for (int64_t w = gtid; w < nwords; w += gstride) a.fbm[old3][w] = 0u;  // collects level it + 2
    LevelIO<OffT> io;
    io.in = a.fr[it & 1];
    io.out = a.fr[(it + 1) & 1];
    io.chunk_in = a.chunk[it & 1];
    io.chunk_out = a.chunk[(it + 1) & 1];
    io.counter_out = &c->counter[nxt3];
    io.levels = a.levels;
    io.parents = a.parents;
    io.fbm_out = keep_fbm ? a.fbm[nxt3] : nullptr;
    io.L = it + 1;
    io.probe_mode = a.probe_mode;
    io.old_id = a.old_id;
    io.nf = nf;
    io.r = (OffT)r;
    io.list_cap = (a.bitmap_mode && !bottom_up) ? a.list_cap : kNoListCap;
    io.dropped = &c->dropped[cur3];
    io.vis_below = (uint32_t)min(pfx_w * 32, (int64_t)a.n);
    if (WITH_BU && bottom_up)
      bu_level<OffT, BU_WCAP>(a.off, a.cols, a.bitmap, a.fbm[cur3], a.n, a.pk, io, bu_buf,
                              (int64_t)blockIdx.x * (BLOCK / 32) + warp, (int64_t)gridDim.x * (BLOCK / 32));
    else if constexpr (WT)
      td_level_warp<OffT, E, CLAIM>(a.off, a.cols, a.bitmap, a.n, a.pk, &c->error, io, *wsm,
                                    (int64_t)blockIdx.x * (BLOCK / 32) + warp, (int64_t)gridDim.x * (BLOCK / 32));
    else
      td_level<OffT, BLOCK, E, CLAIM>(a.off, a.cols, a.bitmap, a.n, a.pk, &c->error, io, smem, sh, blockIdx.x,
                                      gridDim.x);
    grid_barrier(c, gridDim.x, a.spin_limit);
    if (a.bitmap_mode) {
      // the level dropped its list: rebuild it from the next-frontier bitmap (kept: a
      // bottom-up level reads it), then every CTA installs the rebuilt counter
      if (threadIdx.x == 0) s_stop = *(volatile unsigned*)&c->dropped[cur3] != 0;
      __syncthreads();
      if (s_stop) {
        unpack_bitmap<OffT>(a.off, a.old_id, a.fbm[nxt3], a.n, a.pk, a.fr[(it + 1) & 1], a.chunk[(it + 1) & 1],
                            &c->bm_counter[cur3], false, sh, blockIdx.x, gridDim.x);
        grid_barrier(c, gridDim.x, a.spin_limit);
        if (threadIdx.x == 0) c->counter[nxt3] = *(volatile unsigned long long*)&c->bm_counter[cur3];
        if (blockIdx.x == 0 && threadIdx.x == 0) c->unpacked_levels += 1;
      }
      __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (it < kMaxLevelTimes) {
        unsigned long long ns;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ns));
        c->level_ns[it] = ns;
        c->level_bu[it] = bottom_up ? 1 : 0;
        c->level_nf[it] = nf;
      }
      const long long nn = a.pk.count(*(volatile unsigned long long*)&c->counter[nxt3]);
      c->edges2 += r;
      if (nn > 0) {
        c->depth += 1;
        c->reached += nn;
      }
    }
  }
}

template <typename OffT>
__global__ void k_init_persist(const OffT* __restrict__ off, int64_t n, int32_t root, const int32_t* new_id,
                               int32_t* levels, int32_t* parents, uint32_t* bitmap, uint32_t* fbm0, uint32_t* fbm1,
                               uint32_t* fbm2, FrontierBuf<OffT> f0, TileDesc<OffT>* chunk0, PCtl* c, Packed pk) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += stride) {  // outputs are indexed by caller ids
    const bool is_root = i == root;
    levels[i] = is_root ? 0 : -1;
    parents[i] = is_root ? root : -1;
  }
  const int32_t rn = new_id ? new_id[root] : root;  // the root's internal id
  const int64_t nw = (n + 31) / 32;
  for (int64_t w = tid; w < nw; w += stride) {
    const uint32_t rb = (w == (rn >> 5)) ? (1u << (rn & 31)) : 0u;
    bitmap[w] = rb;
    fbm0[w] = rb;
    fbm1[w] = 0u;
    fbm2[w] = 0u;
  }
  const OffT o0 = off[rn], deg = off[rn + 1] - o0;
  const int64_t nchunks = ((int64_t)deg + kChunk - 1) / kChunk;
  for (int64_t ch = tid; ch < nchunks; ch += stride) chunk0[ch] = TileDesc<OffT>{0, root, o0 + (OffT)(ch * kChunk)};
  if (tid == 0) {
    f0.v[0] = root;  // the queue holds caller ids
    f0.cum[0] = 0;
    f0.base[0] = o0;
    c->counter[0] = pk.make(1, (long long)deg);
    c->counter[1] = 0;
    c->counter[2] = 0;
    c->bar_count = 0;
    c->bar_gen = 0;
    c->error = 0;
    c->depth = 1;
    c->reached = 1;
    c->edges2 = 0;
    c->steps_bottom_up = 0;
    c->unpacked_levels = 0;
    for (int i = 0; i < 3; ++i) {
      c->bm_counter[i] = 0;
      c->dropped[i] = 0;
      c->pfx[i] = 0xffffffffu;
    }
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(c->start_ns));
  }
}

__global__ void k_write_count(const Ctl* ctl, Packed pk, int64_t* out) {
  // after an expansion the next frontier's counter sits at parity 1 (level-1 parity 0)
  const int nxt = ((ctl->level - 2) & 1) ^ 1;
  *out = pk.count(ctl->counter[nxt]);
}

// ---------------------------------------------------------------------------------------
// Host-side launchers

void launch_write_count(Ctl* ctl, Packed pk, int64_t* out, cudaStream_t st) {
  k_write_count<<<1, 1, 0, st>>>(ctl, pk, out);
}

template <typename OffT>
void launch_init_single(const GraphDev& g, int32_t root, int32_t* levels, int32_t* parents, SingleWs& ws,
                        cudaStream_t st, bool clear_fbm) {
  const int block = 256;
  const int grid = g.num_sms * 8;
  k_init_single<OffT><<<grid, block, 0, st>>>(reinterpret_cast<const OffT*>(g.off), g.n, root, g.new_id, levels,
                                               parents, ws.bitmap, ws.fr<OffT>(0), ws.desc<OffT>(0), ws.ctl, g.pk,
                                               clear_fbm ? ws.fbm[0] : nullptr, clear_fbm ? ws.fbm[1] : nullptr);
}

template <typename OffT>
void launch_unpack_level(const GraphDev& g, const ExpandArgs<OffT>& a, cudaStream_t st) {
  k_unpack_level<OffT><<<g.num_sms * 4, 256, 0, st>>>(a);
}

// Unpack of a caller's bitmap into the workspace frontier of parity `par` (bfs_expand_bitmap):
// the vertex list is copied out to `next` and its length to *count_dev.
template <typename OffT>
__global__ void __launch_bounds__(256) k_unpack_caller(const OffT* __restrict__ off, uint32_t* bitmap, int64_t n,
                                                       Packed pk, FrontierBuf<OffT> out, TileDesc<OffT>* chunk,
                                                       unsigned long long* counter) {
  __shared__ ExpandShared<OffT> sh;
  unpack_bitmap<OffT>(off, nullptr, bitmap, n, pk, out, chunk, counter, false, sh, blockIdx.x, gridDim.x);
}

__global__ void k_count_out(const unsigned long long* counter, Packed pk, int64_t* out) {
  *out = pk.count(*counter);
}

template <typename OffT>
cudaError_t unpack_bitmap_to_list(const GraphDev& g, SingleWs& ws, int par, const uint32_t* bitmap, int32_t* next,
                                  int64_t* count_dev, cudaStream_t st) {
  unsigned long long* counter = &ws.ctl->bm_counter;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  k_unpack_caller<OffT><<<g.num_sms * 4, 256, 0, st>>>(reinterpret_cast<const OffT*>(g.off),
                                                        const_cast<uint32_t*>(bitmap), g.n, g.pk, ws.fr<OffT>(par),
                                                        ws.desc<OffT>(par), counter);
  k_count_out<<<1, 1, 0, st>>>(counter, g.pk, count_dev);
  int64_t count = 0;
  if ((e = cudaMemcpyAsync(&count, count_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return e;
  if (count > 0 && (e = cudaMemcpyAsync(next, ws.v[par], sizeof(int32_t) * (size_t)count, cudaMemcpyDeviceToDevice,
                                        st)) != cudaSuccess)
    return e;
  return cudaStreamSynchronize(st);
}

template <typename OffT>
void launch_scan_frontier(const GraphDev& g, const int32_t* front, int64_t nf, int32_t level, int32_t* levels,
                          int32_t* parents, SingleWs& ws, cudaStream_t st) {
  const OffT* off = reinterpret_cast<const OffT*>(g.off);
  const int cur = (level - 1) & 1;  // the expansion of `level` reads buffer parity cur
  cudaMemsetAsync(&ws.ctl->error, 0, sizeof(unsigned), st);
  const int parts = ws.scan_parts;
  OffT* partial = reinterpret_cast<OffT*>(ws.scan_partial);
  k_scan_partials<OffT><<<parts, 256, 0, st>>>(off, g.n, front, nf, partial, ws.ctl);
  const long long max_edges = std::min<long long>((long long)g.pk.mask, (ws.chunk_cap - 1) * (long long)kChunk);
  k_scan_top<OffT><<<1, 1024, 0, st>>>(partial, parts, nf, ws.ctl, g.pk, level, levels, parents, max_edges);
  k_scan_final<OffT><<<parts, 256, 0, st>>>(off, g.n, front, nf, partial, ws.fr<OffT>(cur), ws.desc<OffT>(cur),
                                            ws.ctl);
}

// Sets a kernel's dynamic shared memory size and the smallest shared-memory carveout that
// keeps the CTAs per SM its registers and warps allow, so that the rest of the SM's 256 KB
// is L1 for the visited-bitmap probes (the driver otherwise picks a larger carveout than the
// warp tiles' small claim buffers need). Returns the CTAs per SM.
template <typename K>
static int fit_carveout(K kern, int block, size_t dyn_bytes) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_bytes);
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  int full = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&full, kern, block, dyn_bytes) != cudaSuccess || full < 1) {
    cudaGetLastError();
    return 1;
  }
  cudaFuncAttributes fa{};
  int dev = 0, smem_sm = 0;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      smem_sm <= 0) {
    cudaGetLastError();
    return full;
  }
  const size_t need = (size_t)full * (dyn_bytes + fa.sharedSizeBytes + 1024);  // 1 KB reserved per CTA
  const int pct = (int)std::min<size_t>(100, std::max<size_t>(1, (need * 100 + smem_sm - 1) / smem_sm));
  int got = 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&got, kern, block, dyn_bytes) != cudaSuccess || got < full) {
    cudaGetLastError();
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return full;
  }
  return got;
}

template <typename OffT, int BLOCK, int E, int CLAIM, bool WT, int TPS>
static cudaError_t launch_expand_t(const ExpandArgs<OffT>& a, int grid, cudaStream_t st) {
  constexpr size_t bytes = ShapeSmem<OffT, BLOCK, E, CLAIM, WT>::bytes;
  auto kern = k_expand<OffT, BLOCK, E, CLAIM, WT, TPS>;
  static bool attr_set = false;  // per template instance; set once per process
  if (!attr_set) {
    fit_carveout(kern, BLOCK, bytes);
    attr_set = true;
  }
  kern<<<grid, BLOCK, bytes, st>>>(a);
  return cudaGetLastError();
}

template <typename OffT, int BLOCK, int E, int CLAIM, bool WT, int TPS>
static int occupancy_t(int num_sms) {
  constexpr size_t bytes = ShapeSmem<OffT, BLOCK, E, CLAIM, WT>::bytes;
  return fit_carveout(k_expand<OffT, BLOCK, E, CLAIM, WT, TPS>, BLOCK, bytes) * num_sms;
}

// Table of compiled shapes (BLOCK, E, CLAIM, tiles, TPS): tiles 0 = one tile of BLOCK x E
// edges per CTA (CLAIM = CTA claim buffer), 1 = one tile of 32 x E edges per warp (CLAIM =
// claim buffer per warp); TPS = resident threads per SM the registers are sized for. The
// autotuner chooses among them.
#define GBFS_EXPAND_SHAPES(X)  \
  X(0, 256, 4, 2048, 0, 1536)  \
  X(1, 256, 4, 1536, 0, 1536)  \
  X(2, 256, 2, 1024, 0, 1536)  \
  X(3, 128, 4, 1024, 0, 1536)  \
  X(4, 128, 4, 128, 1, 1536)   \
  X(5, 128, 4, 128, 1, 1024)   \
  X(6, 128, 8, 256, 1, 1024)   \
  X(7, 128, 4, 128, 1, 1280)   \
  X(8, 128, 4, 256, 1, 1280)   \
  X(9, 512, 4, 128, 1, 1024)

const ExpandShape kExpandShapes[] = {
#define X(id, b, e, c, w, t) {id, b, e, c, w},
    GBFS_EXPAND_SHAPES(X)
#undef X
};
const int kNumExpandShapes = sizeof(kExpandShapes) / sizeof(kExpandShapes[0]);

template <typename OffT, int BLOCK, int E, int CLAIM, bool WT, int TPS>
static cudaError_t launch_persistent_t(const PersistArgs<OffT>& a, int grid, cudaStream_t st) {
  constexpr size_t bytes = ShapeSmem<OffT, BLOCK, E, CLAIM, WT>::bytes;
  auto kern = a.allow_bottom_up ? k_bfs_persistent<OffT, BLOCK, E, CLAIM, true, WT, TPS>
                                : k_bfs_persistent<OffT, BLOCK, E, CLAIM, false, WT, TPS>;
  static bool attr_set[2] = {false, false};
  if (!attr_set[a.allow_bottom_up ? 1 : 0]) {
    fit_carveout(kern, BLOCK, bytes);  // the same settings the grid size was computed under
    attr_set[a.allow_bottom_up ? 1 : 0] = true;
  }
  PersistArgs<OffT> copy = a;
  void* params[] = {&copy};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kern), dim3(grid), dim3(BLOCK), params, bytes, st);
}

// All CTAs of a cooperative launch must be resident at once: occupancy x SMs.
template <typename OffT, int BLOCK, int E, int CLAIM, bool WT, int TPS>
static int persistent_grid_t(int num_sms, bool with_bu) {
  constexpr size_t bytes = ShapeSmem<OffT, BLOCK, E, CLAIM, WT>::bytes;
  auto kern = with_bu ? k_bfs_persistent<OffT, BLOCK, E, CLAIM, true, WT, TPS>
                      : k_bfs_persistent<OffT, BLOCK, E, CLAIM, false, WT, TPS>;
  return fit_carveout(kern, BLOCK, bytes) * num_sms;
}

template <typename OffT>
cudaError_t launch_persistent(int shape, const PersistArgs<OffT>& a, int grid, cudaStream_t st) {
  switch (shape) {
#define X(id, b, e, c, w, t) \
  case id: return launch_persistent_t<OffT, b, e, c, w != 0, t>(a, grid, st);
    GBFS_EXPAND_SHAPES(X)
#undef X
  }
  return cudaErrorInvalidValue;
}

template <typename OffT>
int persistent_grid(int shape, int num_sms, bool with_bu) {
  switch (shape) {
#define X(id, b, e, c, w, t) \
  case id: return persistent_grid_t<OffT, b, e, c, w != 0, t>(num_sms, with_bu);
    GBFS_EXPAND_SHAPES(X)
#undef X
  }
  return num_sms;
}

template <typename OffT>
void launch_init_persist(const GraphDev& g, int32_t root, int32_t* levels, int32_t* parents, SingleWs& ws,
                         cudaStream_t st) {
  k_init_persist<OffT><<<g.num_sms * 8, 256, 0, st>>>(reinterpret_cast<const OffT*>(g.off), g.n, root, g.new_id,
                                                      levels, parents, ws.bitmap, ws.fbm[0], ws.fbm[1], ws.fbm[2],
                                                      ws.fr<OffT>(0), ws.desc<OffT>(0), ws.pctl, g.pk);
}

template <typename OffT>
cudaError_t launch_expand(int shape, const ExpandArgs<OffT>& a, int grid, cudaStream_t st) {
  switch (shape) {
#define X(id, b, e, c, w, t) \
  case id: return launch_expand_t<OffT, b, e, c, w != 0, t>(a, grid, st);
    GBFS_EXPAND_SHAPES(X)
#undef X
  }
  return cudaErrorInvalidValue;
}

template <typename OffT>
int expand_grid(int shape, int num_sms) {
  switch (shape) {
#define X(id, b, e, c, w, t) \
  case id: return occupancy_t<OffT, b, e, c, w != 0, t>(num_sms);
    GBFS_EXPAND_SHAPES(X)
#undef X
  }
  return num_sms;
}

template void launch_init_single<int32_t>(const GraphDev&, int32_t, int32_t*, int32_t*, SingleWs&, cudaStream_t, bool);
template void launch_init_single<int64_t>(const GraphDev&, int32_t, int32_t*, int32_t*, SingleWs&, cudaStream_t, bool);
template void launch_unpack_level<int32_t>(const GraphDev&, const ExpandArgs<int32_t>&, cudaStream_t);
template void launch_unpack_level<int64_t>(const GraphDev&, const ExpandArgs<int64_t>&, cudaStream_t);
template cudaError_t unpack_bitmap_to_list<int32_t>(const GraphDev&, SingleWs&, int, const uint32_t*, int32_t*,
                                                    int64_t*, cudaStream_t);
template cudaError_t unpack_bitmap_to_list<int64_t>(const GraphDev&, SingleWs&, int, const uint32_t*, int32_t*,
                                                    int64_t*, cudaStream_t);
template void launch_scan_frontier<int32_t>(const GraphDev&, const int32_t*, int64_t, int32_t, int32_t*,
                                            int32_t*, SingleWs&, cudaStream_t);
template void launch_scan_frontier<int64_t>(const GraphDev&, const int32_t*, int64_t, int32_t, int32_t*,
                                            int32_t*, SingleWs&, cudaStream_t);
template cudaError_t launch_expand<int32_t>(int, const ExpandArgs<int32_t>&, int, cudaStream_t);
template cudaError_t launch_expand<int64_t>(int, const ExpandArgs<int64_t>&, int, cudaStream_t);
template int expand_grid<int32_t>(int, int);
template int expand_grid<int64_t>(int, int);
template cudaError_t launch_persistent<int32_t>(int, const PersistArgs<int32_t>&, int, cudaStream_t);
template cudaError_t launch_persistent<int64_t>(int, const PersistArgs<int64_t>&, int, cudaStream_t);
template int persistent_grid<int32_t>(int, int, bool);
template int persistent_grid<int64_t>(int, int, bool);
template void launch_init_persist<int32_t>(const GraphDev&, int32_t, int32_t*, int32_t*, SingleWs&, cudaStream_t);
template void launch_init_persist<int64_t>(const GraphDev&, int32_t, int32_t*, int32_t*, SingleWs&, cudaStream_t);

}  // namespace gbfs
