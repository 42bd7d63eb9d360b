// Multi-source BFS kernels: up to 64 searches advance together, one bit per root in a
// 64-bit visited mask V[v] and in per-frontier masks F_t[v]. The frontier of a wave is the
// list of vertices with F_t[v] != 0; each of their rows is read once per level and serves
// every root that has the vertex in its frontier. Per edge (u, v):
//     new = F_t[u] & ~V[v];  old = atomicOr(&V[v], new);  claimed = new & ~old
// (Algorithm 3's visited test and claim, one bit per root); for every claimed bit b the
// level and parent of (b, v) are written (Algorithm 3's output writes), and v joins frontier
// t + 1 when atomicOr(&F_{t+1}[v], claimed) returns 0 (first touch), through the same
// buffered append with the fused degree scan as the single-source kernel. Thread-to-edge
// mapping is the single-source one (Sec. 3.4 and 3.4.1). The paper has no batched form;
// batching multiplies the work done per column read.
#include <cuda_runtime.h>

#include "batch.h"
#include "batch_append.cuh"
#include "batch_order.cuh"
#include "common.cuh"
#include "device_util.cuh"
#include "kernels.h"

namespace gbfs {

__global__ void k_fill(int32_t* p, int64_t count, int32_t value) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const bool aligned = (reinterpret_cast<uintptr_t>(p) & 15) == 0;
  if (aligned) {
    int4* q = reinterpret_cast<int4*>(p);
    const int64_t nv = count / 4;
    const int4 val = make_int4(value, value, value, value);
    for (int64_t i = tid; i < nv; i += stride) q[i] = val;
    for (int64_t i = nv * 4 + tid; i < count; i += stride) p[i] = value;
  } else {
    for (int64_t i = tid; i < count; i += stride) p[i] = value;
  }
}

void launch_fill(int32_t* p, int64_t count, int32_t value, int num_sms, cudaStream_t st) {
  if (count > 0) k_fill<<<num_sms * 8, 256, 0, st>>>(p, count, value);
}

template <typename OffT>
__global__ void k_batch_clear(BatchArgs<OffT> a) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = tid; v < a.n; v += stride) {
    a.visited[v] = 0ull;
    a.fmask[0][v] = 0ull;
    a.fmask[1][v] = 0ull;
    a.fmask[2][v] = 0ull;
    a.evc[v] = 0;
    a.fmark[v] = 0;
    if (a.dense_idx) a.dense_idx[v] = -1;
  }
  if (a.dense_idx || a.dense_ident)
    for (int64_t r = tid; r < a.dense_cap; r += stride) a.dense_mask[r] = 0ull;
  if (a.done)
    for (int64_t w = tid; w < (a.n + 31) / 32; w += stride) a.done[w] = 0u;
  if (tid == 0) {
    a.ctl->ovf_count = 0;
    a.ctl->emit_done = 0;
    a.ctl->dense_count = 0;
    a.ctl->recorded = 0;
  }
}

template <typename OffT>
void launch_batch_clear(const BatchArgs<OffT>& a, int num_sms, cudaStream_t st) {
  k_batch_clear<OffT><<<num_sms * 8, 256, 0, st>>>(a);
}

__global__ void k_clear_bits(unsigned long long* visited, int64_t n, unsigned long long keep) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = tid; v < n; v += stride) {
    const unsigned long long x = visited[v];
    if (x & ~keep) visited[v] = x & keep;
  }
}

void launch_clear_bits(unsigned long long* visited, int64_t n, unsigned long long mask, int num_sms,
                       cudaStream_t st) {
  if (mask) k_clear_bits<<<num_sms * 8, 256, 0, st>>>(visited, n, ~mask);
}

// Adds roots to the frontier the next expansion will read (frontier t = level - 1). With
// fresh != 0 a new wave starts at frontier 0. Thread 0 places the (at most 64) roots; then
// the block writes the chunk index of their rows (a hub root's row spans many chunks).
template <typename OffT>
__global__ void k_batch_seed(BatchArgs<OffT> a, const RootSeed* seeds, int n_seeds, int fresh) {
  __shared__ OffT s_cum[kMaxWave], s_deg[kMaxWave], s_base[kMaxWave];
  __shared__ int32_t s_k[kMaxWave], s_v[kMaxWave];
  __shared__ int s_new, s_cur;
  if (threadIdx.x == 0) {
    BatchCtl* c = a.ctl;
    if (fresh) {
      c->counter[0] = c->counter[1] = 0;
      c->done[0] = c->done[1] = 0;
      c->level = 1;
      c->cont = 1;
      c->prev_count = 0;
      c->error = 0;
      c->alive[0] = c->alive[1] = 0;
      c->bu = 0;
      c->bu_levels = 0;
      c->seen = 0;
      for (int b = 0; b < kMaxWave; ++b) c->bitcnt[b] = 0ull;
    }
    const int t = c->level - 1;
    const int cur = t & 1, q3 = t % 3;
    long long cnt = a.pk.count(c->counter[cur]);
    long long e = a.pk.edges(c->counter[cur]);
    const WaveSlots* sl = a.slots;
    int added = 0;
    for (int i = 0; i < n_seeds; ++i) {
      const int32_t vc = seeds[i].v;                  // caller id (indexes the outputs)
      const int32_t v = a.new_id ? a.new_id[vc] : vc;  // internal id
      const unsigned long long m = seeds[i].mask;
      c->alive[cur] |= m;  // roots with a frontier (bottom-up levels look for these bits)
      a.visited[v] |= m;
      const unsigned long long old = a.fmask[q3][v];
      a.fmask[q3][v] = old | m;
      for (unsigned long long bits = m; bits; bits &= bits - 1) {
        const int b = __ffsll((long long)bits) - 1;
        sl->lvl[b][vc] = 0;
        sl->par[b][vc] = vc;
      }
      if (old == 0) {
        const OffT o = a.off[v], d = a.off[v + 1] - o;
        a.qv[q3][cnt] = v;
        a.cum[cur][cnt] = (OffT)e;
        a.base[cur][cnt] = o - (OffT)e;
        s_cum[added] = (OffT)e;
        s_deg[added] = d;
        s_base[added] = o - (OffT)e;
        s_k[added] = (int32_t)cnt;
        s_v[added] = v;
        ++added;
        ++cnt;
        e += (long long)d;
      }
    }
    c->counter[cur] = a.pk.make(cnt, e);
    c->cont = cnt > 0;
    s_new = added;
    s_cur = cur;
  }
  __syncthreads();
  TileDesc<OffT>* chunk = a.chunk[s_cur];
  for (int r = 0; r < s_new; ++r) {
    const OffT c0 = (s_cum[r] + kChunk - 1) / kChunk, c1 = (s_cum[r] + s_deg[r] + kChunk - 1) / kChunk;
    for (OffT ch = c0 + (OffT)threadIdx.x; ch < c1; ch += (OffT)blockDim.x)
      chunk[ch] = TileDesc<OffT>{s_k[r], s_v[r], s_base[r] + ch * (OffT)kChunk};
  }
}

template <typename OffT>
void launch_batch_seed(const BatchArgs<OffT>& a, const RootSeed* seeds_dev, int n_seeds, int wave_level,
                       bool fresh, cudaStream_t st) {
  (void)wave_level;
  k_batch_seed<OffT><<<1, 256, 0, st>>>(a, seeds_dev, n_seeds, fresh ? 1 : 0);
}

template <typename OffT, int BLOCK, int E, int CLAIM>
struct BatchSmem {
  static constexpr int T = BLOCK * E;
  static constexpr int CAP = T + 1;
  static constexpr size_t off_f = 0;  // uint64 masks first (8-byte aligned)
  static constexpr size_t off_base = off_f + 8 * CAP;
  static constexpr size_t off_rel = off_base + sizeof(OffT) * CAP;
  static constexpr size_t off_u = off_rel + 4 * (CAP + 1);
  static constexpr size_t off_claim = ((off_u + 4 * CAP) + 15) & ~size_t(15);
  static constexpr size_t bytes = off_claim + sizeof(int2) * CLAIM;
};

constexpr unsigned long long kSmallFrontierDiv = 16384;

// One bottom-up level of a wave (the multi-source form of Beamer's step, the paper's
// related work, Sec. 6): every vertex v still missing some active root's bit scans its row
// and takes, from each neighbour u, the bits of F_t[u] it still needs (each bit's parent is
// the first u that has it), stopping once it has them all. No atomics: each vertex is
// owned by one lane (warp w takes vertices 32 w ... 32 w + 31). Claims become parent events
// and next-frontier entries exactly as in the top-down step, so the emit kernel writes the
// outputs in both cases.
template <typename OffT, int WCAP>
__device__ void batch_bu_level(const BatchArgs<OffT>& a, const unsigned long long* __restrict__ F,
                               unsigned long long* Fn, unsigned long long active, int nxt, int q3n, int2* wbuf,
                               int32_t* const* s_par, int32_t* const* s_lvl, const int32_t* s_start, int L,
                               unsigned long long* s_alive, int* s_rec) {
  static_assert(WCAP >= 64, "per-warp claim buffer too small");
  constexpr int P = (WCAP + 31) / 32;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * wpb;
  int nc = 0;  // warp-uniform
  unsigned long long mine = 0ull;
  bool rec = false;  // this thread wrote a claim record
  for (int64_t w = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); w * 32 < a.n; w += nwarps) {
    const int64_t x = w * 32 + lane;
    const int32_t v = (int32_t)x;
    unsigned long long acc = 0ull;
    int32_t deg = 0;
    if (x < a.n) {
      const unsigned long long need = active & ~a.visited[v];
      if (need) {
        const OffT b = a.off[v], e = a.off[v + 1];
        deg = (int32_t)(e - b);
        int nev = a.defer ? a.evc[v] : 0;  // this lane owns v: no other writer this level
        for (OffT i = b; i < e && acc != need; ++i) {
          const uint32_t u = (uint32_t)__ldg(a.cols + i);
          if (u >= (uint64_t)a.n) {
            atomicOr(&a.ctl->error, kErrColumnRange);
            continue;
          }
          const unsigned long long f = F[u] & need & ~acc;
          if (f) {
            acc |= f;
            const int32_t uc = a.old_id ? __ldg(a.old_id + u) : (int32_t)u;
            rec |= record_claim(a, v, f, uc, L, nev, s_par, s_lvl, s_start);
            if (!single_bit(f)) ++nev;
          }
        }
        if (acc) {  // this lane owns v: plain stores
          a.visited[v] |= acc;
          Fn[v] = acc;
          a.evc[v] = nev;
          mine |= acc;
        }
      }
    }
    const bool claimed = acc != 0ull;
    const unsigned ball = __ballot_sync(full, claimed);
    if (ball) {
      if (nc + __popc(ball) > WCAP) {
        __syncwarp();
        batch_warp_flush<OffT, P>(a, nxt, q3n, wbuf, nc);
        nc = 0;
      }
      if (claimed) wbuf[nc + __popc(ball & lanemask_lt())] = make_int2(v, deg);
      nc += __popc(ball);
    }
  }
  __syncwarp();
  if (nc > 0) batch_warp_flush<OffT, P>(a, nxt, q3n, wbuf, nc);
  if (mine) atomicOr(s_alive, mine);
  if (rec) *s_rec = 1;
}

// The top-down step of a wave with warp-sized tiles (the batched form of the single-source
// warp tiles): warp w expands tiles w, w + W, ... of 32 E edges on its own, so no CTA-wide
// barrier is needed inside a level. Edge e's frontier entry k = max{k : cum[k] <= e}
// (the binary search of Algorithm 3): a tile inside one row takes it from its tile descriptor; a tile
// over at most 32 entries holds them one per lane (row start in the tile, column base,
// caller id, frontier mask) and searches them with shuffles; a tile over more entries
// searches the scan. Per edge (u, v): new = F_t[u] & ~V[v], claimed = new & ~atomicOr(V[v],
// new); each claim records a parent event, and the first claim of v in this level appends v
// to frontier t + 1 through the warp's claim buffer.
template <typename OffT, int E, int WCAP, bool DONE>
__device__ void batch_td_warp(const BatchArgs<OffT>& a, int L, int cur, int nxt, int q3, int q3n, int64_t nf,
                              OffT r, int2* wbuf, int32_t* const* s_par, int32_t* const* s_lvl,
                              const int32_t* s_start, unsigned long long* s_alive, int* s_rec) {
  constexpr int TW = 32 * E;
  static_assert(TW % kChunk == 0, "warp tiles must start on chunk-index boundaries");
  static_assert(WCAP >= TW && WCAP % 32 == 0, "claim buffer must hold one full tile");
  constexpr int P = WCAP / 32;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  BatchCtl* ctl = a.ctl;
  const unsigned long long* F = a.fmask[q3];
  unsigned long long* Fn = a.fmask[q3n];
  const int32_t* qv = a.qv[q3];
  const OffT* cum = a.cum[cur];
  const OffT* basep = a.base[cur];
  const TileDesc<OffT>* din = a.chunk[cur];
  const int64_t ntiles = ((int64_t)r + TW - 1) / TW;
  const int64_t wpb = blockDim.x >> 5;
  int nc = 0;  // warp-uniform
  unsigned long long mine = 0ull;
  bool rec = false;  // this thread wrote a claim record
  // Done marks (waves whose roots all start at level 0): the roots still searching are those
  // of frontier t; a vertex whose visited mask holds all of them can never be claimed again
  // (the set only shrinks), so its mask is not read. A missing mark only costs the read.
  const bool ordered = wave_ordered(a, nf);  // no appends: the next frontier is rebuilt in vertex order
  const bool marks = ordered && a.order_marks;  // ... from byte marks
  uint32_t* done = DONE ? a.done : nullptr;
  const unsigned long long act = DONE ? *(volatile unsigned long long*)&ctl->alive[cur] : 0ull;
  for (int64_t tile = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); tile < ntiles; tile += (int64_t)gridDim.x * wpb) {
    const OffT e0 = (OffT)(tile * TW);
    const int cnt = (int)min((OffT)TW, r - e0);
    const TileDesc<OffT> d0 = din[e0 / kChunk];
    const int32_t klo = d0.k;
    const int32_t kend = (e0 + cnt < r) ? din[(e0 + cnt) / kChunk].k : (int32_t)(nf - 1);
    const bool one_row = klo == kend;
    const int s = kend - klo + 1;
    const bool fast = s <= 32;
    // entry data: the row's (one_row, same on every lane) or entry klo + lane's
    int32_t e_rel = 0x7fffffff, e_u = 0;
    OffT e_base = 0;
    unsigned long long e_f = 0ull;
    if (one_row) {
      e_f = F[d0.u];
      e_u = a.old_id ? __ldg(a.old_id + d0.u) : d0.u;
    } else if (fast && lane < s) {
      const int32_t u = qv[klo + lane];
      e_rel = (int32_t)max(cum[klo + lane] - e0, (OffT)0);  // entry klo starts at or before the tile
      e_base = basep[klo + lane];
      e_f = F[u];
      e_u = a.old_id ? __ldg(a.old_id + u) : u;
    }
    int32_t vv[E], uu[E];
    unsigned long long ff[E];
    OffT col[E];
    bool ok[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int er = lane + 32 * j;
      ok[j] = er < cnt;
      uu[j] = e_u;
      ff[j] = e_f;
      col[j] = d0.col + er;
      if (!one_row && fast) {
        // k = max{i : rel_i <= er} by a binary search over the lanes (rel_0 = 0 <= er)
        int k = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          const int rc = __shfl_sync(full, e_rel, k + step);
          if (rc <= er) k += step;
        }
        col[j] = __shfl_sync(full, e_base, k) + e0 + er;
        uu[j] = __shfl_sync(full, e_u, k);
        ff[j] = __shfl_sync(full, e_f, k);
      }
      if (ok[j] && !one_row && !fast) {
        // more than 32 entries (short rows): search the scan directly
        const OffT e = e0 + er;
        const int32_t kk = binsearch_maxle(cum, (int64_t)klo, (int64_t)kend + 1, e);
        const int32_t u = qv[kk];
        col[j] = basep[kk] + e;
        uu[j] = a.old_id ? __ldg(a.old_id + u) : u;
        ff[j] = F[u];
      }
    }
#pragma unroll
    for (int j = 0; j < E; ++j) vv[j] = ok[j] ? ld_nc(a.cols + col[j]) : 0;
    unsigned long long nb[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      if (ok[j] && (uint32_t)vv[j] >= (uint64_t)a.n) {
        atomicOr(&ctl->error, kErrColumnRange);
        ok[j] = false;
      }
      if constexpr (DONE) {
        // a vertex marked done holds every searching root's bit: no 64-bit visited-mask read
        // (the marks are read from L2, so that one set during the level is seen at once)
        if (ok[j] && ((__ldcg(done + ((uint32_t)vv[j] >> 5)) >> (vv[j] & 31)) & 1u)) ok[j] = false;
        const unsigned long long vm = ok[j] ? a.visited[vv[j]] : ~0ull;
        nb[j] = ff[j] & ~vm;
        // complete but not yet marked (its last bit came at an earlier level): mark it
        if (ok[j] && (vm & act) == act) atomicOr(done + ((uint32_t)vv[j] >> 5), 1u << (vv[j] & 31));
      } else {
        nb[j] = ok[j] ? (ff[j] & ~a.visited[vv[j]]) : 0ull;
      }
    }
    unsigned long long claimed[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      claimed[j] = 0ull;
      if (nb[j]) {
        const unsigned long long old = atomicOr(a.visited + vv[j], nb[j]);
        claimed[j] = nb[j] & ~old;
        if (DONE && ((old | nb[j]) & act) == act) atomicOr(done + ((uint32_t)vv[j] >> 5), 1u << (vv[j] & 31));
      }
    }
    unsigned wc = 0;  // bit j: some lane of the warp claimed with edge j (warp-uniform)
#pragma unroll
    for (int j = 0; j < E; ++j)
      if (__ballot_sync(full, claimed[j] != 0ull)) wc |= 1u << j;
    if (!wc) continue;  // most edges of a large level find every bit taken
    int slot[E];
    unsigned long long fold[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      slot[j] = 0;
      fold[j] = 1ull;
      if (claimed[j]) {
        if (!single_bit(claimed[j])) slot[j] = atomicAdd(a.evc + vv[j], 1);
        fold[j] = atomicOr(Fn + vv[j], claimed[j]);
      }
    }
    bool first[E];
    int32_t deg[E];
    int tot = 0;
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int32_t v = vv[j];
      const bool fresh = claimed[j] && fold[j] == 0ull;  // v enters the next frontier with this claim
      if (fresh && marks) a.fmark[v] = 1;
      first[j] = fresh && !ordered;  // ordered: k_batch_order lists it
      deg[j] = first[j] ? (int32_t)(a.off[v + 1] - a.off[v]) : 0;
      tot += __popc(__ballot_sync(full, first[j]));
      if (claimed[j]) {
        mine |= claimed[j];
        // parent record: the outputs are written after the wave (or the level) from it
        rec |= record_claim(a, v, claimed[j], uu[j], L, slot[j], s_par, s_lvl, s_start);
      }
    }
    if (nc + tot > WCAP) {
      __syncwarp();
      batch_warp_flush<OffT, P>(a, nxt, q3n, wbuf, nc);
      nc = 0;
    }
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const unsigned b = __ballot_sync(full, first[j]);
      if (first[j]) wbuf[nc + __popc(b & lanemask_lt())] = make_int2(vv[j], deg[j]);
      nc += __popc(b);
    }
  }
  __syncwarp();
  if (nc > 0) batch_warp_flush<OffT, P>(a, nxt, q3n, wbuf, nc);
  // OR of the lanes' claimed bits, one shared atomic per warp
  unsigned lo = __reduce_or_sync(full, (unsigned)mine), hi = __reduce_or_sync(full, (unsigned)(mine >> 32));
  if (lane == 0 && (lo | hi)) atomicOr(s_alive, ((unsigned long long)hi << 32) | lo);
  if (rec) *s_rec = 1;
}

// TPS: resident threads per SM the registers are sized for (0: the compiler's choice).
template <typename OffT, int BLOCK, int E, int CLAIM, bool WT, int TPS>
__global__ void __launch_bounds__(BLOCK, TPS / BLOCK) k_expand_batch(BatchArgs<OffT> a) {
  using S = BatchSmem<OffT, BLOCK, E, CLAIM>;
  constexpr int T = S::T, CAP = S::CAP;
  static_assert(WT || CLAIM >= T, "claim buffer must hold one full tile");
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* s_f = reinterpret_cast<unsigned long long*>(smem + S::off_f);
  OffT* s_base = reinterpret_cast<OffT*>(smem + S::off_base);
  int32_t* s_rel = reinterpret_cast<int32_t*>(smem + S::off_rel);
  int32_t* s_u = reinterpret_cast<int32_t*>(smem + S::off_u);
  // claim buffers: the CTA's (CTA tiles), or CLAIM entries per warp (warp tiles)
  int2* s_claim = reinterpret_cast<int2*>(smem + (WT ? 0 : S::off_claim));
  __shared__ int32_t* s_lvl[kMaxWave];
  __shared__ int32_t* s_par[kMaxWave];
  __shared__ int32_t s_start[kMaxWave];
  __shared__ OffT s_warp[33];
  __shared__ unsigned long long s_resv, s_alive;
  __shared__ int s_nclaim, s_klo, s_kend, s_rec;

  BatchCtl* ctl = a.ctl;
  const int L = *(volatile int*)&ctl->level;
  const int t = L - 1;
  const int cur = t & 1, nxt = cur ^ 1, q3 = t % 3, q3n = (t + 1) % 3, q3p = (t + 2) % 3;
  const unsigned long long pc = *(volatile unsigned long long*)&ctl->counter[cur];
  const int64_t nf = a.pk.count(pc);
  const OffT r = (OffT)a.pk.edges(pc);
  const long long prev = *(volatile long long*)&ctl->prev_count;
  const bool ordered = wave_ordered(a, nf);  // no appends: the next frontier is rebuilt in vertex order
  const bool marks = ordered && a.order_marks;  // ... from byte marks
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < kMaxWave) {
    s_lvl[threadIdx.x] = a.slots->lvl[threadIdx.x];
    s_par[threadIdx.x] = a.slots->par[threadIdx.x];
    s_start[threadIdx.x] = a.slots->start[threadIdx.x];
  }
  if (threadIdx.x == 0) {
    s_nclaim = 0;
    s_alive = 0ull;
    s_rec = 0;
  }
  // Frontier t - 1 is no longer read by anyone: clear its masks so that the buffer can
  // collect frontier t + 2.
  {
    const int64_t tid = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * BLOCK;
    for (int64_t k = tid; k < prev; k += stride) a.fmask[q3p][a.qv[q3p][k]] = 0ull;
  }
  const unsigned long long* F = a.fmask[q3];
  unsigned long long* Fn = a.fmask[q3n];
  const int32_t* qv = a.qv[q3];
  const OffT* cum = a.cum[cur];
  const OffT* basep = a.base[cur];
  const TileDesc<OffT>* chunk_in = a.chunk[cur];
  const int64_t ntiles = ((int64_t)r + T - 1) / T;
  const int bu = a.allow_bu ? *(volatile int*)&ctl->bu : 0;  // chosen when the previous level closed

  constexpr int WCAP = WT ? CLAIM : CLAIM / (BLOCK / 32);  // claim entries per warp
  if (bu) {
    __syncthreads();  // slot pointers staged
    batch_bu_level<OffT, WCAP>(a, F, Fn, *(volatile unsigned long long*)&ctl->alive[cur], nxt, q3n,
                               s_claim + warp * WCAP, s_par, s_lvl, s_start, L, &s_alive, &s_rec);
  } else if constexpr (WT) {
    __syncthreads();  // slot pointers staged
    if (a.done)  // grid-uniform
      batch_td_warp<OffT, E, WCAP, true>(a, L, cur, nxt, q3, q3n, nf, r, s_claim + warp * WCAP, s_par, s_lvl,
                                         s_start, &s_alive, &s_rec);
    else
      batch_td_warp<OffT, E, WCAP, false>(a, L, cur, nxt, q3, q3n, nf, r, s_claim + warp * WCAP, s_par, s_lvl,
                                          s_start, &s_alive, &s_rec);
  }
  bool rec = false;  // this thread wrote a claim record (CTA tiles)
  for (int64_t tile = (bu || WT) ? ntiles : (int64_t)blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const OffT e0 = (OffT)(tile * T);
    const int cnt = (int)min((OffT)T, r - e0);
    __syncthreads();
    if (threadIdx.x == 0) {
      s_klo = chunk_in[e0 / kChunk].k;
      s_kend = (e0 + cnt < r) ? chunk_in[(e0 + cnt) / kChunk].k : (int32_t)(nf - 1);
    }
    __syncthreads();
    const int klo = s_klo;
    const int s = s_kend - klo + 1;
    const bool fast = s <= CAP;
    if (fast) {
      for (int i = threadIdx.x; i < s; i += BLOCK) {
        const int32_t u = qv[klo + i];
        s_rel[i] = (int32_t)max(cum[klo + i] - e0, (OffT)0);
        s_base[i] = basep[klo + i];
        s_u[i] = a.old_id ? __ldg(a.old_id + u) : u;  // only ever written out as a parent
        s_f[i] = F[u];
      }
      if (threadIdx.x == 0) s_rel[s] = 0x7fffffff;
      __syncthreads();
    }
    int32_t vv[E], uu[E];
    unsigned long long ff[E];
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
        ff[j] = 0ull;
        col[j] = 0;
        if (ok[j]) {
          if (fast) {
            int steps = 0;
            while (s_rel[k + 1] <= er && steps < 4) { ++k; ++steps; }
            if (s_rel[k + 1] <= er) k = binsearch_maxle(s_rel, k, s, er);
            col[j] = s_base[k] + e0 + er;
            uu[j] = s_u[k];
            ff[j] = s_f[k];
          } else {
            const OffT e = e0 + er;
            const int32_t kk = binsearch_maxle(cum, (int64_t)klo, (int64_t)s_kend + 1, e);
            col[j] = basep[kk] + e;
            const int32_t u = qv[kk];
            uu[j] = a.old_id ? __ldg(a.old_id + u) : u;
            ff[j] = F[u];
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < E; ++j) vv[j] = ok[j] ? ld_nc(a.cols + col[j]) : 0;
    unsigned long long nb[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      if (ok[j] && (uint32_t)vv[j] >= (uint64_t)a.n) {
        atomicOr(&ctl->error, kErrColumnRange);
        ok[j] = false;
      }
      nb[j] = ok[j] ? (ff[j] & ~a.visited[vv[j]]) : 0ull;
    }
    // Claims in phases, so that each kind of atomic / load is in flight for all E edges at
    // once rather than one round trip after another.
    unsigned long long claimed[E];
#pragma unroll
    for (int j = 0; j < E; ++j) claimed[j] = nb[j] ? nb[j] & ~atomicOr(a.visited + vv[j], nb[j]) : 0ull;
    int slot[E];
    unsigned long long fold[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      slot[j] = 0;
      fold[j] = 1ull;
      if (claimed[j]) {
        if (!single_bit(claimed[j])) slot[j] = atomicAdd(a.evc + vv[j], 1);
        fold[j] = atomicOr(Fn + vv[j], claimed[j]);
      }
    }
    unsigned long long mine = 0ull;
    bool first[E];
    OffT o0[E], o1[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int32_t v = vv[j];
      const bool fresh = claimed[j] && fold[j] == 0ull;  // v enters the next frontier with this claim
      if (fresh && marks) a.fmark[v] = 1;
      first[j] = fresh && !ordered;  // ordered: k_batch_order lists it
      o0[j] = 0;
      o1[j] = 0;
      if (first[j]) {
        o0[j] = a.off[v];
        o1[j] = a.off[v + 1];
      }
      if (claimed[j]) {
        mine |= claimed[j];
        // parent record: the outputs are written after the wave (or the level) from it
        rec |= record_claim(a, v, claimed[j], uu[j], L, slot[j], s_par, s_lvl, s_start);
      }
    }
    if (mine) atomicOr(&s_alive, mine);
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const unsigned ball = __ballot_sync(0xffffffffu, first[j]);
      if (ball) {
        const int leader = __ffs(ball) - 1;
        int pos = 0;
        if (lane == leader) pos = atomicAdd(&s_nclaim, __popc(ball));
        pos = __shfl_sync(0xffffffffu, pos, leader);
        if (first[j]) s_claim[pos + __popc(ball & lanemask_lt())] = make_int2(vv[j], (int32_t)(o1[j] - o0[j]));
      }
    }
    __syncthreads();
    const int nc = s_nclaim;
    if (nc > CLAIM - T) {
      batch_flush<OffT, BLOCK, CLAIM>(a, nxt, q3n, s_claim, nc, s_warp, &s_resv);
      __syncthreads();
      if (threadIdx.x == 0) s_nclaim = 0;
    }
  }
  if (rec) s_rec = 1;
  __syncthreads();
  const int nc = bu ? 0 : s_nclaim;
  if (nc > 0) batch_flush<OffT, BLOCK, CLAIM>(a, nxt, q3n, s_claim, nc, s_warp, &s_resv);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_alive) atomicOr(&ctl->alive[nxt], s_alive);
    if (s_rec) *(volatile unsigned*)&ctl->recorded = 1u;
    __threadfence();
    const unsigned tdone = atomicAdd(&ctl->done[cur], 1u);
    if (tdone == gridDim.x - 1) {
      __threadfence();
      const unsigned long long pn = atomicAdd(&ctl->counter[nxt], 0ull);
      const long long nn = a.pk.count(pn);
      if (a.allow_bu) {
        // direction of the next level (Beamer's heuristic on the wave's union frontier):
        // bottom-up while the next frontier's edges are a large share of the unexplored
        // ones and it grows, top-down again once it is small and shrinking
        const long long seen = ctl->seen + (long long)r;
        const long long rn = a.pk.edges(pn);
        const long long unexplored = a.nnz - seen;
        ctl->seen = seen;
        ctl->bu_levels += bu;
        ctl->bu = bu ? !(nn * (long long)a.beta < a.n && nn < nf) : (rn * (long long)a.alpha > unexplored && nn > nf);
        ctl->bu_strict = ctl->bu && rn > unexplored;  // the rule when some root's frontier is small
      }
      ctl->prev_count = nf;
      ctl->counter[cur] = 0;
      ctl->done[cur] = 0;
      ctl->alive[cur] = 0;
      ctl->level = L + 1;
      // an ordered expansion appended nothing: the next frontier exists if some root claimed
      const bool more = ordered ? *(volatile unsigned long long*)&ctl->alive[nxt] != 0ull : nn > 0;
      ctl->cont = more;
      if (a.use_cond) cudaGraphSetConditional(a.cond, more ? 1u : 0u);
    }
  }
}

// After the expansion of frontier t (wave level L = t + 1): for every vertex v claimed in
// it, F_{t+1}[v] holds the bits claimed and the per-vertex records hold the claimers of
// claims of several bits (single-bit claims were written at claim time). Their levels
// (L - start[b]) and parents are written in vertex order: a warp takes 32 consecutive
// vertices and loops over the union of their recorded bits, so each store covers 32
// consecutive entries of one root's row. When few vertices were claimed the vertices come
// from the next frontier list instead (scattered, cheaper than a full pass). Records that
// did not fit the per-vertex slots are applied last; the last CTA resets the overflow count.
// COUNT_ONLY (waves with deferred outputs and bottom-up levels allowed): only the per-root
// frontier sizes and the direction choice; no output writes, and the events stay.
template <typename OffT, bool COUNT_ONLY>
__global__ void __launch_bounds__(256) k_batch_emit(BatchArgs<OffT> a) {
  __shared__ int32_t* s_lvl[kMaxWave];
  __shared__ int32_t* s_par[kMaxWave];
  __shared__ int32_t s_start[kMaxWave];
  __shared__ unsigned long long s_cnt[kMaxWave];
  BatchCtl* ctl = a.ctl;
  // Nothing to write when the level's claims were all written at claim time (single root
  // bits, the rule on grids) and there is no direction choice to make: every CTA sees the
  // same words, so the whole grid leaves.
  if (!COUNT_ONLY && !a.allow_bu && !*(volatile unsigned*)&ctl->recorded &&
      !*(volatile unsigned long long*)&ctl->ovf_count)
    return;
  const int Lnext = *(volatile int*)&ctl->level;  // already advanced by the expansion
  const int L = Lnext - 1;
  const int t = L - 1;
  const int nxt = (t & 1) ^ 1, q3n = (t + 1) % 3;
  const long long nn = a.pk.count(*(volatile unsigned long long*)&ctl->counter[nxt]);
  if (threadIdx.x < kMaxWave) {
    s_lvl[threadIdx.x] = a.slots->lvl[threadIdx.x];
    s_par[threadIdx.x] = a.slots->par[threadIdx.x];
    s_start[threadIdx.x] = a.slots->start[threadIdx.x];
    s_cnt[threadIdx.x] = 0ull;
  }
  __syncthreads();
  const unsigned long long* Fn = a.fmask[q3n];
  const int lane = threadIdx.x & 31;
  // per-root sizes of the new frontier (only needed to choose bottom-up levels): lane l
  // counts roots l and l + 32
  unsigned long long cnt_lo = 0ull, cnt_hi = 0ull;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool ordered = !COUNT_ONLY && nn * 8 > a.n;  // a full pass pays only when many vertices were claimed
  const int64_t items = ordered ? (a.n + 31) / 32 : (nn + 31) / 32;
  for (int64_t w = gwarp; w < items; w += nwarps) {
    int32_t v = -1, vc = -1;  // internal id (masks, events) and caller id (outputs)
    if (ordered) {  // consecutive caller ids: coalesced output rows
      const int64_t x = w * 32 + lane;
      if (x < a.n) {
        vc = (int32_t)x;
        v = a.new_id ? __ldg(a.new_id + vc) : vc;
      }
    } else {
      const int64_t k = w * 32 + lane;
      if (k < nn) {
        v = a.qv[q3n][k];
        vc = a.old_id ? __ldg(a.old_id + v) : v;
      }
    }
    const unsigned long long f = v >= 0 ? Fn[v] : 0ull;
    int ne = 0;
    int32_t eu[kEventSlots];
    unsigned long long em[kEventSlots];
    unsigned long long evb = 0ull;  // bits with a record (the others were written at claim time)
    if (f && !COUNT_ONLY) {
      ne = min(a.evc[v], kEventSlots);
#pragma unroll
      for (int k = 0; k < kEventSlots; ++k) {
        if (k < ne) {
          const ClaimEvent ce = a.ev[(size_t)v * a.ev_slots + k];
          eu[k] = ce.u;
          em[k] = ce.mask;
          evb |= ce.mask;
        } else {
          eu[k] = 0;
          em[k] = 0ull;
        }
      }
      if (ne) a.evc[v] = 0;
    }
    const unsigned long long want = a.allow_bu ? f : evb;  // bits the loop below visits
    const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)want);
    const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(want >> 32));
    unsigned long long any = ((unsigned long long)hi << 32) | lo;
    while (any) {
      const int b = __ffsll((long long)any) - 1;
      any &= any - 1;
      if (a.allow_bu) {
        const unsigned c = __popc(__ballot_sync(0xffffffffu, (f >> b) & 1ull));
        if (lane == (b & 31)) (b < 32 ? cnt_lo : cnt_hi) += c;
      }
      if (!COUNT_ONLY && ((evb >> b) & 1ull)) {
        s_lvl[b][vc] = L - s_start[b];
#pragma unroll
        for (int k = 0; k < kEventSlots; ++k)
          if ((em[k] >> b) & 1ull) s_par[b][vc] = eu[k];
      }
    }
  }
  // overflow records (after every slot record of the level is consumed above)
  const long long novf =
      COUNT_ONLY ? 0 : min((long long)*(volatile unsigned long long*)&ctl->ovf_count, a.ovf_cap);
  for (long long o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < novf; o += (int64_t)gridDim.x * blockDim.x) {
    const OvfEvent e = a.ovf[o];
    for (unsigned long long bits = e.mask; bits; bits &= bits - 1) {
      const int b = __ffsll((long long)bits) - 1;
      s_lvl[b][e.v] = e.level - s_start[b];
      s_par[b][e.v] = e.u;
    }
  }
  if (a.allow_bu) {
    if (cnt_lo) atomicAdd(&s_cnt[lane], cnt_lo);
    if (cnt_hi) atomicAdd(&s_cnt[lane + 32], cnt_hi);
  }
  __syncthreads();
  if (a.allow_bu && threadIdx.x < kMaxWave && s_cnt[threadIdx.x])
    atomicAdd(&ctl->bitcnt[threadIdx.x], s_cnt[threadIdx.x]);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ctl->emit_done, 1u) == gridDim.x - 1) {
      __threadfence();
      if (!COUNT_ONLY) {
        ctl->ovf_count = 0;  // with deferred outputs the overflow list lasts the wave
        ctl->recorded = 0;
      }
      ctl->emit_done = 0;
      if (a.allow_bu) {
        // A bottom-up level makes every vertex look for the bits of every active root, so a
        // root with a small frontier (one in a small component, say) makes nearly every row
        // be scanned to its end, which costs about the unexplored edges: with such a root
        // (under n / kSmallFrontierDiv vertices), go bottom-up only if the frontier's edges
        // exceed the unexplored ones. (Swept on R-MAT s22 / s24 and uniform waves: 1/16384
        // kept the uniform and most of the R-MAT gain and removed a 3.5x loss on waves with
        // roots in small components; 1/64 and 1/1024 gave up more.)
        const unsigned long long m = *(volatile unsigned long long*)&ctl->alive[nxt];
        bool small = false;
        for (unsigned long long bits = m; bits; bits &= bits - 1)
          small |= ctl->bitcnt[__ffsll((long long)bits) - 1] * kSmallFrontierDiv < (unsigned long long)a.n;
        if (small) ctl->bu = ctl->bu_strict;
        for (int b = 0; b < kMaxWave; ++b) ctl->bitcnt[b] = 0ull;
      }
    }
  }
}

template <typename OffT>
void launch_batch_emit(const BatchArgs<OffT>& a, int num_sms, cudaStream_t st) {
  k_batch_emit<OffT, false><<<num_sms * 8, 256, 0, st>>>(a);
}

template <typename OffT>
void launch_batch_count(const BatchArgs<OffT>& a, int num_sms, cudaStream_t st) {
  k_batch_emit<OffT, true><<<num_sms * 8, 256, 0, st>>>(a);
}

// The outputs of a wave with deferred outputs, written once after its last level. Every
// event of the wave is still in the per-vertex slots (with its wave level), so entry
// (b, vc) is: -1 if bit b never reached vc; else the level and parent of the event holding
// bit b. A warp takes 32 consecutive caller ids and writes, for every slot b, 32 consecutive
// entries of b's level row and of its parent row: every output line is written exactly once
// (no fill beforehand, no partial lines per level). Entries with no event are left alone:
// the roots (written when seeded), and claims that did not fit the slots, which the overflow
// list applies here too (those entries are disjoint from the ones written from slots).
template <typename OffT>
__global__ void __launch_bounds__(256) k_batch_final(BatchArgs<OffT> a) {
  constexpr int K = kEventSlotsWave;
  static_assert(K == 8, "the event index of a bit is assembled from three masks");
  __shared__ int32_t* s_lvl[kMaxWave];
  __shared__ int32_t* s_par[kMaxWave];
  __shared__ int32_t s_start[kMaxWave];
  __shared__ int32_t s_el[8][K][32];  // per warp: event k's level and claimer, lane-major
  __shared__ int32_t s_eu[8][K][32];
  if (threadIdx.x < kMaxWave) {
    s_lvl[threadIdx.x] = a.slots->lvl[threadIdx.x];
    s_par[threadIdx.x] = a.slots->par[threadIdx.x];
    s_start[threadIdx.x] = a.slots->start[threadIdx.x];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int nb = a.n_slots;
  for (int64_t w = gwarp; w * 32 < a.n; w += nwarps) {
    const int64_t x = w * 32 + lane;
    const bool in = x < a.n;
    const int32_t vc = (int32_t)x;
    unsigned long long vis = 0ull, evm = 0ull, m0 = 0ull, m1 = 0ull, m2 = 0ull, dm = 0ull;
    int32_t drow = -1;
    if (in) {
      const int32_t v = a.new_id ? __ldg(a.new_id + vc) : vc;
      vis = a.visited[v];
      const int ne = vis ? min(a.evc[v], K) : 0;
      if (ne == K && (a.dense_idx || a.dense_ident)) {  // claims past the slots: the vertex's dense row
        drow = a.dense_ident ? v : a.dense_idx[v];
        if (drow >= 0) dm = a.dense_mask[drow];
      }
      for (int k = 0; k < ne; ++k) {
        const ClaimEvent ce = a.ev[(size_t)v * K + k];
        s_el[wib][k][lane] = ce.level;
        s_eu[wib][k][lane] = ce.u;
        // events hold disjoint bits: bit i of the index of bit b's event is bit b of m_i
        evm |= ce.mask;
        if (k & 1) m0 |= ce.mask;
        if (k & 2) m1 |= ce.mask;
        if (k & 4) m2 |= ce.mask;
      }
    }
    __syncwarp();
    // Bits reached without an event or a dense-row entry (roots, claims on the overflow list
    // or written at claim time) are written apart: skip them.
    const unsigned long long skip = vis & ~evm & ~dm;
    for (int half = 0; half < 2; ++half) {
      const unsigned vlo = (unsigned)(vis >> (32 * half)), slo = (unsigned)(skip >> (32 * half));
      const unsigned a0 = (unsigned)(m0 >> (32 * half)), a1 = (unsigned)(m1 >> (32 * half)),
                     a2 = (unsigned)(m2 >> (32 * half)), dlo = (unsigned)(dm >> (32 * half));
      const int bend = min(32, nb - 32 * half);
      for (int i = 0; i < bend; ++i) {
        const int b = 32 * half + i;
        if (!in || ((slo >> i) & 1u)) continue;
        int32_t lv = -1, pu = -1;
        if ((dlo >> i) & 1u) {
          lv = a.dense_lvl[(size_t)drow * kMaxWave + b] - s_start[b];
          pu = a.dense_par[(size_t)drow * kMaxWave + b];
        } else if ((vlo >> i) & 1u) {
          const int k = ((a0 >> i) & 1u) | (((a1 >> i) & 1u) << 1) | (((a2 >> i) & 1u) << 2);
          lv = s_el[wib][k][lane] - s_start[b];
          pu = s_eu[wib][k][lane];
        }
        s_lvl[b][vc] = lv;
        s_par[b][vc] = pu;
      }
    }
    __syncwarp();
  }
  const long long novf = min((long long)*(volatile unsigned long long*)&a.ctl->ovf_count, a.ovf_cap);
  for (long long o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < novf; o += (int64_t)gridDim.x * blockDim.x) {
    const OvfEvent e = a.ovf[o];
    for (unsigned long long bits = e.mask; bits; bits &= bits - 1) {
      const int b = __ffsll((long long)bits) - 1;
      s_lvl[b][e.v] = e.level - s_start[b];
      s_par[b][e.v] = e.u;
    }
  }
}

// The next frontier of an ordered expansion (wave_ordered on the expanded frontier's size),
// rebuilt in vertex order: entries are in vertex order within a round; rounds land in any
// order. Where the rounds are cut depends on the graph (MARKS = BatchArgs::order_marks): a
// degree-relabelled graph puts its hubs at the lowest ids, so rounds of 16 x blockDim.x
// vertices there would leave the hubs' tile descriptors (22 % of the edges of R-MAT s22 in
// the first 4096 vertices) to one CTA. Two kernels, so that each keeps its own register count
// (the mask variant 32, for 8 resident CTAs per SM).
template <typename OffT, bool MARKS>
__global__ void __launch_bounds__(256) k_batch_order(BatchArgs<OffT> a) {
  BatchCtl* ctl = a.ctl;
  if (!wave_ordered(a, *(volatile long long*)&ctl->prev_count)) return;  // grid-uniform
  const int t = *(volatile int*)&ctl->level - 2;  // the expansion that just closed
  const int nxt = (t & 1) ^ 1, q3n = (t + 1) % 3;
  __shared__ OffT s_warp[33];
  __shared__ unsigned long long s_resv;
  if constexpr (MARKS)
    order_from_marks(a, ctl, nxt, q3n, s_warp, &s_resv);
  else
    order_from_masks(a, ctl, nxt, q3n, s_warp, &s_resv);
}

template <typename OffT>
void launch_batch_order(const BatchArgs<OffT>& a, int num_sms, cudaStream_t st) {
  if (a.order_marks)
    k_batch_order<OffT, true><<<num_sms * 8, 256, 0, st>>>(a);
  else
    k_batch_order<OffT, false><<<num_sms * 8, 256, 0, st>>>(a);
}

template <typename OffT>
void launch_batch_final(const BatchArgs<OffT>& a, int num_sms, cudaStream_t st) {
  k_batch_final<OffT><<<num_sms * 8, 256, 0, st>>>(a);
}

// Dynamic shared memory of a batched shape: CTA tiles stage their entries and share one
// claim buffer; warp tiles need only CLAIM claim entries per warp.
template <typename OffT, int BLOCK, int E, int CLAIM, bool WT>
constexpr size_t batch_smem_bytes() {
  return WT ? (size_t)(BLOCK / 32) * CLAIM * sizeof(int2) : BatchSmem<OffT, BLOCK, E, CLAIM>::bytes;
}

template <typename OffT, int BLOCK, int E, int CLAIM, bool WT, int TPS>
static cudaError_t launch_batch_expand_t(const BatchArgs<OffT>& a, int grid, cudaStream_t st) {
  constexpr size_t bytes = batch_smem_bytes<OffT, BLOCK, E, CLAIM, WT>();
  auto kern = k_expand_batch<OffT, BLOCK, E, CLAIM, WT, TPS>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  kern<<<grid, BLOCK, bytes, st>>>(a);
  return cudaGetLastError();
}

template <typename OffT, int BLOCK, int E, int CLAIM, bool WT, int TPS>
static int batch_grid_t(int num_sms) {
  constexpr size_t bytes = batch_smem_bytes<OffT, BLOCK, E, CLAIM, WT>();
  auto kern = k_expand_batch<OffT, BLOCK, E, CLAIM, WT, TPS>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, bytes) != cudaSuccess) per_sm = 1;
  return (per_sm > 0 ? per_sm : 1) * num_sms;
}

// Compiled shapes of the batched expansion (BLOCK, E, CLAIM, tiles, TPS): tiles 0 = CTA
// tiles of BLOCK x E edges (CLAIM = CTA claim buffer), 1 = warp tiles of 32 x E edges (CLAIM
// = claim entries per warp); TPS = resident threads per SM the registers are sized for (0:
// the compiler's choice). The autotuner picks one.
#define GBFS_BATCH_SHAPES(X)  \
  X(0, 256, 4, 2048, 0, 0)    \
  X(1, 256, 2, 2048, 0, 0)    \
  X(2, 128, 4, 1024, 0, 0)    \
  X(3, 512, 2, 2048, 0, 0)    \
  X(4, 256, 4, 128, 1, 0)     \
  X(5, 128, 4, 128, 1, 0)     \
  X(6, 256, 8, 256, 1, 0)     \
  X(7, 128, 4, 128, 1, 1280)  \
  X(8, 128, 4, 128, 1, 1536)

const ExpandShape kBatchShapes[] = {
#define X(id, b, e, c, w, t) {id, b, e, c, w},
    GBFS_BATCH_SHAPES(X)
#undef X
};
const int kNumBatchShapes = sizeof(kBatchShapes) / sizeof(kBatchShapes[0]);

template <typename OffT>
cudaError_t launch_batch_expand(int shape, const BatchArgs<OffT>& a, int grid, cudaStream_t st) {
  switch (shape) {
#define X(id, b, e, c, w, t) \
  case id: return launch_batch_expand_t<OffT, b, e, c, w != 0, t>(a, grid, st);
    GBFS_BATCH_SHAPES(X)
#undef X
  }
  return cudaErrorInvalidValue;
}

template <typename OffT>
int batch_expand_grid(int shape, int num_sms) {
  switch (shape) {
#define X(id, b, e, c, w, t) \
  case id: return batch_grid_t<OffT, b, e, c, w != 0, t>(num_sms);
    GBFS_BATCH_SHAPES(X)
#undef X
  }
  return num_sms;
}

// Per-slot statistics from the outputs: stats[3 b + 0] = sum of degrees of reached
// vertices (2 m_c), [3 b + 1] = reached count, [3 b + 2] = max level + 1.
template <typename OffT>
__global__ void k_batch_stats(const OffT* __restrict__ off, const int32_t* __restrict__ new_id, int64_t n,
                              const WaveSlots* slots, long long* stats) {
  __shared__ long long s_red[3][32];
  const int b = blockIdx.y;
  const int32_t* lv = slots->lvl[b];
  long long e2 = 0, reached = 0, depth = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t l = lv[v];
    if (l >= 0) {
      const int64_t x = new_id ? new_id[v] : v;  // the outputs are in caller ids
      e2 += (long long)(off[x + 1] - off[x]);
      ++reached;
      depth = max(depth, (long long)l + 1);
    }
  }
  for (int d = 16; d; d >>= 1) {
    e2 += __shfl_xor_sync(0xffffffffu, e2, d);
    reached += __shfl_xor_sync(0xffffffffu, reached, d);
    depth = max(depth, __shfl_xor_sync(0xffffffffu, depth, d));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_red[0][w] = e2;
    s_red[1][w] = reached;
    s_red[2][w] = depth;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long a0 = 0, a1 = 0, a2 = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a0 += s_red[0][i];
      a1 += s_red[1][i];
      a2 = max(a2, s_red[2][i]);
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(&stats[3 * b + 0]), (unsigned long long)a0);
    atomicAdd(reinterpret_cast<unsigned long long*>(&stats[3 * b + 1]), (unsigned long long)a1);
    atomicMax(&stats[3 * b + 2], a2);
  }
}

template <typename OffT>
void launch_batch_stats(const OffT* off, const int32_t* new_id, int64_t n, const WaveSlots* slots, int n_slots,
                        long long* stats, int num_sms, cudaStream_t st) {
  cudaMemsetAsync(stats, 0, sizeof(long long) * 3 * n_slots, st);
  dim3 grid((unsigned)std::max(1, num_sms * 2 / std::max(1, n_slots / 8)), (unsigned)n_slots);
  k_batch_stats<OffT><<<grid, 256, 0, st>>>(off, new_id, n, slots, stats);
}

template <typename OffT>
__global__ void k_level_stats(const OffT* __restrict__ off, const int32_t* __restrict__ new_id, int64_t n,
                              const int32_t* __restrict__ lv, long long* out) {
  __shared__ long long s_red[3][32];
  long long e2 = 0, reached = 0, depth = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t l = lv[v];
    if (l >= 0) {
      const int64_t x = new_id ? new_id[v] : v;  // the outputs are in caller ids
      e2 += (long long)(off[x + 1] - off[x]);
      ++reached;
      depth = max(depth, (long long)l + 1);
    }
  }
  for (int d = 16; d; d >>= 1) {
    e2 += __shfl_xor_sync(0xffffffffu, e2, d);
    reached += __shfl_xor_sync(0xffffffffu, reached, d);
    depth = max(depth, __shfl_xor_sync(0xffffffffu, depth, d));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_red[0][w] = e2;
    s_red[1][w] = reached;
    s_red[2][w] = depth;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long a0 = 0, a1 = 0, a2 = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a0 += s_red[0][i];
      a1 += s_red[1][i];
      a2 = max(a2, s_red[2][i]);
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(&out[0]), (unsigned long long)a0);
    atomicAdd(reinterpret_cast<unsigned long long*>(&out[1]), (unsigned long long)a1);
    atomicMax(&out[2], a2);
  }
}

template <typename OffT>
void launch_level_stats(const OffT* off, const int32_t* new_id, int64_t n, const int32_t* levels, long long* out,
                        int num_sms, cudaStream_t st) {
  cudaMemsetAsync(out, 0, sizeof(long long) * 3, st);
  k_level_stats<OffT><<<num_sms * 2, 256, 0, st>>>(off, new_id, n, levels, out);
}

#define INST(OffT)                                                                                          \
  template void launch_batch_clear<OffT>(const BatchArgs<OffT>&, int, cudaStream_t);                       \
  template void launch_batch_emit<OffT>(const BatchArgs<OffT>&, int, cudaStream_t);                        \
  template void launch_batch_count<OffT>(const BatchArgs<OffT>&, int, cudaStream_t);                       \
  template void launch_batch_final<OffT>(const BatchArgs<OffT>&, int, cudaStream_t);                       \
  template void launch_batch_order<OffT>(const BatchArgs<OffT>&, int, cudaStream_t);                       \
  template void launch_batch_seed<OffT>(const BatchArgs<OffT>&, const RootSeed*, int, int, bool, cudaStream_t); \
  template cudaError_t launch_batch_expand<OffT>(int, const BatchArgs<OffT>&, int, cudaStream_t);           \
  template int batch_expand_grid<OffT>(int, int);                                                           \
  template void launch_batch_stats<OffT>(const OffT*, const int32_t*, int64_t, const WaveSlots*, int, long long*, int, \
                                         cudaStream_t);                                                     \
  template void launch_level_stats<OffT>(const OffT*, const int32_t*, int64_t, const int32_t*, long long*, int, \
                                         cudaStream_t);
INST(int32_t)
INST(int64_t)
#undef INST

}  // namespace gbfs
