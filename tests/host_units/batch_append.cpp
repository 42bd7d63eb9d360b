// CPU unit tests of the appends of a wave's next frontier (batch_warp_flush, batch_flush in
// batch_append.cuh), run on the SIMT emulator (simt_emu.h). Warps (or a CTA) flush buffers of
// claimed vertices (vertex, degree), several flushes after one another on top of an earlier
// reservation, with zero-degree vertices, rows of many chunks (more than 32: written
// warp-wide), partly filled buffers, int32 and int64 offsets (past 2^32). Afterwards:
//  * the packed counter holds the earlier reservation plus every flushed (count, edges);
//  * every flush's entries are one contiguous slot range in the order of its buffer, and the
//    list holds every buffered vertex once, nothing past the count;
//  * the degree scan runs on from the earlier reservation's edges (cum[k + 1] = cum[k] +
//    deg(v_k)), and base[k] = off[v_k] - cum[k];
//  * every chunk start c * kChunk in the appended edge range names the entry whose range holds
//    it (the binary search of Algorithm 3), that entry's vertex and column entry; descriptors
//    outside the range stay untouched.
// Prints "ok" and returns 0, or reports the first failure and returns 1.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "batch_append.cuh"

thread_local gbfs_host_dim3 threadIdx, blockIdx;
gbfs_host_dim3 blockDim, gridDim;
thread_local simt::Block* simt::t_block;

using gbfs::kChunk;

static uint64_t rng_state = 0xA0761D6478BD642Full;
static uint64_t rnd() {  // xorshift64*
  rng_state ^= rng_state >> 12;
  rng_state ^= rng_state << 25;
  rng_state ^= rng_state >> 27;
  return rng_state * 0x2545F4914F6CDD1Dull;
}
static int64_t below(int64_t n) { return n > 0 ? (int64_t)(rnd() % (uint64_t)n) : 0; }

static int failures = 0;
#define CHECK(cond, ...)                               \
  do {                                                 \
    if (!(cond) && failures++ == 0) {                  \
      std::printf("FAIL %s:%d: ", __FILE__, __LINE__); \
      std::printf(__VA_ARGS__);                        \
      std::printf("\n");                               \
    }                                                  \
  } while (0)

constexpr int kWcap = 128;  // a warp's claim buffer (the warp-tile shapes' CLAIM)
constexpr int kBlock = 64, kCtaClaim = 300;  // a CTA's buffer: not a multiple of the block

// `flushes` rounds; in each, every buffer of the round is flushed by its warp (CTA = false:
// `warps` warps of one block, each with its own buffer) or by the whole block (CTA = true, one
// buffer). Vertices are distinct across the whole test, as claims of one level are.
template <typename OffT, bool CTA>
static void check_appends(int warps, int flushes, OffT off0, bool hubs) {
  const int cap = CTA ? kCtaClaim : kWcap;
  const int buffers = CTA ? flushes : warps * flushes;
  const int64_t n = (int64_t)buffers * cap + 1 + below(50);
  std::vector<int64_t> deg((size_t)n);
  for (auto& d : deg) {
    const int64_t r = below(100);
    d = r < 15 ? 0 : r < 90 ? 1 + below(20) : r < 98 ? 1 + below(700) : (hubs ? 4097 + below(6000) : below(200));
  }
  std::vector<OffT> off((size_t)n + 1);
  off[0] = off0;
  for (int64_t v = 0; v < n; ++v) off[(size_t)v + 1] = off[(size_t)v] + (OffT)deg[(size_t)v];
  std::vector<int32_t> perm((size_t)n);
  for (int64_t v = 0; v < n; ++v) perm[(size_t)v] = (int32_t)v;
  for (int64_t v = n - 1; v > 0; --v) std::swap(perm[(size_t)v], perm[(size_t)below(v + 1)]);
  // the buffers: random fill levels, distinct vertices
  std::vector<std::vector<int2>> buf((size_t)buffers);
  size_t next = 0;
  int64_t want_count = 0, want_edges = 0;
  for (auto& b : buf) {
    const int nc = below(5) == 0 ? cap : (int)below(cap + 1);
    for (int i = 0; i < nc; ++i) {
      const int32_t v = perm[next++];
      b.push_back(make_int2(v, (int)deg[(size_t)v]));
      want_edges += deg[(size_t)v];
    }
    want_count += nc;
  }
  // an earlier reservation on the counter: appends continue after it
  const int64_t c0 = below(1000), e0 = below(1 << 20);
  // slack past the appended range: a wrong scan shows up as a stray write, not a crash
  const int64_t slots = c0 + want_count + 1, chunks = 2 * ((e0 + want_edges) / kChunk) + 64;
  std::vector<int32_t> qv((size_t)slots, -7);
  std::vector<OffT> cum((size_t)slots, (OffT)-7), base((size_t)slots, (OffT)-7);
  std::vector<gbfs::TileDesc<OffT>> desc((size_t)chunks, gbfs::TileDesc<OffT>{-7, -7, (OffT)-7});
  gbfs::BatchCtl ctl{};
  const int t = (int)below(6), nxt = (t & 1) ^ 1, q3n = (t + 1) % 3;
  gbfs::BatchArgs<OffT> a{};
  a.off = off.data();
  a.n = n;
  a.qv[q3n] = qv.data();
  a.cum[nxt] = cum.data();
  a.base[nxt] = base.data();
  a.chunk[nxt] = desc.data();
  a.ctl = &ctl;
  a.pk = gbfs::Packed{40, (1ull << 40) - 1};
  ctl.counter[nxt] = a.pk.make(c0, e0);
  std::vector<int64_t> first_slot((size_t)buffers, -1);
  gridDim = gbfs_host_dim3{1, 1, 1};
  for (int f = 0; f < flushes; ++f) {
    if (CTA) {
      std::vector<int2>& b = buf[(size_t)f];
      std::vector<int2> s_claim(b);
      s_claim.resize(cap);
      OffT s_warp[33];
      unsigned long long s_resv = 0;
      first_slot[(size_t)f] = a.pk.count(ctl.counter[nxt]);
      simt::run_block(kBlock, 0, [&] {
        gbfs::batch_flush<OffT, kBlock, kCtaClaim>(a, nxt, q3n, s_claim.data(), (int)b.size(), s_warp, &s_resv);
      });
    } else {
      simt::run_block(32 * warps, 0, [&] {
        const int w = (int)(threadIdx.x / 32);
        const std::vector<int2>& b = buf[(size_t)(f * warps + w)];
        gbfs::batch_warp_flush<OffT, (kWcap + 31) / 32>(a, nxt, q3n, b.data(), (int)b.size());
      });
    }
  }
  const char* kind = CTA ? "cta" : "warp";
  const int64_t count = a.pk.count(ctl.counter[nxt]), edges = a.pk.edges(ctl.counter[nxt]);
  CHECK(count == c0 + want_count && edges == e0 + want_edges, "%s: counter (%lld, %lld), want (%lld, %lld)", kind,
        (long long)count, (long long)edges, (long long)(c0 + want_count), (long long)(e0 + want_edges));
  if (count != c0 + want_count) return;
  for (int64_t k = 0; k < c0; ++k) CHECK(qv[(size_t)k] == -7, "%s: slot %lld of the earlier reservation written", kind, (long long)k);
  CHECK(qv[(size_t)count] == -7, "%s: slot past the count written", kind);
  // each buffer's entries: one contiguous range in buffer order (warps of a round in any order)
  std::vector<int64_t> where((size_t)n, -1);
  for (int64_t k = c0; k < count; ++k) {
    const int32_t v = qv[(size_t)k];
    CHECK(v >= 0 && v < n && where[(size_t)v] < 0, "%s: slot %lld holds %d", kind, (long long)k, v);
    if (v >= 0 && v < n) where[(size_t)v] = k;
  }
  for (int bi = 0; bi < buffers; ++bi) {
    const std::vector<int2>& b = buf[(size_t)bi];
    for (size_t i = 0; i < b.size(); ++i) {
      const int64_t k = where[(size_t)b[i].x];
      CHECK(k >= 0, "%s: buffered vertex %d missing", kind, b[i].x);
      if (i > 0) CHECK(k == where[(size_t)b[i - 1].x] + 1, "%s: buffer %d not contiguous in order at %zu", kind, bi, i);
    }
    if (CTA && !b.empty()) CHECK(where[(size_t)b[0].x] == first_slot[(size_t)bi], "%s: flush %d not at its reservation", kind, bi);
  }
  if (failures) return;  // the checks below index by the list's entries
  // scan, bases, descriptors
  for (int64_t k = c0; k < count; ++k) {
    const OffT want = k == c0 ? (OffT)e0 : cum[(size_t)k - 1] + (OffT)deg[(size_t)qv[(size_t)k - 1]];
    CHECK(cum[(size_t)k] == want, "%s: cum[%lld] = %lld, want %lld", kind, (long long)k, (long long)cum[(size_t)k], (long long)want);
    CHECK(base[(size_t)k] == off[(size_t)qv[(size_t)k]] - cum[(size_t)k], "%s: base[%lld] wrong", kind, (long long)k);
  }
  if (failures) return;  // the walk below follows the scan
  int64_t k = c0;
  for (int64_t c = 0; c < chunks; ++c) {
    const int64_t e = c * kChunk;
    const gbfs::TileDesc<OffT>& d = desc[(size_t)c];
    if (e < e0 || e >= e0 + want_edges) {
      CHECK(d.k == -7, "%s: descriptor %lld outside the appended edges written", kind, (long long)c);
      continue;
    }
    while (k + 1 < count && (int64_t)cum[(size_t)k] + deg[(size_t)qv[(size_t)k]] <= e) ++k;
    CHECK(d.k == (int32_t)k && d.u == qv[(size_t)k] && d.col == base[(size_t)k] + (OffT)e,
          "%s: descriptor %lld = (%d, %d, %lld), want (%lld, %d, %lld)", kind, (long long)c, d.k, d.u, (long long)d.col,
          (long long)k, qv[(size_t)k], (long long)(base[(size_t)k] + (OffT)e));
  }
}

int main() {
  check_appends<int32_t, false>(1, 1, 0, false);
  check_appends<int32_t, false>(2, 3, 0, true);
  check_appends<int32_t, false>(4, 2, 0, true);
  check_appends<int64_t, false>(3, 2, (int64_t)5 << 32, true);
  check_appends<int32_t, true>(1, 1, 0, false);
  check_appends<int32_t, true>(1, 4, 0, true);
  check_appends<int64_t, true>(1, 3, (int64_t)3 << 31, true);
  for (int t = 0; t < 6; ++t) {
    check_appends<int32_t, false>(1 + (int)below(4), 1 + (int)below(3), 0, below(2) != 0);
    check_appends<int32_t, true>(1, 1 + (int)below(4), 0, below(2) != 0);
  }
  if (failures) {
    std::printf("%d failures\n", failures);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
