// CPU unit tests of the two passes that rebuild an ordered wave level's next frontier in
// vertex order, run block by block on the SIMT emulator (simt_emu.h):
//  * order_from_masks, one vertex per thread over the 64-bit root masks F_{t+1};
//  * order_from_marks, 16 vertices per thread over the byte marks.
// On random graphs (zero-degree vertices, hub rows of more than 32 tile chunks, vertex counts
// that are not multiples of 16, int32 and int64 offsets, offsets past 2^32) and random
// marked sets (none, sparse, dense, all), every pass must produce:
//  * the list: each marked vertex exactly once, ascending within every round of consecutive
//    vertices one block takes, each round's entries in one contiguous slot range;
//  * the degree scan: cum[0] = 0 and cum[k + 1] = cum[k] + deg(v_k) (the reservations keep
//    slot and edge ranges in step), and the packed counter holds (count, edges);
//  * the column bases base[k] = off[v_k] - cum[k];
//  * the tile descriptors: every chunk start c * kChunk below the edge total names the entry
//    whose edge range holds it (the binary search of Algorithm 3), that entry's vertex and
//    column entry base + c * kChunk, and nothing past the total is written;
//  * the byte marks all cleared afterwards (the mask pass leaves the masks as they were).
// Prints "ok" and returns 0, or reports the first failure and returns 1.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "batch_order.cuh"

thread_local gbfs_host_dim3 threadIdx, blockIdx;
gbfs_host_dim3 blockDim, gridDim;
thread_local simt::Block* simt::t_block;

using gbfs::kChunk;

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
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

// One ordered level: n vertices with the given degrees (offsets starting at off0), marked
// vertices `in`; the pass runs on `grid` blocks of `threads` emulated threads, one block at a
// time. MARKS selects the byte-mark pass.
template <typename OffT, bool MARKS>
static void check_order(const std::vector<int64_t>& deg, const std::vector<char>& in, OffT off0, int grid,
                        int threads) {
  const int64_t n = (int64_t)deg.size();
  std::vector<OffT> off((size_t)n + 1);
  off[0] = off0;
  for (int64_t v = 0; v < n; ++v) off[(size_t)v + 1] = off[(size_t)v] + (OffT)deg[(size_t)v];
  int64_t want_count = 0, want_edges = 0;
  for (int64_t v = 0; v < n; ++v)
    if (in[(size_t)v]) {
      ++want_count;
      want_edges += deg[(size_t)v];
    }
  const int64_t chunks = want_edges / kChunk + 2, slack = 8;  // slack: descriptors past the total stay untouched
  std::vector<unsigned long long> fmask((size_t)n, 0ull);
  for (int64_t v = 0; v < n; ++v)
    if (in[(size_t)v]) fmask[(size_t)v] = 1ull << below(64) | (rnd() & (rnd() & rnd()));
  const std::vector<unsigned long long> fmask0 = fmask;
  std::vector<uint4> mark_words((size_t)(n + 15) / 16, make_uint4(0u, 0u, 0u, 0u));
  uint8_t* marks = reinterpret_cast<uint8_t*>(mark_words.data());
  for (int64_t v = 0; v < n; ++v) marks[v] = in[(size_t)v] ? 1 : 0;
  std::vector<int32_t> qv((size_t)n + 1, -7);
  std::vector<OffT> cum((size_t)n + 1, (OffT)-7), base((size_t)n + 1, (OffT)-7);
  std::vector<gbfs::TileDesc<OffT>> desc((size_t)(chunks + slack), gbfs::TileDesc<OffT>{-7, -7, (OffT)-7});
  gbfs::BatchCtl ctl{};
  const int t = (int)below(6), nxt = (t & 1) ^ 1, q3n = (t + 1) % 3;  // any level's buffer indices
  gbfs::BatchArgs<OffT> a{};
  a.off = off.data();
  a.n = n;
  a.fmask[q3n] = fmask.data();
  a.fmark = marks;
  a.qv[q3n] = qv.data();
  a.cum[nxt] = cum.data();
  a.base[nxt] = base.data();
  a.chunk[nxt] = desc.data();
  a.ctl = &ctl;
  a.pk = gbfs::Packed{40, (1ull << 40) - 1};
  a.order_marks = MARKS ? 1 : 0;
  gridDim = gbfs_host_dim3{(unsigned)grid, 1, 1};
  for (int b = 0; b < grid; ++b) {
    OffT s_warp[33];
    unsigned long long s_resv = 0;
    simt::run_block(threads, (unsigned)b, [&] {
      if (MARKS)
        gbfs::order_from_marks(a, &ctl, nxt, q3n, s_warp, &s_resv);
      else
        gbfs::order_from_masks(a, &ctl, nxt, q3n, s_warp, &s_resv);
    });
  }
  const char* pass = MARKS ? "marks" : "masks";
  const int64_t count = a.pk.count(ctl.counter[nxt]), edges = a.pk.edges(ctl.counter[nxt]);
  CHECK(count == want_count && edges == want_edges, "%s: counter (%lld, %lld), want (%lld, %lld)", pass,
        (long long)count, (long long)edges, (long long)want_count, (long long)want_edges);
  if (count != want_count) return;
  // the list: a permutation of the marked vertices, rounds contiguous and ascending
  std::vector<int32_t> got(qv.begin(), qv.begin() + count), want;
  for (int64_t v = 0; v < n; ++v)
    if (in[(size_t)v]) want.push_back((int32_t)v);
  std::vector<int32_t> sorted = got;
  std::sort(sorted.begin(), sorted.end());
  CHECK(sorted == want, "%s: the list is not the marked set", pass);
  CHECK(qv[(size_t)count] == -7, "%s: list entry past the count written", pass);
  if (failures) return;  // the checks below index by the list's entries
  const int64_t round = (int64_t)threads * (MARKS ? 16 : 1);
  for (int64_t k = 0; k + 1 < count; ++k) {
    const int32_t u = got[(size_t)k], w = got[(size_t)k + 1];
    if (u / round == w / round) CHECK(u < w, "%s: round of %d not ascending at slot %lld", pass, u, (long long)k);
  }
  std::vector<int64_t> first((size_t)(n / round + 1), -1), last((size_t)(n / round + 1), -1), seen((size_t)(n / round + 1), 0);
  for (int64_t k = 0; k < count; ++k) {
    const int64_t r = got[(size_t)k] / round;
    if (first[(size_t)r] < 0) first[(size_t)r] = k;
    last[(size_t)r] = k;
    ++seen[(size_t)r];
  }
  for (size_t r = 0; r < seen.size(); ++r)
    if (seen[r]) CHECK(last[r] - first[r] + 1 == seen[r], "%s: round %zu split over the list", pass, r);
  // scan values, column bases, descriptors
  for (int64_t k = 0; k < count; ++k) {
    const int32_t v = got[(size_t)k];
    const OffT want_cum = k == 0 ? (OffT)0 : cum[(size_t)k - 1] + (OffT)deg[(size_t)got[(size_t)k - 1]];
    CHECK(cum[(size_t)k] == want_cum, "%s: cum[%lld] = %lld, want %lld", pass, (long long)k, (long long)cum[(size_t)k],
          (long long)want_cum);
    CHECK(base[(size_t)k] == off[(size_t)v] - cum[(size_t)k], "%s: base[%lld] wrong", pass, (long long)k);
  }
  if (failures) return;  // the walk below follows the scan
  int64_t k = 0;
  for (int64_t c = 0; c < chunks + slack; ++c) {
    const int64_t e = c * kChunk;
    const gbfs::TileDesc<OffT>& d = desc[(size_t)c];
    if (e >= want_edges) {
      CHECK(d.k == -7, "%s: descriptor %lld past the edge total written", pass, (long long)c);
      continue;
    }
    while (k + 1 < count && (int64_t)cum[(size_t)k] + deg[(size_t)got[(size_t)k]] <= e) ++k;  // entry holding e
    CHECK(d.k == (int32_t)k && d.u == got[(size_t)k] && d.col == base[(size_t)k] + (OffT)e,
          "%s: descriptor %lld = (%d, %d, %lld), want (%lld, %d, %lld)", pass, (long long)c, d.k, d.u, (long long)d.col,
          (long long)k, got[(size_t)k], (long long)(base[(size_t)k] + (OffT)e));
  }
  if (MARKS) {
    bool clear = true;
    for (int64_t i = 0; i < (int64_t)mark_words.size() * 16; ++i) clear = clear && marks[i] == 0;
    CHECK(clear, "%s: byte marks left set", pass);
  }
  CHECK(fmask == fmask0, "%s: frontier masks changed", pass);
}

// Degrees the way an ordered level sees them: zero-degree vertices, short rows, rows over a
// few chunks, and optionally hub rows spanning more than 32 chunks (written warp-wide).
static std::vector<int64_t> degrees(int64_t n, bool hubs) {
  std::vector<int64_t> d((size_t)n);
  for (auto& x : d) {
    const int64_t r = below(100);
    x = r < 15 ? 0 : r < 85 ? 1 + below(12) : r < 97 ? 1 + below(600) : (hubs ? 4097 + below(9000) : below(300));
  }
  return d;
}

static std::vector<char> marked(int64_t n, int64_t per_1024) {
  std::vector<char> in((size_t)n);
  for (auto& x : in) x = below(1024) < per_1024;
  return in;
}

template <typename OffT>
static void check_both(int64_t n, int64_t per_1024, bool hubs, OffT off0, int grid, int threads) {
  const std::vector<int64_t> d = degrees(n, hubs);
  const std::vector<char> in = marked(n, per_1024);
  check_order<OffT, false>(d, in, off0, grid, threads);
  check_order<OffT, true>(d, in, off0, grid, threads);
}

int main() {
  check_both<int32_t>(1, 1024, false, 0, 1, 32);           // one vertex, marked
  check_both<int32_t>(1000, 0, true, 0, 2, 64);            // nothing marked: no reservation, no writes
  check_both<int32_t>(2047, 1024, true, 0, 3, 64);         // every vertex, ragged n
  check_both<int32_t>(5001, 64, true, 0, 2, 64);           // sparse
  check_both<int32_t>(3333, 300, true, 0, 4, 128);         // dense, several rounds per block
  check_both<int32_t>(4099, 700, false, 0, 1, 256);        // one block, the kernel's block size
  check_both<int64_t>(2500, 500, true, (int64_t)3 << 32, 3, 64);   // offsets past 2^32
  check_both<int64_t>(1234, 1024, false, (int64_t)1 << 31, 2, 96); // int64, three warps per block
  for (int t = 0; t < 6; ++t)
    check_both<int32_t>(1 + below(3000), below(1025), below(2) != 0, 0, 1 + (int)below(4), 32 * (1 + (int)below(4)));
  if (failures) {
    std::printf("%d failures\n", failures);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
