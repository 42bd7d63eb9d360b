// CPU unit tests of the scalar device helpers of the CUDA library, compiled as host code:
//  * binsearch_maxle (the thread -> edge binary search of Algorithm 3) against
//    std::upper_bound - 1 on random and adversarial non-decreasing sequences (runs of equal
//    values = zero-degree frontier entries), int32 and int64, whole and partial ranges,
//    and the monotonicity of the map in the searched value (Sec. 3.4.1);
//  * write_chunks / write_descs: every chunk boundary c * kChunk inside an entry's edge
//    range [cum, cum + deg) gets that entry (and its parent and column entry), nothing
//    else is touched; over a whole frontier the chunk index equals the binary-search answer
//    at every boundary;
//  * Packed: the (count, edges) word of the fused append adds component-wise;
//  * mark_bits: every pattern of four 0/1 byte marks maps to its 4-bit vertex mask.
// Prints "ok" and returns 0, or reports the first failure and returns 1.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "device_util.cuh"

using gbfs::kChunk;

static uint64_t rng_state = 0x2545F4914F6CDD1Dull;
static uint64_t rnd() {  // xorshift64*
  rng_state ^= rng_state >> 12;
  rng_state ^= rng_state << 25;
  rng_state ^= rng_state >> 27;
  return rng_state * 0x2545F4914F6CDD1Dull;
}
static int64_t below(int64_t n) { return n > 0 ? (int64_t)(rnd() % (uint64_t)n) : 0; }

static int failures = 0;
#define CHECK(cond, ...)                          \
  do {                                            \
    if (!(cond) && failures++ == 0) {             \
      std::printf("FAIL %s:%d: ", __FILE__, __LINE__); \
      std::printf(__VA_ARGS__);                   \
      std::printf("\n");                          \
    }                                             \
  } while (0)

// Degrees with the shapes a frontier has: zero-degree entries, runs, hubs.
static std::vector<int64_t> degrees(int64_t n, int64_t big) {
  std::vector<int64_t> d((size_t)n);
  for (auto& x : d) {
    const int64_t r = below(10);
    x = r < 3 ? 0 : r < 8 ? below(40) : below(big);
  }
  return d;
}

template <typename T>
static void check_binsearch(int64_t n, int64_t big) {
  const std::vector<int64_t> d = degrees(n, big);
  std::vector<T> cum((size_t)n);
  T acc = 0;
  for (int64_t k = 0; k < n; ++k) {
    cum[(size_t)k] = acc;
    acc += (T)d[(size_t)k];
  }
  const T total = acc;
  // searched values: every scan boundary and its neighbours, plus random ones, in order
  std::vector<T> xs;
  for (int64_t k = 0; k < n; ++k)
    for (T dx = -1; dx <= 1; ++dx)
      if (cum[(size_t)k] + dx >= 0) xs.push_back(cum[(size_t)k] + dx);
  for (int i = 0; i < 200; ++i) xs.push_back((T)below((int64_t)total + 3));
  xs.push_back(total);
  std::sort(xs.begin(), xs.end());
  int64_t prev = -1;
  for (const T x : xs) {
    const int64_t want = (int64_t)(std::upper_bound(cum.begin(), cum.end(), x) - cum.begin()) - 1;
    const int64_t got = (int64_t)gbfs::binsearch_maxle<T, int64_t>(cum.data(), 0, n, x);
    CHECK(got == want, "binsearch_maxle(x=%lld) = %lld, want %lld (n=%lld)", (long long)x, (long long)got,
          (long long)want, (long long)n);
    CHECK(got >= prev, "map not monotone at x=%lld", (long long)x);
    prev = got;
    // a partial range [lo, hi) with cum[lo] <= x
    const int64_t lo = below(want + 1), hi = want + 1 + below(n - want);
    const int64_t want2 = (int64_t)(std::upper_bound(cum.begin() + lo, cum.begin() + hi, x) - cum.begin()) - 1;
    const int64_t got2 = (int64_t)gbfs::binsearch_maxle<T, int64_t>(cum.data(), lo, hi, x);
    CHECK(got2 == want2, "binsearch_maxle on [%lld, %lld) x=%lld: %lld, want %lld", (long long)lo, (long long)hi,
          (long long)x, (long long)got2, (long long)want2);
  }
}

template <typename OffT>
static void check_chunks(int64_t n, int64_t big, OffT start) {
  const std::vector<int64_t> d = degrees(n, big);
  std::vector<OffT> cum((size_t)n);
  OffT acc = start;  // the scan may start anywhere (an int64 level edge space, say)
  for (int64_t k = 0; k < n; ++k) {
    cum[(size_t)k] = acc;
    acc += (OffT)d[(size_t)k];
  }
  const OffT c_lo = start / kChunk, c_hi = acc / kChunk + 2;
  std::vector<int32_t> chunk((size_t)(c_hi - c_lo), -7);
  std::vector<gbfs::TileDesc<OffT>> desc((size_t)(c_hi - c_lo), gbfs::TileDesc<OffT>{-7, -7, (OffT)-7});
  for (int64_t k = 0; k < n; ++k) {
    const OffT base = (OffT)(1000 * k) - cum[(size_t)k];  // off[v] - cum with off[v] = 1000 k
    gbfs::write_chunks<OffT>(chunk.data() - c_lo, cum[(size_t)k], (OffT)d[(size_t)k], (int32_t)k);
    gbfs::write_descs<OffT>(desc.data() - c_lo, cum[(size_t)k], (OffT)d[(size_t)k], (int32_t)k, (int32_t)(7 * k + 1),
                            base);
  }
  for (OffT c = c_lo; c < c_hi; ++c) {
    const OffT e = c * kChunk;
    const size_t i = (size_t)(c - c_lo);
    if (e < start || e >= acc) {  // outside the level's edge space: untouched
      CHECK(chunk[i] == -7 && desc[i].k == -7, "chunk %lld outside the edge space was written", (long long)c);
      continue;
    }
    const int64_t want = (int64_t)(std::upper_bound(cum.begin(), cum.end(), e) - cum.begin()) - 1;
    CHECK(chunk[i] == want, "chunk[%lld] = %d, want %lld", (long long)c, chunk[i], (long long)want);
    CHECK(desc[i].k == want && desc[i].u == (int32_t)(7 * want + 1), "desc[%lld] entry/parent wrong", (long long)c);
    CHECK(desc[i].col == (OffT)(1000 * want) + (e - cum[(size_t)want]), "desc[%lld].col wrong", (long long)c);
    CHECK(d[(size_t)want] > 0, "zero-degree entry %lld owns chunk %lld", (long long)want, (long long)c);
  }
}

static void check_packed() {
  for (int count_bits = 20; count_bits <= 32; ++count_bits) {
    gbfs::Packed pk{64 - count_bits, (1ull << (64 - count_bits)) - 1};
    for (int t = 0; t < 2000; ++t) {
      const long long c1 = below(1ll << (count_bits - 1)), c2 = below(1ll << (count_bits - 1));
      const long long e1 = (long long)below((long long)(pk.mask >> 1)), e2 = (long long)below((long long)(pk.mask >> 1));
      const unsigned long long p = pk.make(c1, e1) + pk.make(c2, e2);
      CHECK(pk.count(p) == c1 + c2 && pk.edges(p) == e1 + e2, "packed add (%lld,%lld)+(%lld,%lld)", c1, e1, c2, e2);
    }
  }
}

static void check_mark_bits() {
  for (unsigned m = 0; m < 16; ++m) {
    unsigned x = 0;  // byte j = 1 for each bit j of m
    for (int j = 0; j < 4; ++j)
      if ((m >> j) & 1u) x |= 1u << (8 * j);
    CHECK(gbfs::mark_bits(x) == m, "mark_bits(0x%08x) = %u, want %u", x, gbfs::mark_bits(x), m);
  }
}

int main() {
  for (int t = 0; t < 300; ++t) {
    check_binsearch<int32_t>(1 + below(300), 1 + below(5000));
    check_binsearch<int64_t>(1 + below(300), 1 + below(1ll << 20));
  }
  check_binsearch<int32_t>(1, 1);  // a single entry
  for (int t = 0; t < 300; ++t) {
    check_chunks<int32_t>(1 + below(400), 1 + below(20000), 0);
    check_chunks<int64_t>(1 + below(400), 1 + below(1ll << 16), (int64_t)below(1ll << 33));
  }
  check_packed();
  check_mark_bits();
  if (failures) {
    std::printf("%d failures\n", failures);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
