// CPU unit tests of the library's warp- and block-collective helpers, run on the SIMT
// emulator of simt_emu.h:
//  * warp_inclusive_scan against std::inclusive_scan (int32, int64);
//  * block_exclusive_scan against std::exclusive_scan and the block total, 1 to 8 warps
//    (the exclusive scan of frontier degrees, Sec. 3.4);
//  * write_chunks_warp / write_descs_warp against the per-entry write_chunks / write_descs
//    for warps mixing invalid lanes, zero degrees, short rows and hub rows that cross more
//    than 32 chunk boundaries (written by the whole warp).
// Prints "ok" and returns 0, or reports the first failure and returns 1.
#include <algorithm>
#include <cstdio>
#include <numeric>
#include <vector>

#include "device_util.cuh"

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
#define CHECK(cond, ...)                                   \
  do {                                                     \
    if (!(cond) && failures++ == 0) {                      \
      std::printf("FAIL %s:%d: ", __FILE__, __LINE__);     \
      std::printf(__VA_ARGS__);                            \
      std::printf("\n");                                   \
    }                                                      \
  } while (0)

template <typename T>
static void check_warp_scan(T range) {
  std::vector<T> x(64), got(64);
  for (auto& v : x) v = (T)below((int64_t)range);
  simt::run_block(64, 0, [&] { got[threadIdx.x] = gbfs::warp_inclusive_scan<T>(x[threadIdx.x]); });
  for (int w = 0; w < 2; ++w) {
    std::vector<T> want(32);
    std::inclusive_scan(x.begin() + 32 * w, x.begin() + 32 * w + 32, want.begin());
    for (int l = 0; l < 32; ++l)
      CHECK(got[32 * w + l] == want[l], "warp_inclusive_scan warp %d lane %d: %lld want %lld", w, l,
            (long long)got[32 * w + l], (long long)want[l]);
  }
}

template <typename T>
static void check_block_scan(int nthreads, T range) {
  std::vector<T> x((size_t)nthreads), got((size_t)nthreads), tot((size_t)nthreads);
  for (auto& v : x) v = below(4) == 0 ? 0 : (T)below((int64_t)range);
  std::vector<T> s_warp(33);
  simt::run_block(nthreads, 0, [&] {
    T total;
    got[threadIdx.x] = gbfs::block_exclusive_scan<T>(x[threadIdx.x], s_warp.data(), &total);
    tot[threadIdx.x] = total;
  });
  std::vector<T> want((size_t)nthreads);
  std::exclusive_scan(x.begin(), x.end(), want.begin(), (T)0);
  const T sum = std::accumulate(x.begin(), x.end(), (T)0);
  for (int i = 0; i < nthreads; ++i) {
    CHECK(got[(size_t)i] == want[(size_t)i], "block_exclusive_scan(%d threads) thread %d: %lld want %lld", nthreads, i,
          (long long)got[(size_t)i], (long long)want[(size_t)i]);
    CHECK(tot[(size_t)i] == sum, "block_exclusive_scan total %lld want %lld", (long long)tot[(size_t)i],
          (long long)sum);
  }
}

template <typename OffT>
static void check_warp_writers(OffT start, int64_t hub) {
  // one entry per lane: valid flag, degree, scan position, entry index, caller id, base
  std::vector<int> valid(32);
  std::vector<OffT> deg(32), cum(32), base(32);
  std::vector<int32_t> k(32), u(32);
  OffT acc = start;
  for (int l = 0; l < 32; ++l) {
    valid[(size_t)l] = below(8) != 0;
    const int64_t r = below(10);
    deg[(size_t)l] = valid[(size_t)l] ? (OffT)(r < 2 ? 0 : r < 7 ? below(300) : below(hub)) : 0;
    cum[(size_t)l] = acc;
    acc += deg[(size_t)l];
    k[(size_t)l] = (int32_t)(100 + l);
    u[(size_t)l] = (int32_t)(7000 + 3 * l);
    base[(size_t)l] = (OffT)(5000 * l) - cum[(size_t)l];
  }
  const OffT c_lo = start / kChunk, c_hi = acc / kChunk + 2;
  const size_t nc = (size_t)(c_hi - c_lo);
  std::vector<int32_t> chunk_w(nc, -7), chunk_s(nc, -7);
  std::vector<gbfs::TileDesc<OffT>> desc_w(nc, {-7, -7, (OffT)-7}), desc_s(nc, {-7, -7, (OffT)-7});
  simt::run_block(32, 0, [&] {
    const int l = (int)threadIdx.x;
    gbfs::write_chunks_warp<OffT>(chunk_w.data() - c_lo, valid[(size_t)l], cum[(size_t)l], deg[(size_t)l],
                                  k[(size_t)l]);
    gbfs::write_descs_warp<OffT>(desc_w.data() - c_lo, valid[(size_t)l], cum[(size_t)l], deg[(size_t)l], k[(size_t)l],
                                 u[(size_t)l], base[(size_t)l]);
  });
  for (int l = 0; l < 32; ++l)
    if (valid[(size_t)l]) {
      gbfs::write_chunks<OffT>(chunk_s.data() - c_lo, cum[(size_t)l], deg[(size_t)l], k[(size_t)l]);
      gbfs::write_descs<OffT>(desc_s.data() - c_lo, cum[(size_t)l], deg[(size_t)l], k[(size_t)l], u[(size_t)l],
                              base[(size_t)l]);
    }
  for (size_t i = 0; i < nc; ++i) {
    CHECK(chunk_w[i] == chunk_s[i], "write_chunks_warp chunk %lld: %d want %d", (long long)(c_lo + (OffT)i),
          chunk_w[i], chunk_s[i]);
    CHECK(desc_w[i].k == desc_s[i].k && desc_w[i].u == desc_s[i].u && desc_w[i].col == desc_s[i].col,
          "write_descs_warp desc %lld differs", (long long)(c_lo + (OffT)i));
  }
}

int main() {
  for (int t = 0; t < 8; ++t) {
    check_warp_scan<int32_t>(1000);
    check_warp_scan<int64_t>(1ll << 40);
  }
  for (int nthreads : {32, 64, 128, 256})
    for (int t = 0; t < 3; ++t) {
      check_block_scan<int32_t>(nthreads, 5000);
      check_block_scan<int64_t>(nthreads, 1ll << 36);
    }
  for (int t = 0; t < 25; ++t) {
    check_warp_writers<int32_t>((int32_t)below(1 << 20), 40 * kChunk);
    check_warp_writers<int64_t>((int64_t)below(1ll << 34), 200 * kChunk);
  }
  if (failures) {
    std::printf("%d failures\n", failures);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
