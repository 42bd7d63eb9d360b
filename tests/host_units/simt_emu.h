// A small SIMT emulator for CPU unit tests of the library's warp- and block-collective
// helpers: every emulated GPU thread is an OS thread; the warp intrinsics the helpers use
// (__ballot_sync, __any_sync, __shfl_sync, __shfl_up_sync, full-warp masks only) exchange
// values through a per-warp slot array between two barriers, __syncwarp and __syncthreads
// are warp and block barriers, and the device atomics the headers use act on host memory. The
// intrinsic semantics follow the CUDA programming guide's definitions. Included ahead of the
// library headers (g++ -include), in place of their CUDA device environment.
#pragma once
#include <cassert>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

struct gbfs_host_dim3 {
  unsigned x, y, z;
};
extern thread_local gbfs_host_dim3 threadIdx, blockIdx;
extern gbfs_host_dim3 blockDim, gridDim;

namespace simt {

struct Barrier {
  std::mutex m;
  std::condition_variable cv;
  int n = 0, arrived = 0;
  unsigned long gen = 0;
  void wait() {
    std::unique_lock<std::mutex> lk(m);
    const unsigned long g = gen;
    if (++arrived == n) {
      arrived = 0;
      ++gen;
      cv.notify_all();
      return;
    }
    cv.wait(lk, [&] { return gen != g; });
  }
};

struct Warp {
  Barrier bar;
  uint64_t slot[32];
};

struct Block {
  Barrier bar;
  std::vector<Warp> warps;
};

extern thread_local Block* t_block;

// Every lane of the calling warp contributes v; out receives all 32 contributions.
inline void exchange(uint64_t v, uint64_t out[32]) {
  Warp& w = t_block->warps[threadIdx.x / 32];
  w.slot[threadIdx.x % 32] = v;
  w.bar.wait();
  std::memcpy(out, w.slot, sizeof w.slot);
  w.bar.wait();  // nobody overwrites a slot before every lane has read it
}

template <class T>
uint64_t to_bits(T v) {
  static_assert(sizeof(T) <= 8, "64-bit values at most");
  uint64_t b = 0;
  std::memcpy(&b, &v, sizeof(T));
  return b;
}
template <class T>
T from_bits(uint64_t b) {
  T v;
  std::memcpy(&v, &b, sizeof(T));
  return v;
}

// Runs f on one block of nthreads emulated threads (a multiple of 32), block index bx.
inline void run_block(int nthreads, unsigned bx, const std::function<void()>& f) {
  assert(nthreads % 32 == 0 && nthreads > 0);
  Block blk;
  blk.bar.n = nthreads;
  blk.warps = std::vector<Warp>((size_t)nthreads / 32);
  for (auto& w : blk.warps) w.bar.n = 32;
  blockDim = gbfs_host_dim3{(unsigned)nthreads, 1, 1};
  std::vector<std::thread> ts;
  ts.reserve((size_t)nthreads);
  for (int i = 0; i < nthreads; ++i)
    ts.emplace_back([&, i] {
      threadIdx = gbfs_host_dim3{(unsigned)i, 0, 0};
      blockIdx = gbfs_host_dim3{bx, 0, 0};
      t_block = &blk;
      f();
    });
  for (auto& t : ts) t.join();
}

}  // namespace simt

inline unsigned __ballot_sync(unsigned mask, int pred) {
  assert(mask == 0xffffffffu);
  uint64_t all[32];
  simt::exchange(pred ? 1u : 0u, all);
  unsigned r = 0;
  for (int l = 0; l < 32; ++l) r |= (all[l] ? 1u : 0u) << l;
  return r;
}

template <class T>
T __shfl_sync(unsigned mask, T v, int src) {
  assert(mask == 0xffffffffu);
  uint64_t all[32];
  simt::exchange(simt::to_bits(v), all);
  return simt::from_bits<T>(all[src & 31]);
}

template <class T>
T __shfl_up_sync(unsigned mask, T v, unsigned d) {
  assert(mask == 0xffffffffu);
  uint64_t all[32];
  simt::exchange(simt::to_bits(v), all);
  const unsigned lane = threadIdx.x % 32;
  return lane >= d ? simt::from_bits<T>(all[lane - d]) : v;
}

inline int __any_sync(unsigned mask, int pred) { return __ballot_sync(mask, pred) != 0u; }

inline int __ffs(unsigned x) { return __builtin_ffs((int)x); }
inline int __ffsll(long long x) { return __builtin_ffsll(x); }
inline int __popc(unsigned x) { return __builtin_popcount(x); }
inline void __syncthreads() { simt::t_block->bar.wait(); }
inline void __syncwarp(unsigned mask = 0xffffffffu) {
  assert(mask == 0xffffffffu);
  simt::t_block->warps[threadIdx.x / 32].bar.wait();
}
inline int min(int x, int y) { return x < y ? x : y; }  // the device integer min

// Device atomics on host memory (sequentially consistent; each returns the old value).
inline unsigned long long atomicAdd(unsigned long long* p, unsigned long long v) {
  return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST);
}
inline int atomicAdd(int* p, int v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
inline unsigned long long atomicOr(unsigned long long* p, unsigned long long v) {
  return __atomic_fetch_or(p, v, __ATOMIC_SEQ_CST);
}
inline int atomicCAS(int* p, int cmp, int val) {
  __atomic_compare_exchange_n(p, &cmp, val, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST);
  return cmp;
}
unsigned __ldcg(const unsigned*);  // declared for the headers; not used by these tests
template <class T>
T __ldg(const T* p) {  // read-only load: a plain load on the host
  return *p;
}
