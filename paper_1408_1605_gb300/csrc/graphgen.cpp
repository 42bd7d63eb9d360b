// Seeded synthetic graph inputs: R-MAT, uniform G(n,m) and 3D-grid edge lists, a
// symmetric CSR builder and a root picker.
//
// This is input preparation, shared by the CPU oracle tests and the GPU path alike. It
// holds none of the BFS arithmetic. The R-MAT workload stands in for the Graph500
// generator the paper uses (Sec. 3.2 and Sec. 4: R-MAT, about edge_factor * 2^scale
// edges, each edge made undirected by adding its opposite). The Graph500 code itself is
// not available, so this is an own generator with the same parameters; byte parity with
// Graph500 is not claimed.
//
// Randomness: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014) used as a counter-based generator: value(i) = mix(state0 +
// (i + 1) * gamma). Every random draw is a pure function of (seed, stream, index), so the
// output does not depend on the thread count.

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Independent streams per purpose, so that e.g. the permutation never reuses edge draws.
enum : uint64_t { kStreamRmat = 1, kStreamPerm = 2, kStreamUniform = 3, kStreamRoots = 4 };

inline uint64_t stream_state(uint64_t seed, uint64_t stream) {
  return mix64(seed * kGamma + stream * 0xD1B54A32D192ED03ull + 0x2545F4914F6CDD1Dull);
}

inline uint64_t draw(uint64_t state0, uint64_t index) { return mix64(state0 + (index + 1) * kGamma); }

// Uniform integer in [0, bound) by the multiply-high method (Lemire 2019).
inline uint64_t bounded(uint64_t r, uint64_t bound) {
  return (uint64_t)(((unsigned __int128)r * bound) >> 64);
}

int thread_count(int requested) {
  if (requested > 0) return requested;
  const char* env = std::getenv("GBFS_GEN_THREADS");
  if (env && std::atoi(env) > 0) return std::atoi(env);
  unsigned hc = std::thread::hardware_concurrency();
  return hc ? (int)hc : 1;
}

template <class F>
void parallel_for(int64_t n, int nthreads, F&& fn) {
  if (n <= 0) return;
  nthreads = (int)std::max<int64_t>(1, std::min<int64_t>(nthreads, n));
  if (nthreads == 1) {
    fn(0, n);
    return;
  }
  std::vector<std::thread> pool;
  pool.reserve(nthreads);
  for (int t = 0; t < nthreads; ++t) {
    int64_t lo = n * t / nthreads, hi = n * (t + 1) / nthreads;
    pool.emplace_back([&fn, lo, hi] { fn(lo, hi); });
  }
  for (auto& th : pool) th.join();
}

// Dynamic scheduling in chunks, for work with skewed cost (rows of R-MAT graphs).
template <class F>
void parallel_chunks(int64_t n, int64_t chunk, int nthreads, F&& fn) {
  if (n <= 0) return;
  std::atomic<int64_t> next{0};
  auto worker = [&] {
    for (;;) {
      int64_t lo = next.fetch_add(chunk, std::memory_order_relaxed);
      if (lo >= n) break;
      fn(lo, std::min(n, lo + chunk));
    }
  };
  nthreads = (int)std::max<int64_t>(1, std::min<int64_t>(nthreads, (n + chunk - 1) / chunk));
  std::vector<std::thread> pool;
  for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
}

// Text edge lists, the form in which public graph collections such as SNAP (the source of
// the paper's real-world inputs, Sec. 5, Table 3) distribute their graphs: one pair "u v"
// per line, ids non-negative decimal integers separated by blanks, tabs or a comma. Blank
// lines and lines that start with '#' or '%' are skipped, anything after the second id
// (a weight, a timestamp) is ignored, and a '\r' before the '\n' is accepted.
struct ParsePiece {
  int64_t pairs = 0;
  int64_t max_id = -1;
  int64_t err_pos = -1;  // byte offset of the first bad line's start
  int err = 0;           // -3: id above INT32_MAX - 1; -5: malformed line
};

inline bool is_blank(char c) { return c == ' ' || c == '\t' || c == '\r' || c == '\v' || c == '\f'; }
inline bool is_sep(char c) { return c == ' ' || c == '\t' || c == ','; }
inline bool is_digit(char c) { return c >= '0' && c <= '9'; }

inline int64_t next_line(const char* text, int64_t len, int64_t p) {
  const void* nl = p < len ? std::memchr(text + p, '\n', (size_t)(len - p)) : nullptr;
  return nl ? (const char*)nl - text + 1 : len;
}

// Parses every line that starts in [lo, hi); a line may run past hi. With src non-NULL
// the pairs are written from index 0 of src / dst. Stops at the first bad line.
ParsePiece parse_lines(const char* text, int64_t len, int64_t lo, int64_t hi, int32_t* src, int32_t* dst) {
  ParsePiece r;
  const uint64_t kMaxId = (uint64_t)INT32_MAX - 1;  // n = max id + 1 must fit in int32
  int64_t p = lo;
  while (p < hi) {
    const int64_t start = p;
    while (p < len && is_blank(text[p])) ++p;
    if (p >= len || text[p] == '\n' || text[p] == '#' || text[p] == '%') {
      p = next_line(text, len, p);
      continue;
    }
    uint64_t id[2] = {0, 0};
    for (int f = 0; f < 2; ++f) {
      if (f == 1) {
        if (p >= len || !is_sep(text[p])) { r.err = -5; r.err_pos = start; return r; }
        while (p < len && is_sep(text[p])) ++p;
      }
      if (p >= len || !is_digit(text[p])) { r.err = -5; r.err_pos = start; return r; }
      uint64_t x = 0;
      for (; p < len && is_digit(text[p]); ++p) {
        x = x * 10 + (uint64_t)(text[p] - '0');
        if (x > kMaxId) { r.err = -3; r.err_pos = start; return r; }
      }
      id[f] = x;
    }
    if (p < len && text[p] != '\n' && !is_sep(text[p]) && !is_blank(text[p])) {
      r.err = -5;
      r.err_pos = start;
      return r;
    }
    if (src) {
      src[r.pairs] = (int32_t)id[0];
      dst[r.pairs] = (int32_t)id[1];
    }
    ++r.pairs;
    r.max_id = std::max<int64_t>(r.max_id, (int64_t)std::max(id[0], id[1]));
    p = next_line(text, len, p);
  }
  return r;
}

}  // namespace

extern "C" {

// Parses a text edge list (format above) held in text[0, len). Pieces of the text, split
// at line starts, are parsed by separate threads; the pairs keep the file's order. With
// src == NULL only counts. Otherwise writes the pairs to src / dst (capacity cap each).
// *max_id receives the largest id (-1 if there is no pair). Returns the number of pairs;
// -1 on bad arguments or too small a capacity; -3 if an id exceeds 2^31 - 2; -5 on a
// malformed line. On -3 / -5, *err_pos receives the byte offset where the first bad line
// starts.
int64_t gg_parse_edge_list(const char* text, int64_t len, int32_t* src, int32_t* dst, int64_t cap,
                           int64_t* max_id, int64_t* err_pos, int nthreads) {
  if (len < 0 || (len > 0 && !text) || (src && (!dst || cap < 0))) return -1;
  nthreads = thread_count(nthreads);
  const int T = (int)std::max<int64_t>(1, std::min<int64_t>(nthreads, len / (1 << 16) + 1));
  std::vector<int64_t> cut((size_t)T + 1, len);
  cut[0] = 0;
  for (int t = 1; t < T; ++t) {
    const int64_t s = len * t / T;
    cut[(size_t)t] = (text[s - 1] == '\n') ? s : next_line(text, len, s);
  }
  for (int t = T - 1; t >= 1; --t) cut[(size_t)t] = std::min(cut[(size_t)t], cut[(size_t)t + 1]);
  std::vector<ParsePiece> part((size_t)T);
  parallel_for(T, T, [&](int64_t t0, int64_t t1) {
    for (int64_t t = t0; t < t1; ++t)
      part[(size_t)t] = parse_lines(text, len, cut[(size_t)t], cut[(size_t)t + 1], nullptr, nullptr);
  });
  int64_t total = 0, mx = -1;
  for (const ParsePiece& q : part) {
    if (q.err) {
      if (err_pos) *err_pos = q.err_pos;
      return q.err;
    }
    total += q.pairs;
    mx = std::max(mx, q.max_id);
  }
  if (max_id) *max_id = mx;
  if (!src) return total;
  if (total > cap) return -1;
  std::vector<int64_t> at((size_t)T, 0);
  for (int t = 1; t < T; ++t) at[(size_t)t] = at[(size_t)t - 1] + part[(size_t)t - 1].pairs;
  parallel_for(T, T, [&](int64_t t0, int64_t t1) {
    for (int64_t t = t0; t < t1; ++t)
      parse_lines(text, len, cut[(size_t)t], cut[(size_t)t + 1], src + at[(size_t)t], dst + at[(size_t)t]);
  });
  return total;
}

// R-MAT edge list: n_edges = edge_factor * 2^scale directed pairs (the undirected edges
// before symmetrization). Quadrant per bit level with probabilities (a, b, c, 1-a-b-c):
// a -> (0,0), b -> (0,1), c -> (1,0), d -> (1,1); the first draw sets the most significant
// bit. With permute != 0 the vertex ids are relabelled by a seeded Fisher-Yates shuffle.
// Returns 0 on success, -1 on bad arguments.
int gg_rmat_edges(int scale, int64_t n_edges, double a, double b, double c, uint64_t seed,
                  int permute, int32_t* src, int32_t* dst, int nthreads) {
  if (scale < 1 || scale > 31 || n_edges < 0 || !src || !dst) return -1;
  if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return -1;
  // Each 64-bit draw serves two bit levels: its high and low 32-bit halves are compared
  // against the cumulative quadrant thresholds scaled to 2^32.
  const double two32 = 4294967296.0;
  const uint64_t tA = (uint64_t)(a * two32);
  const uint64_t tAB = (uint64_t)((a + b) * two32);
  const uint64_t tABC = (uint64_t)((a + b + c) * two32);
  const uint64_t s0 = stream_state(seed, kStreamRmat);
  const uint64_t draws_per_edge = (uint64_t)(scale + 1) / 2;
  nthreads = thread_count(nthreads);
  parallel_for(n_edges, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      uint32_t u = 0, v = 0;
      const uint64_t base = (uint64_t)i * draws_per_edge;
      uint64_t r = 0;
      for (int l = 0; l < scale; ++l) {
        if ((l & 1) == 0) r = draw(s0, base + (uint64_t)(l >> 1));
        const uint64_t x = (l & 1) ? (r & 0xFFFFFFFFull) : (r >> 32);
        // quadrant without branches (they mispredict at these probabilities):
        // [0, tA) -> (0,0), [tA, tAB) -> (0,1), [tAB, tABC) -> (1,0), [tABC, 2^32) -> (1,1)
        const uint32_t ga = x >= tA, gab = x >= tAB, gabc = x >= tABC;
        u = (u << 1) | gab;
        v = (v << 1) | (ga ^ gab ^ gabc);
      }
      src[i] = (int32_t)u;
      dst[i] = (int32_t)v;
    }
  });
  if (permute) {
    const int64_t n = int64_t(1) << scale;
    std::vector<int32_t> perm((size_t)n);
    for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = (int32_t)i;
    const uint64_t p0 = stream_state(seed, kStreamPerm);
    for (int64_t i = n - 1; i > 0; --i) {
      const int64_t j = (int64_t)bounded(draw(p0, (uint64_t)i), (uint64_t)(i + 1));
      std::swap(perm[(size_t)i], perm[(size_t)j]);
    }
    parallel_for(n_edges, nthreads, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) {
        src[i] = perm[(size_t)src[i]];
        dst[i] = perm[(size_t)dst[i]];
      }
    });
  }
  return 0;
}

// Uniform random pairs: both endpoints uniform in [0, n).
int gg_uniform_edges(int64_t n, int64_t n_edges, uint64_t seed, int32_t* src, int32_t* dst,
                     int nthreads) {
  if (n < 1 || n > INT32_MAX || n_edges < 0 || !src || !dst) return -1;
  const uint64_t s0 = stream_state(seed, kStreamUniform);
  parallel_for(n_edges, thread_count(nthreads), [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      src[i] = (int32_t)bounded(draw(s0, 2 * (uint64_t)i), (uint64_t)n);
      dst[i] = (int32_t)bounded(draw(s0, 2 * (uint64_t)i + 1), (uint64_t)n);
    }
  });
  return 0;
}

// Number of undirected edges of the non-periodic X x Y x Z 6-neighbour grid.
int64_t gg_grid3d_edge_count(int64_t X, int64_t Y, int64_t Z) {
  if (X < 1 || Y < 1 || Z < 1) return -1;
  return (X - 1) * Y * Z + X * (Y - 1) * Z + X * Y * (Z - 1);
}

// Non-periodic 3D grid, vertex id = x + X * (y + Y * z); one pair per undirected edge,
// towards +x, +y and +z.
int gg_grid3d_edges(int64_t X, int64_t Y, int64_t Z, int32_t* src, int32_t* dst, int nthreads) {
  if (X < 1 || Y < 1 || Z < 1 || X * Y * Z > INT32_MAX || !src || !dst) return -1;
  // Edges of each z-plane are written at a fixed position, so planes run in parallel.
  const int64_t per_plane_xy = (X - 1) * Y + X * (Y - 1);
  const int64_t per_plane_z = X * Y;
  parallel_for(Z, thread_count(nthreads), [&](int64_t zlo, int64_t zhi) {
    for (int64_t z = zlo; z < zhi; ++z) {
      int64_t e = z * (per_plane_xy + per_plane_z);
      for (int64_t y = 0; y < Y; ++y)
        for (int64_t x = 0; x < X; ++x) {
          const int64_t id = x + X * (y + Y * z);
          if (x + 1 < X) { src[e] = (int32_t)id; dst[e] = (int32_t)(id + 1); ++e; }
          if (y + 1 < Y) { src[e] = (int32_t)id; dst[e] = (int32_t)(id + X); ++e; }
        }
      if (z + 1 < Z)
        for (int64_t i = 0; i < per_plane_z; ++i) {
          const int64_t id = i + X * Y * z;
          src[e] = (int32_t)id;
          dst[e] = (int32_t)(id + X * Y);
          ++e;
        }
    }
  });
  return 0;
}

// Symmetric CSR from an edge list: every pair (u, v) with u != v contributes u->v and
// v->u; self-loops are dropped, each row is sorted ascending and duplicates are removed.
// offsets_out: int64[n + 1]; cols_out: int32 with room for 2 * n_edges entries. On
// success returns the number of CSR entries (offsets_out[n]); -1 on bad arguments, -2 on
// allocation failure, -3 on an endpoint out of range.
int64_t gg_build_csr(int64_t n, int64_t n_edges, const int32_t* src, const int32_t* dst,
                     int64_t* offsets_out, int32_t* cols_out, int nthreads) {
  if (n < 0 || n > INT32_MAX || n_edges < 0 || !offsets_out) return -1;
  if (n_edges > 0 && (!src || !dst || !cols_out)) return -1;
  nthreads = thread_count(nthreads);
  // Both directions of every non-loop pair are first grouped by source bucket (a range of
  // consecutive vertex ids) with per-thread counts, so that no two threads ever write the
  // same place; then each bucket, on its own, is laid out as rows, and every row is sorted
  // and its duplicates removed. (A per-vertex atomic cursor was 4x slower: the R-MAT hubs
  // made every thread contend for the same counters.)
  int bbits = 0;
  while ((int64_t(1) << bbits) < n) ++bbits;
  const int kBucketBits = 12;
  const int shift = std::max(0, bbits - kBucketBits);
  const int64_t nb = n > 0 ? ((n - 1) >> shift) + 1 : 1;  // buckets
  const int T = (int)std::max<int64_t>(1, std::min<int64_t>(nthreads, std::max<int64_t>(n_edges, 1)));
  std::atomic<int> bad{0};
  std::vector<int64_t> cnt, bstart;
  std::vector<int32_t> pu, pv, tmp;
  try {
    cnt.assign((size_t)T * (size_t)nb, 0);
    bstart.assign((size_t)nb + 1, 0);
  } catch (...) {
    return -2;
  }
  auto range = [&](int t, int64_t& lo, int64_t& hi) {
    lo = n_edges * t / T;
    hi = n_edges * (t + 1) / T;
  };
  // 1. per-thread counts per bucket
  parallel_for(T, T, [&](int64_t t0, int64_t t1) {
    for (int64_t t = t0; t < t1; ++t) {
      int64_t lo, hi;
      range((int)t, lo, hi);
      int64_t* c = cnt.data() + (size_t)t * (size_t)nb;
      for (int64_t i = lo; i < hi; ++i) {
        const int32_t u = src[i], v = dst[i];
        if (u < 0 || v < 0 || u >= n || v >= n) { bad.store(1); continue; }
        if (u == v) continue;
        ++c[u >> shift];
        ++c[v >> shift];
      }
    }
  });
  if (bad.load()) return -3;
  // 2. positions: bucket-major, thread-minor
  int64_t acc = 0;
  for (int64_t b = 0; b < nb; ++b) {
    bstart[(size_t)b] = acc;
    for (int t = 0; t < T; ++t) {
      int64_t& c = cnt[(size_t)t * (size_t)nb + (size_t)b];
      const int64_t k = c;
      c = acc;
      acc += k;
    }
  }
  bstart[(size_t)nb] = acc;
  try {
    pu.resize((size_t)acc);
    pv.resize((size_t)acc);
    tmp.resize((size_t)acc);
  } catch (...) {
    return -2;
  }
  // 3. scatter the pairs into their buckets (each thread into its own slots)
  parallel_for(T, T, [&](int64_t t0, int64_t t1) {
    for (int64_t t = t0; t < t1; ++t) {
      int64_t lo, hi;
      range((int)t, lo, hi);
      int64_t* c = cnt.data() + (size_t)t * (size_t)nb;
      for (int64_t i = lo; i < hi; ++i) {
        const int32_t u = src[i], v = dst[i];
        if (u == v) continue;
        int64_t p = c[u >> shift]++;
        pu[(size_t)p] = u;
        pv[(size_t)p] = v;
        p = c[v >> shift]++;
        pu[(size_t)p] = v;
        pv[(size_t)p] = u;
      }
    }
  });
  // 4. per bucket: rows (counting sort by source), then sort + dedup each row
  std::vector<int64_t> off((size_t)n + 1, 0), newdeg((size_t)n + 1, 0);
  parallel_chunks(nb, 1, nthreads, [&](int64_t b0, int64_t b1) {
    std::vector<int64_t> cur;
    for (int64_t b = b0; b < b1; ++b) {
      const int64_t vlo = b << shift, vhi = std::min<int64_t>(n, (b + 1) << shift);
      const int64_t plo = bstart[(size_t)b], phi = bstart[(size_t)b + 1];
      cur.assign((size_t)(vhi - vlo) + 1, 0);
      for (int64_t p = plo; p < phi; ++p) ++cur[(size_t)(pu[(size_t)p] - vlo) + 1];
      for (int64_t k = 0; k < vhi - vlo; ++k) cur[(size_t)k + 1] += cur[(size_t)k];
      for (int64_t u = vlo; u < vhi; ++u) off[(size_t)u] = plo + cur[(size_t)(u - vlo)];
      for (int64_t p = plo; p < phi; ++p) tmp[(size_t)(plo + cur[(size_t)(pu[(size_t)p] - vlo)]++)] = pv[(size_t)p];
      for (int64_t u = vlo; u < vhi; ++u) {
        int32_t* rb = tmp.data() + off[(size_t)u];
        int32_t* re = tmp.data() + (u + 1 < vhi ? off[(size_t)u + 1] : phi);
        std::sort(rb, re);
        newdeg[(size_t)u] = std::unique(rb, re) - rb;
      }
    }
  });
  off[(size_t)n] = acc;
  pu.clear();
  pu.shrink_to_fit();
  pv.clear();
  pv.shrink_to_fit();
  // 5. compacted offsets and copy
  acc = 0;
  for (int64_t u = 0; u < n; ++u) {
    offsets_out[u] = acc;
    acc += newdeg[(size_t)u];
  }
  offsets_out[n] = acc;
  parallel_chunks(n, 4096, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t u = lo; u < hi; ++u) {
      const int64_t d = newdeg[(size_t)u];
      if (d) std::memcpy(cols_out + offsets_out[u], tmp.data() + off[(size_t)u], (size_t)d * sizeof(int32_t));
    }
  });
  return acc;
}

// k distinct roots with degree > 0, drawn from the seeded stream in order. Returns the
// number written (< k only if fewer than k vertices have degree > 0).
int64_t gg_pick_roots(int64_t n, const int64_t* offsets, int64_t k, uint64_t seed, int32_t* out) {
  if (n < 1 || !offsets || k < 0 || (k > 0 && !out)) return -1;
  int64_t eligible = 0;
  for (int64_t v = 0; v < n; ++v) eligible += offsets[v + 1] > offsets[v];
  const int64_t want = std::min(k, eligible);
  std::vector<uint8_t> taken((size_t)n, 0);
  const uint64_t s0 = stream_state(seed, kStreamRoots);
  int64_t got = 0;
  for (uint64_t t = 0; got < want; ++t) {
    const int64_t v = (int64_t)bounded(draw(s0, t), (uint64_t)n);
    if (offsets[v + 1] == offsets[v] || taken[(size_t)v]) continue;
    taken[(size_t)v] = 1;
    out[got++] = (int32_t)v;
  }
  return got;
}

}  // extern "C"
