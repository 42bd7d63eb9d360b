// CPU unit tests of where a batched wave's claims go (record_claim and the helpers it calls
// in batch.h), run as host code. A claim of one root bit is written out at once (level = wave
// level minus the slot's start, parent u, at the caller id); a claim of several bits takes the
// vertex's next event slot, past the slots its dense row (handed out on first use, or row v
// when the pool holds one per vertex), past a spent pool the overflow list, and past a full
// list it is written out at once. Random claim streams (each root claims a vertex at most
// once, as the visited masks ensure), with and without a caller-id map, with pools and lists
// sized to run out mid-stream, run on one thread and on 64 emulated threads at once (two
// first claims of one vertex racing for a dense row); afterwards every claimed (root, vertex)
// pair must be found exactly once, in an output entry, an event slot, a dense row or an
// overflow record, with its claim's parent and wave level, and record_claim must have
// reported a record exactly for the claims it recorded.
// Prints "ok" and returns 0, or reports the first failure and returns 1.
#include <cstdint>
#include <cstdio>
#include <map>
#include <utility>
#include <vector>

#include "batch.h"

thread_local gbfs_host_dim3 threadIdx, blockIdx;
gbfs_host_dim3 blockDim, gridDim;
thread_local simt::Block* simt::t_block;

using gbfs::kMaxWave;

static uint64_t rng_state = 0xD1B54A32D192ED03ull;
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

struct Claim {
  int32_t v;                // internal id
  unsigned long long bits;  // root bits claimed together
  int32_t u;                // parent (caller id)
  int L;                    // wave level
};

// ev_slots event slots per vertex, dense_cap rows (ident: one per vertex), ovf_cap overflow
// records; `threads` emulated threads share the claims (1: in stream order).
static void check_stream(int n, int ev_slots, long long dense_cap, bool ident, long long ovf_cap, bool relabel,
                         int n_claims, int threads) {
  // the stream: each (root bit, vertex) claimed at most once
  std::vector<unsigned long long> taken((size_t)n, 0ull);
  std::vector<Claim> claims;
  for (int i = 0; i < n_claims; ++i) {
    const int32_t v = (int32_t)below(n);
    unsigned long long bits = 0ull;
    const int k = below(4) == 0 ? 1 : 2 + (int)below(6);  // single-bit claims and multi-bit ones
    for (int j = 0; j < k; ++j) bits |= 1ull << below(kMaxWave);
    bits &= ~taken[(size_t)v];
    if (!bits) continue;
    taken[(size_t)v] |= bits;
    claims.push_back(Claim{v, bits, (int32_t)below(1 << 20), 1 + (int)below(40)});
  }
  std::vector<int32_t> old_id((size_t)n);
  for (int v = 0; v < n; ++v) old_id[(size_t)v] = v;
  if (relabel)
    for (int v = n - 1; v > 0; --v) std::swap(old_id[(size_t)v], old_id[(size_t)below(v + 1)]);
  // buffers, filled with sentinels
  std::vector<int32_t> evc((size_t)n, 0), dense_idx((size_t)n, -1);
  std::vector<gbfs::ClaimEvent> ev((size_t)n * ev_slots + 1, gbfs::ClaimEvent{-9, -9, 0ull});  // + a sentinel
  const long long rows = ident ? n : dense_cap;
  std::vector<int32_t> dpar((size_t)(rows * kMaxWave + 1), -9), dlvl((size_t)(rows * kMaxWave + 1), -9);
  std::vector<unsigned long long> dmask((size_t)rows + 1, 0ull);
  std::vector<gbfs::OvfEvent> ovf((size_t)ovf_cap + 1, gbfs::OvfEvent{-9, -9, 0ull, -9, 0});
  std::vector<std::vector<int32_t>> par(kMaxWave, std::vector<int32_t>((size_t)n, -9)),
      lvl(kMaxWave, std::vector<int32_t>((size_t)n, -9));
  int32_t* s_par[kMaxWave];
  int32_t* s_lvl[kMaxWave];
  int32_t s_start[kMaxWave];
  for (int b = 0; b < kMaxWave; ++b) {
    s_par[b] = par[(size_t)b].data();
    s_lvl[b] = lvl[(size_t)b].data();
    s_start[b] = (int32_t)below(2);
  }
  gbfs::BatchCtl ctl{};
  gbfs::BatchArgs<int32_t> a{};
  a.n = n;
  a.ctl = &ctl;
  a.evc = evc.data();
  a.ev = ev.data();
  a.ev_slots = ev_slots;
  a.ovf = ovf.data();
  a.ovf_cap = ovf_cap;
  a.old_id = relabel ? old_id.data() : nullptr;
  a.dense_ident = ident ? 1 : 0;
  a.dense_idx = ident ? nullptr : (rows > 0 ? dense_idx.data() : nullptr);
  a.dense_par = dpar.data();
  a.dense_lvl = dlvl.data();
  a.dense_mask = dmask.data();
  a.dense_cap = rows;
  std::vector<char> recorded(claims.size(), 0);
  auto run = [&](size_t i) {  // the claim path of the expansion for claim i
    const Claim& c = claims[i];
    const int slot = gbfs::single_bit(c.bits) ? 0 : atomicAdd(a.evc + c.v, 1);
    recorded[i] = gbfs::record_claim(a, c.v, c.bits, c.u, c.L, slot, s_par, s_lvl, s_start) ? 1 : 0;
  };
  if (threads <= 1) {
    for (size_t i = 0; i < claims.size(); ++i) run(i);
  } else {
    simt::run_block(threads, 0, [&] {
      for (size_t i = threadIdx.x; i < claims.size(); i += (size_t)threads) run(i);
    });
  }
  // every (bit, caller vertex) found, once, where the claim put it
  std::map<std::pair<int, int32_t>, std::pair<int32_t, int>> want;  // -> (u, L)
  for (const Claim& c : claims)
    for (int b = 0; b < kMaxWave; ++b)
      if ((c.bits >> b) & 1ull) want[{b, old_id[(size_t)c.v]}] = {c.u, c.L};
  std::map<std::pair<int, int32_t>, int> found;
  auto see = [&](int b, int32_t vc, int32_t u, int L, const char* where) {
    const auto key = std::make_pair(b, vc);
    ++found[key];
    auto it = want.find(key);
    CHECK(it != want.end(), "%s holds bit %d of vertex %d, never claimed", where, b, vc);
    if (it != want.end())
      CHECK(it->second.first == u && it->second.second == L, "%s: bit %d of vertex %d = (%d, %d), want (%d, %d)",
            where, b, vc, u, L, it->second.first, it->second.second);
  };
  for (int b = 0; b < kMaxWave; ++b)
    for (int32_t vc = 0; vc < n; ++vc)
      if (par[(size_t)b][(size_t)vc] != -9) see(b, vc, par[(size_t)b][(size_t)vc], lvl[(size_t)b][(size_t)vc] + s_start[b], "output");
  for (int32_t v = 0; v < n; ++v) {
    const int used = evc[(size_t)v] < ev_slots ? evc[(size_t)v] : ev_slots;
    for (int s = 0; s < used; ++s) {
      const gbfs::ClaimEvent& e = ev[(size_t)v * ev_slots + s];
      CHECK(e.mask != 0ull, "event slot %d of vertex %d empty", s, v);
      for (int b = 0; b < kMaxWave; ++b)
        if ((e.mask >> b) & 1ull) see(b, old_id[(size_t)v], e.u, e.level, "event slot");
    }
    for (int s = used; s < ev_slots; ++s) CHECK(ev[(size_t)v * ev_slots + s].u == -9, "unused slot written");
    const int32_t row = ident ? v : dense_idx[(size_t)v];
    if (row < 0) continue;
    for (int b = 0; b < kMaxWave; ++b)
      if ((dmask[(size_t)row] >> b) & 1ull)
        see(b, old_id[(size_t)v], dpar[(size_t)row * kMaxWave + b], dlvl[(size_t)row * kMaxWave + b], "dense row");
  }
  const long long n_ovf = (long long)ctl.ovf_count < ovf_cap ? (long long)ctl.ovf_count : ovf_cap;
  for (long long o = 0; o < n_ovf; ++o)
    for (int b = 0; b < kMaxWave; ++b)
      if ((ovf[(size_t)o].mask >> b) & 1ull) see(b, ovf[(size_t)o].v, ovf[(size_t)o].u, ovf[(size_t)o].level, "overflow");
  CHECK(ovf[(size_t)ovf_cap].v == -9, "overflow record past the list's end written");
  CHECK(ev[(size_t)n * ev_slots].u == -9, "event slot past the last vertex's written");
  for (const auto& kv : want)
    CHECK(found[kv.first] == 1, "bit %d of vertex %d found %d times", kv.first.first, kv.first.second, found[kv.first]);
  // a record reported exactly when the claim did not go straight to the outputs
  for (size_t i = 0; i < claims.size(); ++i) {
    const Claim& c = claims[i];
    const int b = __builtin_ctzll(c.bits);
    const bool direct = par[(size_t)b][(size_t)old_id[(size_t)c.v]] != -9;
    CHECK(recorded[i] == (direct ? 0 : 1), "claim %zu: record_claim returned %d, outputs %s", i, recorded[i],
          direct ? "written" : "untouched");
  }
}

int main() {
  // (n, event slots, dense rows, one row per vertex, overflow records, caller-id map, claims, threads)
  check_stream(40, 2, 0, false, 0, false, 400, 1);     // no pool, no list: past the slots straight out
  check_stream(40, 2, 5, false, 0, true, 400, 1);      // the pool runs out, then straight out
  check_stream(40, 2, 5, false, 30, true, 600, 1);     // pool, then list, then straight out
  check_stream(40, 8, 0, true, 10, false, 800, 1);     // a row per vertex
  check_stream(300, 4, 20, false, 50, true, 3000, 1);
  check_stream(60, 2, 8, false, 40, true, 1500, 64);   // racing first claims of a row
  check_stream(60, 8, 0, true, 20, true, 1500, 64);
  for (int t = 0; t < 20; ++t) {
    const int n = 1 + (int)below(200);
    check_stream(n, 1 + (int)below(8), below(3) == 0 ? 0 : below(n), below(3) == 0, below(4) == 0 ? 0 : below(300),
                 below(2) == 0, (int)below(4000), below(2) == 0 ? 1 : 32 * (1 + (int)below(3)));
  }
  if (failures) {
    std::printf("%d failures\n", failures);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
