// Serving loop: BFS queries on resident graphs with continuous batching.
//
// Each graph added to a server gets its own wave (multi-source state with 64 bit-slots,
// see bfs_batch_kernels.cu), its own CUDA stream and its own scheduler thread, so the waves
// of different graphs run concurrently on the device and a slow wave does not hold back a
// fast one. A wave advances in bursts of levels; between two bursts its thread
//   * retires slots whose bit left every frontier (the query is complete: its outputs are
//     final), copying results to host buffers where the caller gave host memory;
//   * admits pending queries into free slots, in arrival order per graph, as long as the
//     device-memory budget allows (a query with host outputs needs a device staging buffer
//     of 8 bytes per vertex, charged to the budget until it completes). A query admitted at
//     wave level t starts from its root at that level, so admission never restarts a wave;
//     its levels are the wave level minus t, which makes each result identical to the
//     same query run alone.
// The paper has no serving layer; each query's search is Algorithm 2 / Algorithm 3 with
// R = C = 1, run as one bit of a multi-source wave.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "batch.h"
#include "capi_internal.h"
#include "gbfs.h"

namespace gbfs {

using Clock = std::chrono::steady_clock;

enum ReqState { kPending = 0, kRunning = 1, kDone = 2 };

struct ServeReq {
  uint64_t ticket = 0;
  int graph_id = 0;
  int32_t root = 0;
  int32_t* user_lvl = nullptr;
  int32_t* user_par = nullptr;
  bool host_out = false;
  int32_t* dev_lvl = nullptr;  // where the kernels write
  int32_t* dev_par = nullptr;
  size_t charged = 0;
  int slot = -1;
  int start = 0;               // wave frontier index at admission
  int state = kPending;
  bool cancel = false;
  bfs_status status = BFS_OK;
  std::string message;
  bfs_stats stats{};
  Clock::time_point t_submit, t_admit, t_done;
};

struct ServeGraph;

struct Wave {
  bfs_graph_s* G = nullptr;
  ServeGraph* sg = nullptr;
  GraphDev g;
  BatchBufs b;
  cudaStream_t stream = nullptr;
  int grid = 0;
  int shape = 0;
  int burst = 1;                      // levels to run in the current scheduler round
  std::atomic<bool> active{false};     // read by sibling waves' threads
  std::atomic<int> t{0};              // frontier index the next expansion reads
  uint64_t used = 0;                  // occupied slot bits
  ServeReq* slot_req[kMaxWave] = {};
  WaveSlots* slots_host = nullptr;    // pinned
  BatchCtl* ctl_host = nullptr;       // pinned
  RootSeed* seeds_host = nullptr;     // pinned
  long long* stats_host = nullptr;    // pinned, 3 per slot
  long long* stats_dev = nullptr;     // device, 3 per slot
  unsigned long long pending_clear = 0;  // bits to clear from V before reuse
  Clock::time_point t_cohort;           // when the running cohort started
};

// A resident graph: its queue of pending queries, shared by its waves, and the mean depth
// of its completed queries (deep graphs admit continuously, see young()).
struct ServeGraph {
  int id = 0;
  GraphDev g;
  std::deque<ServeReq*> pending;
  std::vector<Wave*> waves;
  double depth_sum = 0;
  long long depth_n = 0;
  double wave_ms = 0;  // moving average of a cohort's duration, start to last retirement
};

}  // namespace gbfs

struct bfs_server_s {
  bfs_serve_config cfg{};
  int device = -1;
  std::vector<gbfs::Wave*> waves;          // every wave of every graph
  std::vector<gbfs::ServeGraph*> graphs;
  std::map<uint64_t, gbfs::ServeReq*> reqs;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<std::thread> threads;  // one scheduler thread per wave
  bool stop = false;
  bool started = false;
  uint64_t next_ticket = 1;
  size_t mem_used = 0, mem_peak = 0, mem_fixed = 0;
  // report
  uint64_t submitted = 0, completed = 0, cancelled = 0, rejected = 0, failed = 0, levels = 0;
  int running = 0, max_running = 0;
  std::vector<double> latencies_ms;
  long long edges_done = 0;
  bool have_first = false;
  gbfs::Clock::time_point first_submit, last_done;
  std::string fatal;
};

namespace gbfs {

static void free_wave(Wave* w) {
  if (!w) return;
  free_batch_bufs(w->b);
  if (w->stream) cudaStreamDestroy(w->stream);
  if (w->slots_host) cudaFreeHost(w->slots_host);
  if (w->ctl_host) cudaFreeHost(w->ctl_host);
  if (w->seeds_host) cudaFreeHost(w->seeds_host);
  if (w->stats_host) cudaFreeHost(w->stats_host);
  cudaFree(w->stats_dev);
  delete w;
}

template <typename OffT>
static void wave_launch_level(Wave* w) {
  BatchArgs<OffT> a = make_batch_args<OffT>(w->g, w->b);
  launch_batch_expand<OffT>(w->shape, a, w->grid, w->stream);
  launch_batch_order<OffT>(a, w->g.num_sms, w->stream);  // before the emit, which reads the list
  launch_batch_emit<OffT>(a, w->g.num_sms, w->stream);
}

template <typename OffT>
static void wave_seed(Wave* w, int n_seeds, bool fresh) {
  BatchArgs<OffT> a = make_batch_args<OffT>(w->g, w->b);
  if (fresh) launch_batch_clear<OffT>(a, w->g.num_sms, w->stream);
  launch_batch_seed<OffT>(a, reinterpret_cast<const RootSeed*>(w->b.roots_dev), n_seeds, 0, fresh, w->stream);
}

static void finish_req(bfs_server_s* S, ServeReq* r, bfs_status st, const std::string& msg) {
  // called with S->mu held
  r->status = st;
  r->message = msg;
  r->state = kDone;
  r->t_done = Clock::now();
  if (r->charged) {
    cudaFree(r->dev_lvl);
    cudaFree(r->dev_par);
    S->mem_used -= r->charged;
    r->charged = 0;
  }
  if (st == BFS_OK) {
    ++S->completed;
    S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    S->edges_done += r->stats.edges_traversed;
    S->last_done = r->t_done;
  } else if (st == BFS_ERR_CANCELLED) {
    ++S->cancelled;
  } else {
    ++S->failed;
  }
}

// Queries admitted into a running wave at different levels share fewer row reads: on
// graphs with few levels (R-MAT) the large levels of all roots cover the same vertices,
// so a wave takes new queries only while its current cohort is young (at most `window`
// levels old) and otherwise leaves them to an idle or younger wave of the same graph. On
// deep graphs the window grows with the graph's mean query depth.
static int admit_window(const bfs_server_s* S, const ServeGraph* sg) {
  const int base = S->cfg.admit_window > 0 ? S->cfg.admit_window : 3;
  const double mean_depth = sg->depth_n ? sg->depth_sum / (double)sg->depth_n : 0.0;
  return std::max(base, (int)(mean_depth / 4.0));
}

static bool wave_can_admit(const bfs_server_s* S, const Wave* w, int cap_slots) {
  bool slot_free = false;
  for (int b = 0; b < cap_slots; ++b) slot_free |= !((w->used >> b) & 1ull);
  if (!slot_free) return false;
  return !w->active || w->t <= admit_window(S, w->sg);
}

// True when a sibling wave of the same graph is running a young cohort with room: an idle
// wave then leaves the pending queries to it rather than starting a cohort of its own.
static bool sibling_takes(const bfs_server_s* S, const Wave* w, int cap_slots) {
  for (const Wave* x : w->sg->waves)
    if (x != w && x->active && wave_can_admit(S, x, cap_slots)) return true;
  return false;
}

// Whether an idle wave may start a new cohort now (with S->mu held). A wave costs nearly
// the same whether one slot or all are busy, so while a sibling wave of the graph keeps the
// device busy, a new cohort waits until the pending queries fill it or the oldest has
// waited cohort_wait_us; *wait_left receives the time still to wait.
static bool cohort_ready(const bfs_server_s* S, const Wave* w, int cap_slots, Clock::duration* wait_left) {
  *wait_left = Clock::duration::zero();
  const std::deque<ServeReq*>& pending = w->sg->pending;
  if (pending.empty()) return false;
  bool sibling_busy = false;
  for (const Wave* x : w->sg->waves) sibling_busy |= x != w && x->active;
  // default: as long as the graph's cohorts take (the wait then costs at most one cohort)
  const long long wait_us = S->cfg.cohort_wait_us != 0 ? (long long)S->cfg.cohort_wait_us
                                                       : (long long)(1000.0 * w->sg->wave_ms);
  if (!sibling_busy || wait_us < 0 || (int)pending.size() >= cap_slots) return true;
  const auto waited = Clock::now() - pending.front()->t_submit;
  const auto budget = std::chrono::microseconds(wait_us);
  if (waited >= budget) return true;
  *wait_left = budget - waited;
  return false;
}

// One round of a wave: admission, seeding, a burst of levels, retirement. Each wave has
// its own scheduler thread, so a slow wave never holds back the others; the shared
// request bookkeeping is guarded by the server lock.
static void wave_round(bfs_server_s* S, Wave* w) {
  std::vector<ServeReq*> admitted;
  unsigned long long drop = 0;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    std::deque<ServeReq*>& pending = w->sg->pending;
    // pending cancellations
    for (auto it = pending.begin(); it != pending.end();) {
      if ((*it)->cancel) {
        finish_req(S, *it, BFS_ERR_CANCELLED, "cancelled before admission");
        it = pending.erase(it);
      } else {
        ++it;
      }
    }
    const int cap_slots = std::max(1, std::min(kMaxWave, S->cfg.max_wave > 0 ? S->cfg.max_wave : kMaxWave));
    Clock::duration wait_left;
    const bool may_admit = wave_can_admit(S, w, cap_slots) &&
                           (w->active || (!sibling_takes(S, w, cap_slots) && cohort_ready(S, w, cap_slots, &wait_left)));
    while (may_admit && !pending.empty()) {
      int free_bit = -1;
      for (int b = 0; b < cap_slots; ++b)
        if (!((w->used >> b) & 1ull)) {
          free_bit = b;
          break;
        }
      if (free_bit < 0) break;
      ServeReq* r = pending.front();
      const size_t need = r->host_out ? (size_t)w->g.n * 8 : 0;
      if (S->cfg.memory_cap_bytes && S->mem_fixed + S->mem_used + need > S->cfg.memory_cap_bytes)
        break;  // FIFO: wait until running queries release memory
      if (need) {
        if (cudaMalloc(reinterpret_cast<void**>(&r->dev_lvl), (size_t)w->g.n * 4) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void**>(&r->dev_par), (size_t)w->g.n * 4) != cudaSuccess) {
          cudaGetLastError();
          cudaFree(r->dev_lvl);
          r->dev_lvl = nullptr;
          break;  // device memory is short: retry once slots complete
        }
        r->charged = need;
        S->mem_used += need;
        S->mem_peak = std::max(S->mem_peak, S->mem_used + S->mem_fixed);
      } else {
        r->dev_lvl = r->user_lvl;
        r->dev_par = r->user_par;
      }
      pending.pop_front();
      r->slot = free_bit;
      r->start = w->active.load() ? w->t.load() : 0;
      r->state = kRunning;
      r->t_admit = Clock::now();
      w->used |= 1ull << free_bit;
      w->slot_req[free_bit] = r;
      admitted.push_back(r);
      ++S->running;
      S->max_running = std::max(S->max_running, S->running);
    }
    // When this wave cannot take the queries that are waiting (none waiting, no slot, or
    // its cohort is too old), run several levels before looking again: a root's bit never
    // returns to a frontier once its search is done, so the alive mask after the burst
    // still shows every query that finished in it. Deep graphs (hundreds of levels) run
    // longer bursts, also while admitting: a round trip to the host per level would cost
    // far more than the level itself.
    const int lpr = S->cfg.levels_per_round > 0 ? S->cfg.levels_per_round : 8;
    const int depth = w->sg->depth_n ? (int)(w->sg->depth_sum / (double)w->sg->depth_n) : 0;
    const bool admitting = !pending.empty() && wave_can_admit(S, w, cap_slots);
    w->burst = admitting ? std::max(1, depth / 32) : std::max(lpr, depth / 8);
    for (int b = 0; b < kMaxWave; ++b) {
      ServeReq* r = w->slot_req[b];
      if (r && r->cancel && r->state == kRunning) drop |= 1ull << b;
    }
  }
  // seeding (outside the lock; only this wave's thread touches its device state)
  if (!admitted.empty()) {
    const bool fresh = !w->active;
    if (fresh) {
      w->t = 0;
      w->t_cohort = Clock::now();
      for (ServeReq* r : admitted) r->start = 0;
    } else if (w->pending_clear) {
      launch_clear_bits(w->b.visited, w->g.n, w->pending_clear, w->g.num_sms, w->stream);
    }
    w->pending_clear = 0;
    std::map<int32_t, unsigned long long> masks;
    for (ServeReq* r : admitted) {
      w->slots_host->lvl[r->slot] = r->dev_lvl;
      w->slots_host->par[r->slot] = r->dev_par;
      w->slots_host->start[r->slot] = r->start;
      launch_fill(r->dev_lvl, w->g.n, -1, w->g.num_sms, w->stream);
      launch_fill(r->dev_par, w->g.n, -1, w->g.num_sms, w->stream);
      masks[r->root] |= 1ull << r->slot;
    }
    int ns = 0;
    for (auto& kv : masks) w->seeds_host[ns++] = RootSeed{kv.first, kv.second};
    cudaMemcpyAsync(w->b.slots, w->slots_host, sizeof(WaveSlots), cudaMemcpyHostToDevice, w->stream);
    cudaMemcpyAsync(w->b.roots_dev, w->seeds_host, sizeof(RootSeed) * ns, cudaMemcpyHostToDevice, w->stream);
    if (w->g.off64)
      wave_seed<int64_t>(w, ns, fresh);
    else
      wave_seed<int32_t>(w, ns, fresh);
    w->active = true;
  }
  // running-query cancellation: drop the bits at this boundary (no later writes)
  if (drop && w->active) {
    launch_clear_bits(w->b.fmask[w->t.load() % 3], w->g.n, drop, w->g.num_sms, w->stream);
    launch_clear_bits(w->b.visited, w->g.n, drop, w->g.num_sms, w->stream);
    cudaStreamSynchronize(w->stream);
    std::unique_lock<std::mutex> lk(S->mu);
    for (int b = 0; b < kMaxWave; ++b)
      if ((drop >> b) & 1ull) {
        finish_req(S, w->slot_req[b], BFS_ERR_CANCELLED, "cancelled while running");
        w->slot_req[b] = nullptr;
        w->used &= ~(1ull << b);
        --S->running;
      }
  }
  if (!w->active) {
    S->cv_done.notify_all();
    return;
  }
  // a burst of levels
  for (int i = 0; i < w->burst; ++i) {
    if (w->g.off64)
      wave_launch_level<int64_t>(w);
    else
      wave_launch_level<int32_t>(w);
  }
  cudaMemcpyAsync(w->ctl_host, w->b.ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, w->stream);
  cudaError_t e = cudaStreamSynchronize(w->stream);
  std::vector<int> retire;
  if (e == cudaSuccess) {
    const int t_expanded = w->t;  // first frontier of the burst
    w->t = w->ctl_host->level - 1;
    const unsigned long long alive = w->ctl_host->alive[w->t.load() & 1];
    for (int b = 0; b < kMaxWave; ++b) {
      ServeReq* r = w->slot_req[b];
      if (r && r->start <= t_expanded && !((alive >> b) & 1ull)) retire.push_back(b);
    }
    if (!w->ctl_host->cont) {
      w->active = false;
      const double ms = std::chrono::duration<double, std::milli>(Clock::now() - w->t_cohort).count();
      std::lock_guard<std::mutex> lk(S->mu);
      w->sg->wave_ms = w->sg->wave_ms == 0 ? ms : 0.75 * w->sg->wave_ms + 0.25 * ms;
    }
    // statistics and host copies of the retiring slots
    for (int b : retire) {
      ServeReq* r = w->slot_req[b];
      if (w->g.off64)
        launch_level_stats<int64_t>(reinterpret_cast<const int64_t*>(w->g.off), w->g.new_id, w->g.n, r->dev_lvl,
                                    w->stats_dev + 3 * b, w->g.num_sms, w->stream);
      else
        launch_level_stats<int32_t>(reinterpret_cast<const int32_t*>(w->g.off), w->g.new_id, w->g.n, r->dev_lvl,
                                    w->stats_dev + 3 * b, w->g.num_sms, w->stream);
      cudaMemcpyAsync(w->stats_host + 3 * b, w->stats_dev + 3 * b, sizeof(long long) * 3, cudaMemcpyDeviceToHost,
                      w->stream);
      if (r->host_out) {
        cudaMemcpyAsync(r->user_lvl, r->dev_lvl, (size_t)w->g.n * 4, cudaMemcpyDeviceToHost, w->stream);
        cudaMemcpyAsync(r->user_par, r->dev_par, (size_t)w->g.n * 4, cudaMemcpyDeviceToHost, w->stream);
      }
    }
    if (!retire.empty()) e = cudaStreamSynchronize(w->stream);
  }
  std::unique_lock<std::mutex> lk(S->mu);
  S->levels += w->burst;
  if (e != cudaSuccess) {
    const std::string msg = std::string("CUDA error in serving wave: ") + cudaGetErrorString(e);
    cudaGetLastError();
    for (int b = 0; b < kMaxWave; ++b)
      if (w->slot_req[b]) {
        finish_req(S, w->slot_req[b], BFS_ERR_CUDA, msg);
        w->slot_req[b] = nullptr;
        --S->running;
      }
    w->used = 0;
    w->active = false;
    S->fatal = msg;
  } else {
    for (int b : retire) {
      ServeReq* r = w->slot_req[b];
      r->stats.edges_traversed = w->stats_host[3 * b + 0] / 2;
      r->stats.vertices_reached = w->stats_host[3 * b + 1];
      r->stats.depth = (int32_t)w->stats_host[3 * b + 2];
      const Clock::time_point now = Clock::now();
      r->stats.device_ms = std::chrono::duration<double, std::milli>(now - r->t_admit).count();
      r->stats.expand_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
      finish_req(S, r, BFS_OK, "");
      w->sg->depth_sum += r->stats.depth;
      ++w->sg->depth_n;
      w->slot_req[b] = nullptr;
      w->used &= ~(1ull << b);
      w->pending_clear |= 1ull << b;
      --S->running;
    }
    if (w->ctl_host->error & kErrColumnRange) S->fatal = "a column id outside [0, n) was met";
  }
  S->cv_done.notify_all();
}

static void wave_main(bfs_server_s* S, Wave* w) {
  cudaSetDevice(S->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      const int cap_slots = std::max(1, std::min(kMaxWave, S->cfg.max_wave > 0 ? S->cfg.max_wave : kMaxWave));
      auto busy = [&] {
        if (w->active) return true;
        if (w->sg->pending.empty()) return false;
        for (ServeReq* r : w->sg->pending)
          if (r->cancel) return true;
        if (S->stop) return true;
        if (sibling_takes(S, w, cap_slots)) return false;
        Clock::duration left;
        return cohort_ready(S, w, cap_slots, &left);  // else looked at again within 2 ms
      };
      S->cv_work.wait_for(lk, std::chrono::milliseconds(2), [&] { return S->stop || busy(); });
      if (S->stop && !w->active) {  // drain: cancel what has not started, then leave
        for (ServeReq* r : w->sg->pending) finish_req(S, r, BFS_ERR_CANCELLED, "server shutting down");
        w->sg->pending.clear();
        S->cv_done.notify_all();
        break;
      }
      if (!busy()) continue;
    }
    wave_round(S, w);
  }
}

}  // namespace gbfs

using namespace gbfs;

extern "C" {

GBFS_API bfs_status bfs_serve_create(const bfs_serve_config* cfg, bfs_server_t* out) {
  clear_last_error();
  if (!out) return fail(BFS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  auto* S = new (std::nothrow) bfs_server_s();
  if (!S) return fail(BFS_ERR_OOM, "host allocation");
  if (cfg) S->cfg = *cfg;
  if (S->cfg.max_wave < 0 || S->cfg.max_wave > kMaxWave) {
    delete S;
    return fail(BFS_ERR_INVALID_ARG, "max_wave outside [0, 64]");
  }
  if (S->cfg.queue_capacity <= 0) S->cfg.queue_capacity = 1 << 20;
  *out = S;
  return BFS_OK;
}

GBFS_API bfs_status bfs_serve_add_graph(bfs_server_t S, bfs_graph_t G, int* graph_id) {
  clear_last_error();
  if (!S || !G || !graph_id) return fail(BFS_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->started) return fail(BFS_ERR_BUSY, "graphs must be added before the first submission");
  if (S->device >= 0 && G->g.device != S->device) return fail(BFS_ERR_INVALID_ARG, "graphs must share one device");
  cudaError_t e = cudaSetDevice(G->g.device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  const int n_waves = S->cfg.waves_per_graph > 0 ? S->cfg.waves_per_graph : 2;
  const size_t need = batch_bufs_bytes(G->g) * (size_t)n_waves;
  if (S->cfg.memory_cap_bytes && S->mem_fixed + need > S->cfg.memory_cap_bytes)
    return fail(BFS_ERR_OOM, "the graph's wave state exceeds the server's memory budget");
  auto* sg = new (std::nothrow) ServeGraph();
  if (!sg) return fail(BFS_ERR_OOM, "host allocation");
  sg->id = (int)S->graphs.size();
  sg->g = G->g;
  for (int i = 0; i < n_waves; ++i) {
    auto* w = new (std::nothrow) Wave();
    if (!w) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) {
      w->G = G;
      w->sg = sg;
      w->g = G->g;
      e = alloc_batch_bufs(w->g, w->b);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&w->slots_host), sizeof(WaveSlots), 0);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&w->ctl_host), sizeof(BatchCtl), 0);
    if (e == cudaSuccess)
      e = cudaHostAlloc(reinterpret_cast<void**>(&w->seeds_host), sizeof(RootSeed) * kMaxWave, 0);
    if (e == cudaSuccess)
      e = cudaHostAlloc(reinterpret_cast<void**>(&w->stats_host), sizeof(long long) * 3 * kMaxWave, 0);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&w->stats_dev), sizeof(long long) * 3 * kMaxWave);
    if (e != cudaSuccess) {
      free_wave(w);
      for (Wave* x : sg->waves) free_wave(x);
      delete sg;
      return cuda_fail(e, "wave state");
    }
    for (int b = 0; b < kMaxWave; ++b) {
      w->slots_host->lvl[b] = w->slots_host->par[b] = nullptr;
      w->slots_host->start[b] = 0;
    }
    w->shape = G->batch_shape;
    w->grid = w->g.off64 ? batch_expand_grid<int64_t>(w->shape, w->g.num_sms)
                         : batch_expand_grid<int32_t>(w->shape, w->g.num_sms);
    sg->waves.push_back(w);
  }
  S->device = G->g.device;
  S->mem_fixed += need;
  S->mem_peak = std::max(S->mem_peak, S->mem_fixed + S->mem_used);
  for (Wave* w : sg->waves) S->waves.push_back(w);
  S->graphs.push_back(sg);
  *graph_id = sg->id;
  return BFS_OK;
}

GBFS_API bfs_status bfs_serve_submit(bfs_server_t S, int graph_id, int32_t root, int32_t* levels, int32_t* parents,
                                     uint64_t* ticket) {
  clear_last_error();
  if (!S || !levels || !parents || !ticket) return fail(BFS_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(S->mu);
  if (graph_id < 0 || graph_id >= (int)S->graphs.size()) return fail(BFS_ERR_NOT_FOUND, "unknown graph id");
  ServeGraph* sg = S->graphs[graph_id];
  if (root < 0 || root >= sg->g.n) return fail(BFS_ERR_INVALID_ARG, "root outside [0, n)");
  if (S->stop) return fail(BFS_ERR_CANCELLED, "server shutting down");
  size_t queued = 0;
  for (ServeGraph* x : S->graphs) queued += x->pending.size();
  if ((int64_t)queued >= S->cfg.queue_capacity) {
    ++S->rejected;
    return fail(BFS_ERR_BUSY, "request queue is full");
  }
  auto* r = new (std::nothrow) ServeReq();
  if (!r) return fail(BFS_ERR_OOM, "host allocation");
  cudaPointerAttributes at{};
  const bool dev_l = cudaPointerGetAttributes(&at, levels) == cudaSuccess &&
                     (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  const bool dev_p = cudaPointerGetAttributes(&at, parents) == cudaSuccess &&
                     (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  r->ticket = S->next_ticket++;
  r->graph_id = graph_id;
  r->root = root;
  r->user_lvl = levels;
  r->user_par = parents;
  r->host_out = !(dev_l && dev_p);
  r->t_submit = Clock::now();
  if (!S->have_first) {
    S->have_first = true;
    S->first_submit = r->t_submit;
  }
  ++S->submitted;
  S->reqs[r->ticket] = r;
  sg->pending.push_back(r);
  if (!S->started) {
    S->started = true;
    for (Wave* x : S->waves) S->threads.emplace_back(wave_main, S, x);
  }
  *ticket = r->ticket;
  S->cv_work.notify_all();
  return BFS_OK;
}

static bfs_status req_status(bfs_server_s* S, uint64_t ticket, ServeReq** out) {
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return fail(BFS_ERR_NOT_FOUND, "unknown ticket");
  *out = it->second;
  return BFS_OK;
}

GBFS_API bfs_status bfs_serve_poll(bfs_server_t S, uint64_t ticket, int* done) {
  clear_last_error();
  if (!S || !done) return fail(BFS_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(S->mu);
  ServeReq* r;
  bfs_status s = req_status(S, ticket, &r);
  if (s != BFS_OK) return s;
  *done = r->state == kDone;
  return BFS_OK;
}

GBFS_API bfs_status bfs_serve_wait(bfs_server_t S, uint64_t ticket, int timeout_ms) {
  clear_last_error();
  if (!S) return fail(BFS_ERR_INVALID_ARG, "NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  ServeReq* r;
  bfs_status s = req_status(S, ticket, &r);
  if (s != BFS_OK) return s;
  const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
  while (r->state != kDone) {
    if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state != kDone)
      return fail(BFS_ERR_TIMEOUT, "request not complete within the timeout");
  }
  if (r->status != BFS_OK) return fail(r->status, r->message);
  return BFS_OK;
}

GBFS_API bfs_status bfs_serve_cancel(bfs_server_t S, uint64_t ticket) {
  clear_last_error();
  if (!S) return fail(BFS_ERR_INVALID_ARG, "NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  ServeReq* r;
  bfs_status s = req_status(S, ticket, &r);
  if (s != BFS_OK) return s;
  if (r->state != kDone) {
    r->cancel = true;
    S->cv_work.notify_all();
  }
  return BFS_OK;
}

GBFS_API bfs_status bfs_serve_result(bfs_server_t S, uint64_t ticket, bfs_stats* stats) {
  clear_last_error();
  if (!S) return fail(BFS_ERR_INVALID_ARG, "NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  ServeReq* r;
  bfs_status s = req_status(S, ticket, &r);
  if (s != BFS_OK) return s;
  if (r->state != kDone) return fail(BFS_ERR_BUSY, "request not complete");
  if (stats) *stats = r->stats;
  const bfs_status st = r->status;
  const std::string msg = r->message;
  S->reqs.erase(ticket);
  delete r;
  if (st != BFS_OK) return fail(st, msg);
  return BFS_OK;
}

GBFS_API bfs_status bfs_serve_stats(bfs_server_t S, bfs_serve_report* rep) {
  clear_last_error();
  if (!S || !rep) return fail(BFS_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(S->mu);
  bfs_serve_report R{};
  R.submitted = S->submitted;
  R.completed = S->completed;
  R.cancelled = S->cancelled;
  R.rejected = S->rejected;
  R.failed = S->failed;
  R.levels = S->levels;
  R.max_concurrent = S->max_running;
  R.peak_memory_bytes = S->mem_peak;
  std::vector<double> lat = S->latencies_ms;
  std::sort(lat.begin(), lat.end());
  auto pct = [&](double p) {
    if (lat.empty()) return 0.0;
    const size_t i = std::min(lat.size() - 1, (size_t)(p * (double)(lat.size() - 1) + 0.5));
    return lat[i];
  };
  R.latency_p50_ms = pct(0.50);
  R.latency_p99_ms = pct(0.99);
  R.latency_max_ms = lat.empty() ? 0.0 : lat.back();
  double sum = 0;
  for (double x : lat) sum += x;
  R.latency_mean_ms = lat.empty() ? 0.0 : sum / (double)lat.size();
  if (S->have_first && S->completed) {
    R.wall_s = std::chrono::duration<double>(S->last_done - S->first_submit).count();
    R.gteps = R.wall_s > 0 ? (double)S->edges_done / R.wall_s / 1e9 : 0.0;
  }
  R.edges_traversed = S->edges_done;
  *rep = R;
  if (!S->fatal.empty()) return fail(BFS_ERR_CUDA, S->fatal);
  return BFS_OK;
}

GBFS_API bfs_status bfs_serve_destroy(bfs_server_t S) {
  if (!S) return BFS_OK;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_work.notify_all();
  }
  for (auto& th : S->threads)
    if (th.joinable()) th.join();
  if (S->device >= 0) cudaSetDevice(S->device);
  for (Wave* w : S->waves) free_wave(w);
  for (ServeGraph* sg : S->graphs) delete sg;
  for (auto& kv : S->reqs) {
    if (kv.second->charged) {
      cudaFree(kv.second->dev_lvl);
      cudaFree(kv.second->dev_par);
    }
    delete kv.second;
  }
  delete S;
  return BFS_OK;
}

}  // extern "C"
