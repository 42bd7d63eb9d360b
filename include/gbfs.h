/*
 * gbfs: single-GPU level-synchronous BFS for GB300 (sm_103a), C ABI.
 *
 * Method: Bisson, Bernaschi, Mastrostefano, "Parallel Distributed Breadth First Search
 * on the Kepler Architecture" (arXiv 1408.1605), in its one-processor form (processor
 * grid R = C = 1, Sec. 3.2 Algorithm 2 with the exchanges reduced to identities): per
 * level, an exclusive scan of the frontier's degrees (Sec. 3.4), a binary search that
 * maps each thread to child edges (Sec. 3.4, Fig. 2; Sec. 3.4.1), a visited-bitmap claim
 * with atomicOr (Sec. 3.4, Algorithm 3), level / predecessor writes, and appends to the
 * next frontier.
 *
 * Conventions shared by every entry point:
 *  - Graphs are undirected and given as a symmetric CSR (the paper's CSC `col` offsets /
 *    `row` indices pair, Sec. 3.1; for a symmetric matrix CSR and CSC coincide):
 *    row_offsets[n_vertices + 1] (int32 or int64, see flags) and cols int32[n_entries]
 *    holding neighbour ids in [0, n_vertices). Rows need not be sorted. Self-loops and
 *    repeated entries are harmless. A non-symmetric CSR is searched along its stored
 *    (out-)edges.
 *  - Outputs (Sec. 3.1; the initialisation of Algorithm 2): level[v] = hop distance from the root,
 *    pred[v] = a neighbour of v one level closer to the root, level[root] = 0 and
 *    pred[root] = root; vertices not reached get level = pred = -1. When several parents
 *    are valid, which one is written depends on which atomic wins (Sec. 3.4).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Work is enqueued on
 *    it; see each call for when it returns.
 *  - Every call returns a bfs_status; on failure bfs_last_error() describes the cause
 *    (thread-local). Outputs are unspecified after a failure.
 *  - The library owns the device copy of a graph and its work buffers; the caller owns
 *    every array it passes in and keeps ownership after the call.
 *  - Calls that use the same graph handle are serialized by a lock in the handle.
 */
#ifndef GBFS_H
#define GBFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GBFS_API __attribute__((visibility("default")))
#else
#define GBFS_API
#endif

typedef enum bfs_status {
  BFS_OK = 0,
  BFS_ERR_INVALID_ARG = 1,   /* NULL pointer, root out of range, bad flags or sizes */
  BFS_ERR_INVALID_GRAPH = 2, /* malformed CSR (see bfs_graph_create) */
  BFS_ERR_OOM = 3,           /* a device or host allocation failed */
  BFS_ERR_CUDA = 4,          /* a CUDA runtime call failed; message in bfs_last_error() */
  BFS_ERR_TIMEOUT = 5,       /* a bounded wait expired */
  BFS_ERR_BUSY = 6,          /* a queue is full; retry later */
  BFS_ERR_CANCELLED = 7,     /* the request was cancelled */
  BFS_ERR_NOT_FOUND = 8      /* unknown ticket / graph id */
} bfs_status;

typedef struct bfs_graph_s *bfs_graph_t;

/* bfs_graph_create flags */
#define BFS_HOST_PTRS 0x1u     /* row_offsets / cols are host pointers (default) */
#define BFS_DEVICE_PTRS 0x2u   /* row_offsets / cols are device pointers */
#define BFS_OFFSETS_INT32 0x4u /* row_offsets is int32[n_vertices + 1] (default) */
#define BFS_OFFSETS_INT64 0x8u /* row_offsets is int64[n_vertices + 1] */
#define BFS_VALIDATE 0x10u     /* also check every column id and the symmetry (O(n_entries)) */
#define BFS_RELABEL_DEGREE 0x20u /* renumber vertices internally by degree (see bfs_graph_create) */
#define BFS_KEEP_INT64 0x40u     /* keep 64-bit row offsets on the device even when n_entries fits
                                    in int32 (see bfs_graph_create) */

/* Per-search statistics. edges_traversed is m_c, the TEPS numerator of Sec. 4: the
 * number of undirected input edges inside the traversed component, i.e. half the degree
 * sum over reached vertices. */
typedef struct bfs_stats {
  int32_t depth;            /* number of non-empty levels, i.e. max level + 1 */
  int32_t bottom_up_levels; /* levels run bottom-up (BFS_OPT_BOTTOM_UP), else 0 */
  int64_t vertices_reached; /* including the root */
  int64_t edges_traversed;  /* m_c */
  double device_ms;         /* device time of the whole search, CUDA events on `stream` */
  double expand_ms;         /* the level loop alone (all expansion launches), CUDA events */
} bfs_stats;

/* Copies a CSR graph into library-owned device memory on the current CUDA device.
 *   row_offsets: int32 or int64 [n_vertices + 1] per BFS_OFFSETS_*; host or device per
 *                BFS_*_PTRS. cols: int32 [n_entries]. n_vertices in [1, 2^31 - 1].
 *   Checked always: row_offsets[0] == 0, non-decreasing, row_offsets[n] == n_entries.
 *   Checked with BFS_VALIDATE: every column id in range and the CSR symmetric.
 *   BFS_RELABEL_DEGREE: the library stores the graph with its vertices renumbered by
 *     non-increasing degree (ties in input order) and every row sorted, so that in skewed
 *     graphs the visited bits of the few vertices that end most edges share a small part of
 *     the bitmap (Algorithm 3's per-edge non-atomic pre-check then hits the L1 cache).
 *     Done once here, on the device (two extra int32[n] maps; peak extra memory about
 *     2 x n_entries x 4 bytes during the call). It is invisible to callers: roots, levels
 *     and parents stay in the caller's numbering, and results are the same BFS (levels
 *     identical; parents valid). bfs_expand is not available on such a graph.
 *   BFS_KEEP_INT64: the device copy keeps 64-bit row offsets, frontier scan values and
 *     tile-descriptor column entries even when n_entries <= 2^31 - 1 (where the library
 *     otherwise narrows them to 32 bits, which moves fewer bytes). Results are the same; the
 *     flag exists so that the wide path, which graphs above 2^31 - 1 entries need, can be
 *     run and checked on small graphs.
 *   Failures: BFS_ERR_INVALID_ARG (NULL / sizes / flags), BFS_ERR_INVALID_GRAPH (checks
 *   above), BFS_ERR_OOM, BFS_ERR_CUDA. The call is synchronous on `stream`. */
GBFS_API bfs_status bfs_graph_create(const void *row_offsets, const int32_t *cols, int64_t n_vertices,
                                     int64_t n_entries, uint32_t flags, void *stream, bfs_graph_t *out);

/* Releases the graph's device memory and work buffers. Waits for the graph's pending
 * work. NULL is accepted (no-op). */
GBFS_API bfs_status bfs_graph_destroy(bfs_graph_t g);

/* Per-graph options of single-source searches (bfs_run):
 *   BFS_OPT_LOOP: how the level loop runs. BFS_LOOP_GRAPH (default): a CUDA graph with a
 *     conditional WHILE node, one expansion launch per level. BFS_LOOP_PERSISTENT: one
 *     cooperative launch runs every level, separated by a grid barrier whose waits are
 *     bounded (expiry: BFS_ERR_TIMEOUT). BFS_LOOP_HOST: one launch per level and a host
 *     check of the next frontier (for profilers that cannot see graph kernel nodes); with it
 *     bfs_run_batch also drives its waves' levels from the host.
 *   BFS_OPT_BOTTOM_UP: 1 lets a persistent search run large levels bottom-up (every
 *     unvisited vertex looks for a parent in the frontier; Beamer et al., the paper's
 *     related work, Sec. 6) when frontier edges x ALPHA exceed the unexplored edges, and
 *     return to top-down once frontier vertices x BETA < n. Results are the same BFS
 *     (levels identical; parents valid). Default 0: every level top-down (Algorithm 3).
 *     The option also applies to bfs_run_batch: a wave then runs large levels bottom-up
 *     (every vertex pulls the root bits it misses from its neighbours' frontier masks),
 *     switching by the same rule on the wave's union frontier; per_root_stats report the
 *     wave's bottom-up levels. Serving waves stay top-down.
 *   BFS_OPT_ALPHA (default 8; swept on GB300: 8 beat 2, 4, 6, 14 on R-MAT and uniform graphs),
 *   BFS_OPT_BETA (default 24): the switching thresholds.
 *   BFS_OPT_WAIT_LIMIT: polls a CTA makes at a grid barrier of a persistent search before it
 *     gives up (default 2^27, seconds). On expiry the search stops and bfs_run returns
 *     BFS_ERR_TIMEOUT; the device stays usable. 0 makes every wait give up at once (used to
 *     test that path without hanging anything).
 *   BFS_OPT_PROBE: how the visited-bit pre-check of each edge is loaded: 0 through L1
 *     (default for BFS_RELABEL_DEGREE graphs; a stale L1 copy only costs a futile atomic),
 *     1 from L2 only (default otherwise; sees the level's claims sooner).
 *   BFS_OPT_RELABELED (read only): 1 if the graph was created with BFS_RELABEL_DEGREE.
 *   BFS_OPT_PERSIST_CTAS: CTAs per SM of a persistent search (0, the default: as many as
 *     fit). Fewer CTAs make each level boundary cheaper, which pays on graphs of hundreds
 *     of small levels (3D grids); large levels want them all.
 *   BFS_OPT_FRONTIER: how a top-down level hands its next frontier to the next level
 *     (Sec. 5, the switch between a vertex list and a bitmap of the vertices by size).
 *     BFS_FRONTIER_LIST (default): a list of vertex ids with its degree scan, built by the
 *     appends of the expansion. BFS_FRONTIER_AUTO: the same while the list holds at most
 *     ceil(n / 32) entries, i.e. while its 32-bit ids take fewer bits than an n-bit bitmap;
 *     past that the level records its claims only in a bitmap of the next frontier, and the
 *     list is rebuilt from the bitmap after the level (in vertex order, by a warp-centric
 *     unpack that writes ids, scan and tile descriptors). BFS_FRONTIER_BITMAP: every
 *     top-down level hands over a bitmap. Results are the same BFS in every mode.
 *   BFS_OPT_UNPACKED_LEVELS (read only): levels of the last persistent search whose next
 *     frontier was rebuilt from a bitmap (-1 after a search in another loop mode).
 *   BFS_OPT_WAVE_DENSE_ROWS: a batched wave writes a claim of one root bit out at once and
 *     records a claim of several bits (root bits, parent, level) in one of 8 slots of the
 *     claimed vertex; a vertex claimed more often gets a dense row of 64 parents and levels
 *     (512 bytes) from a pool. This option sizes the pool (-1, the default: a row per vertex
 *     when those 520 bytes per vertex take at most a quarter of the free device memory when
 *     the wave buffers are allocated, else n / 16 + 1024 rows; 0: none; at most n) and frees
 *     the graph's wave buffers, which the next wave allocates again. Claims left without
 *     room go to an overflow list of n / 4 + 65536 records, and past it are written out at
 *     once.
 *   BFS_OPT_WAVE_LEVELS, BFS_OPT_WAVE_OVERFLOW (read only): levels run by the last batched
 *     wave on this graph, and how many of its claim records did not fit the per-vertex
 *     slots (they are applied from an overflow list when the wave's outputs are written). */
#define BFS_OPT_LOOP 1
#define BFS_OPT_BOTTOM_UP 2
#define BFS_OPT_ALPHA 3
#define BFS_OPT_BETA 4
#define BFS_OPT_WAIT_LIMIT 5
#define BFS_OPT_PROBE 6
#define BFS_OPT_RELABELED 7
#define BFS_OPT_PERSIST_CTAS 8
#define BFS_OPT_WAVE_LEVELS 9
#define BFS_OPT_WAVE_OVERFLOW 10
#define BFS_OPT_FRONTIER 11
#define BFS_OPT_UNPACKED_LEVELS 12
#define BFS_OPT_WAVE_DENSE_ROWS 13
#define BFS_FRONTIER_LIST 0
#define BFS_FRONTIER_AUTO 1
#define BFS_FRONTIER_BITMAP 2
#define BFS_LOOP_PERSISTENT 0
#define BFS_LOOP_GRAPH 1
#define BFS_LOOP_HOST 2
GBFS_API bfs_status bfs_graph_set_option(bfs_graph_t g, int option, int64_t value);
GBFS_API bfs_status bfs_graph_get_option(bfs_graph_t g, int option, int64_t *value);

/* Per-level profile of the last persistent search on this graph (BFS_LOOP_PERSISTENT):
 * device time of each level (ms, from the device clock at each grid barrier), the size of
 * the frontier it expanded, and whether it ran bottom-up. Writes min(levels, cap) entries
 * (at most 64) of each non-NULL array; *n_levels = levels recorded. Waits for the graph's
 * pending work. BFS_ERR_NOT_FOUND if no persistent search has run. */
GBFS_API bfs_status bfs_level_profile(bfs_graph_t g, int cap, double *level_ms, int64_t *frontier,
                                      int32_t *bottom_up, int *n_levels);

/* Vertex and CSR-entry counts of a graph. */
GBFS_API bfs_status bfs_graph_info(bfs_graph_t g, int64_t *n_vertices, int64_t *n_entries);

/* One single-source BFS from `root` (Algorithm 2 with R = C = 1; kernel per level as in
 * Algorithm 3). levels / parents: int32[n_vertices] each, device memory or host memory
 * (pinned or pageable; detected with cudaPointerGetAttributes, results are then copied
 * back before return). The level loop runs on the device; the call returns once the
 * search has finished when stats != NULL or the outputs are host memory, else as soon as
 * the work is enqueued. Failures: BFS_ERR_INVALID_ARG (root outside [0, n), NULL
 * outputs), BFS_ERR_INVALID_GRAPH (a column id out of range was met during the search),
 * BFS_ERR_OOM, BFS_ERR_CUDA. */
GBFS_API bfs_status bfs_run(bfs_graph_t g, int32_t root, int32_t *levels, int32_t *parents, void *stream,
                            bfs_stats *stats);

/* Multi-source search: up to 64 roots run as one wave, one bit per root in a 64-bit
 * visited mask and 64-bit frontier masks per vertex, so that every row read from the CSR
 * serves all the roots that have the vertex in their frontier. Each root's result is the
 * single-source result (levels identical; parents any valid BFS tree). The paper has no
 * batched form; each root's search is Algorithm 2 / Algorithm 3 with R = C = 1.
 *   roots: HOST int32[n_roots], 1 <= n_roots <= 64, each in [0, n) (repeats allowed).
 *   levels, parents: int32[n_roots][n_vertices] (row b belongs to roots[b]), device memory
 *     or host memory (detected; results copied back before return).
 *   per_root_stats: NULL or bfs_stats[n_roots]; device_ms / expand_ms are the wave's time.
 * The call returns once the work is enqueued unless stats are requested or the outputs
 * are host memory. Failures: BFS_ERR_INVALID_ARG, BFS_ERR_INVALID_GRAPH, BFS_ERR_OOM,
 * BFS_ERR_CUDA. */
GBFS_API bfs_status bfs_run_batch(bfs_graph_t g, const int32_t *roots, int n_roots, int32_t *levels,
                                  int32_t *parents, void *stream, bfs_stats *per_root_stats);

/* One top-down level on caller-held state: the frontier expansion step of Algorithm 2
 * (Algorithm 3) with R = C = 1, including the degree gather and exclusive scan
 * (Sec. 3.4). All pointers are device memory:
 *   frontier int32[n_frontier]: the current frontier (any order, repeats and
 *     zero-degree vertices allowed);
 *   bitmap uint32[ceil(n/32)]: visited bits, bit v % 32 of word v / 32 (Sec. 3.1);
 *   levels, parents int32[n]: written for each newly claimed vertex v as
 *     levels[v] = level, parents[v] = the frontier vertex whose edge claimed v;
 *   next int32[n]: receives the newly claimed vertices, each once, in unspecified order;
 *   next_count int64 (device): receives their number.
 * `level` must be >= 1. The call synchronizes `stream` and returns after the level has
 * completed, so that range errors can be reported. Failures: BFS_ERR_INVALID_ARG (a
 * frontier vertex outside [0, n), a frontier whose edge total exceeds the graph's entry
 * count, or a graph created with BFS_RELABEL_DEGREE), BFS_ERR_INVALID_GRAPH (a column id
 * out of range), BFS_ERR_OOM, BFS_ERR_CUDA. */
GBFS_API bfs_status bfs_expand(bfs_graph_t g, const int32_t *frontier, int64_t n_frontier, int32_t level,
                               uint32_t *bitmap, int32_t *levels, int32_t *parents, int32_t *next,
                               int64_t *next_count, void *stream);

/* The paper's 2D-partitioned search (Sec. 3.2 Algorithm 2, Sec. 3.4 Algorithm 3 with
 * destinations owned by other processor columns, Sec. 3.5 frontier update), emulated on this
 * GPU: the graph is split over an R x C grid of virtual processors (vertex block j R + i
 * owned by P_ij; edge (u, v) held by the processor of u's column block j and v's row block
 * mod R), each with its own local CSC, level and predecessor arrays and visited bitmap, and
 * the expand (within a grid column) and fold (within a grid row) exchanges are copies between
 * their device buffers. Results are the same BFS as bfs_run's (levels identical; parents a
 * valid tree, assembled from the sender-column predecessors of the update kernel).
 *   R, C in [1, 64]; levels, parents: device int32[n_vertices].
 * The partition is built for the call and freed after it; the call synchronizes `stream`.
 * Not available on graphs created with BFS_RELABEL_DEGREE. Failures: BFS_ERR_INVALID_ARG,
 * BFS_ERR_INVALID_GRAPH (a column id out of range), BFS_ERR_OOM, BFS_ERR_CUDA. */
GBFS_API bfs_status bfs_run_2d(bfs_graph_t g, int R, int C, int32_t root, int32_t *levels, int32_t *parents,
                               void *stream);

/* One top-down level on caller-held state, as bfs_expand, that hands over its next frontier
 * as a bitmap (Sec. 5: the specialized expansion that produces a bitmap instead of a list):
 *   next_bitmap uint32[ceil(n/32)] (device): cleared by the call, then bit v % 32 of word
 *     v / 32 set for every vertex v the level claims;
 *   next int32[n] (device) or NULL: if given, the claimed vertices unpacked from next_bitmap
 *     by the warp-centric unpack (each once; in increasing order within each run of
 *     consecutive bitmap words a CTA unpacks, runs in unspecified order);
 *   next_count int64 (device): the number of claimed vertices.
 * Other arguments, the synchronization and the failures as for bfs_expand. */
GBFS_API bfs_status bfs_expand_bitmap(bfs_graph_t g, const int32_t *frontier, int64_t n_frontier, int32_t level,
                                      uint32_t *bitmap, int32_t *levels, int32_t *parents, uint32_t *next_bitmap,
                                      int32_t *next, int64_t *next_count, void *stream);

/* Single-source BFS that allocates nothing, for callers that may not allocate device
 * memory at call time: code whose framework allocator owns all device memory, loops in
 * which cudaMalloc / cudaFree would synchronize the device, services that must not fail
 * with out-of-memory mid-request. The paper has no counterpart; the search is the same
 * as bfs_run's, with every work buffer in one static device array (about 7.4 MB, held by
 * every GPU that loads the library until the process exits).
 *   row_offsets int32[n_vertices + 1], cols int32[n_entries]: device memory, a symmetric
 *     CSR as for bfs_graph_create (the offsets are checked on the device; column ids are
 *     range-checked during the search).
 *   levels, parents int32[n_vertices]: device memory, written as by bfs_run.
 * Limits: 1 <= n_vertices <= 262144 and 0 <= n_entries <= 4194304; larger sizes are
 * rejected with BFS_ERR_INVALID_ARG before any GPU work. The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device current; make
 * that first call before any stream capture. Every call on a device shares the array and
 * re-initializes what must start cleared; two searches using it at the same time on the
 * GPU would race, so the call holds a process-wide lock and returns only after its search
 * has finished on `stream`. Failures: BFS_ERR_INVALID_ARG, BFS_ERR_INVALID_GRAPH,
 * BFS_ERR_CUDA. */
GBFS_API bfs_status bfs_run_noalloc(const int32_t *row_offsets, const int32_t *cols, int64_t n_vertices,
                                    int64_t n_entries, int32_t root, int32_t *levels, int32_t *parents,
                                    void *stream);

/* ---------------------------------------------------------------------------------------
 * Serving: BFS queries on resident graphs with continuous batching. The paper has no
 * serving layer; every query runs as one bit-slot of a multi-source wave (see
 * bfs_run_batch) on its graph, and its result is identical to the same query run alone
 * (levels equal; parents a valid BFS tree).
 *   - Each added graph gets waves_per_graph waves of up to max_wave slots; each wave has its
 *     own CUDA stream and scheduler thread, so waves run concurrently on the device.
 *   - A wave advances in bursts of levels (levels_per_round when it cannot admit, else
 *     one; on deep graphs an eighth, resp. a thirty-second, of the graph's mean query depth
 *     if that is more). Between two bursts, finished queries retire (their bit left every frontier)
 *     and pending queries of its graph are admitted into free slots in arrival order,
 *     starting from their root at the current wave level; a wave is never restarted for
 *     admission. Queries share row reads only while their searches are in step, so a
 *     running wave admits only while its cohort is young (admit_window); otherwise an idle
 *     wave of the graph starts a new cohort.
 *   - A wave's cost depends little on how many of its slots are busy (on skewed graphs every
 *     root's large level covers most of the graph), so an idle wave does not start a cohort
 *     for a single query while a sibling wave of the graph is running: it waits until the
 *     pending queries fill a wave or the oldest has waited cohort_wait_us.
 *   - Admission is gated by memory_cap_bytes: the graphs' wave state plus, for each
 *     running query whose outputs are host memory, a device staging buffer of 8 bytes
 *     per vertex. A query waits in the queue until a slot and the memory are free.
 * --------------------------------------------------------------------------------------- */
typedef struct bfs_server_s *bfs_server_t;

typedef struct bfs_serve_config {
  uint64_t memory_cap_bytes; /* device memory budget (0 = unlimited) */
  int32_t max_wave;          /* slots per graph wave, 1..64 (0 = 64) */
  int32_t queue_capacity;    /* pending queries before submit returns BFS_ERR_BUSY (0 = 2^20) */
  int32_t levels_per_round;  /* levels a wave that cannot admit runs between two
                                admission/retirement checks (0 = 8); 1 checks every level */
  int32_t waves_per_graph;   /* waves (64-slot cohorts) per resident graph (0 = 2) */
  int32_t admit_window;      /* a running wave admits only while its cohort is at most this
                                many levels old (0 = 3); raised to a quarter of the graph's
                                mean query depth on deep graphs */
  int32_t cohort_wait_us;    /* while another wave of the graph is running, an idle wave starts
                                a new cohort only once max_wave queries are pending or the
                                oldest has waited this long (0: the moving average of the
                                graph's cohort durations; < 0: start at once) */
} bfs_serve_config;

typedef struct bfs_serve_report {
  uint64_t submitted, completed, cancelled, rejected, failed;
  uint64_t levels;             /* wave levels run, all graphs */
  int64_t edges_traversed;     /* sum of m_c over completed queries */
  double latency_p50_ms, latency_p99_ms, latency_mean_ms, latency_max_ms; /* submit -> done */
  double wall_s;               /* first submission -> last completion */
  double gteps;                /* edges_traversed / wall_s / 1e9 */
  int32_t max_concurrent;      /* most queries running at once */
  int32_t reserved;
  uint64_t peak_memory_bytes;  /* wave state + staging, at most memory_cap_bytes */
} bfs_serve_report;

/* Creates a server (no graphs yet). cfg may be NULL for defaults. Failures:
 * BFS_ERR_INVALID_ARG (max_wave outside [0, 64]), BFS_ERR_OOM. */
GBFS_API bfs_status bfs_serve_create(const bfs_serve_config *cfg, bfs_server_t *out);

/* Makes a graph resident in the server and allocates its waves' state (about 128 bytes
 * per vertex per wave). The graph handle must outlive the server. Graphs are added before the first
 * submission, all on one device. Failures: BFS_ERR_INVALID_ARG, BFS_ERR_BUSY (already
 * serving), BFS_ERR_OOM (memory budget or device memory), BFS_ERR_CUDA. */
GBFS_API bfs_status bfs_serve_add_graph(bfs_server_t srv, bfs_graph_t g, int *graph_id);

/* Queues one query: BFS from `root` on graph `graph_id`. levels / parents:
 * int32[n_vertices] each, caller-owned, device or host memory (detected), written when the
 * query completes and not touched after bfs_serve_wait / bfs_serve_poll report it done.
 * Non-blocking. Failures: BFS_ERR_INVALID_ARG, BFS_ERR_NOT_FOUND (graph id),
 * BFS_ERR_BUSY (queue full: retry later), BFS_ERR_CANCELLED (server shutting down). */
GBFS_API bfs_status bfs_serve_submit(bfs_server_t srv, int graph_id, int32_t root, int32_t *levels,
                                     int32_t *parents, uint64_t *ticket);

/* *done = 1 once the query has completed, failed or been cancelled. */
GBFS_API bfs_status bfs_serve_poll(bfs_server_t srv, uint64_t ticket, int *done);

/* Blocks until the query is done or timeout_ms passes (BFS_ERR_TIMEOUT). Returns the
 * query's own status once done (BFS_OK, BFS_ERR_CANCELLED, BFS_ERR_CUDA ...). */
GBFS_API bfs_status bfs_serve_wait(bfs_server_t srv, uint64_t ticket, int timeout_ms);

/* Requests cancellation: a pending query is dropped; a running one stops at the next level
 * boundary (no output writes after it is reported done). */
GBFS_API bfs_status bfs_serve_cancel(bfs_server_t srv, uint64_t ticket);

/* Statistics of a completed query (depth, vertices reached, m_c; device_ms = time from
 * admission to completion, expand_ms = time from submission to completion, i.e. the query's
 * latency) and release of its ticket. Returns the query's status; BFS_ERR_BUSY if it is not
 * done yet. */
GBFS_API bfs_status bfs_serve_result(bfs_server_t srv, uint64_t ticket, bfs_stats *stats);

/* Latency percentiles, throughput and counters since creation. */
GBFS_API bfs_status bfs_serve_stats(bfs_server_t srv, bfs_serve_report *report);

/* Stops the scheduler (pending queries are cancelled, running ones finish) and frees the
 * server's device memory. NULL is accepted. */
GBFS_API bfs_status bfs_serve_destroy(bfs_server_t srv);

/* ---------------------------------------------------------------------------------------
 * Kernel shapes and tuning. Each expansion kernel is compiled for a few shapes (threads per
 * CTA, edges per thread, claim-buffer entries, CTA or warp tiles, register budget); the
 * paper picks its edges-per-thread value by a sweep (Sec. 3.4.1, Fig. 3), and bfs_tune does
 * the same sweep per graph, together with the level-loop mode.
 * --------------------------------------------------------------------------------------- */
#define BFS_KERNEL_SINGLE 0 /* single-source expansion (bfs_run, bfs_expand) */
#define BFS_KERNEL_BATCH 1  /* multi-source expansion (bfs_run_batch, serving waves) */

/* Number of compiled shapes of a kernel kind (0 for an unknown kind). */
GBFS_API int bfs_shape_count(int kind);

/* Shape parameters: CTA size, edges per thread, claim-buffer entries, and the tiling:
 * *warp_tiles = 0 when a CTA expands tiles of block x edges_per_thread edges (claim buffer
 * per CTA), 1 when every warp expands its own tiles of 32 x edges_per_thread edges (claim
 * buffer per warp; no CTA-wide barrier inside a level). Any output pointer may be NULL. */
GBFS_API bfs_status bfs_shape_info(int kind, int shape, int *block, int *edges_per_thread, int *claim_buffer,
                                   int *warp_tiles);

/* Selects the shape a graph's later searches use (waits for the graph's pending work). A
 * server takes a graph's batch shape when the graph is added. */
GBFS_API bfs_status bfs_graph_set_shape(bfs_graph_t g, int kind, int shape);
GBFS_API bfs_status bfs_graph_get_shape(bfs_graph_t g, int kind, int *shape);

/* Times the candidates of `kind` on this graph and keeps the fastest.
 *   BFS_KERNEL_SINGLE: candidates c = loop x shape: c < count uses BFS_LOOP_GRAPH with shape
 *     c, count <= c < 2 count BFS_LOOP_PERSISTENT with shape c - count and as many CTAs as
 *     fit, 2 count <= c < 3 count BFS_LOOP_PERSISTENT with shape c - 2 count and 2 CTAs per
 *     SM, 3 count <= c < 4 count the same with 1 CTA per SM (BFS_OPT_PERSIST_CTAS; with
 *     BFS_OPT_BOTTOM_UP set, only the persistent ones; the others report -1). One warm-up
 *     search, then one bfs_run per root; ms_per_shape[c] = mean device ms per root. The
 *     winner's loop mode, CTAs per SM and shape are set on the graph. ms_per_shape: NULL or
 *     double[4 * count].
 *   BFS_KERNEL_BATCH: candidates = shapes; n_roots <= 64; one warm-up wave and one timed
 *     wave per shape; ms_per_shape[s] = device ms per wave (double[count]).
 * count = bfs_shape_count(kind); best_shape: NULL or the winning candidate index.
 * Other calls on the graph must not run meanwhile. Failures as for bfs_run /
 * bfs_run_batch. */
GBFS_API bfs_status bfs_tune(bfs_graph_t g, int kind, const int32_t *roots, int n_roots, int32_t *levels,
                             int32_t *parents, void *stream, double *ms_per_shape, int *best_shape);

/* Message for the last failing call on this thread ("" if none). */
GBFS_API const char *bfs_last_error(void);

/* Library version string. */
GBFS_API const char *bfs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GBFS_H */
