/*
 * BFS oracle: TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct CPU reference for what the GPU path computes. Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load this file's
 * library; the product path never does. It shares no code with the CUDA library.
 *
 * What it computes (the paper, Sec. 2.2, Algorithm 1, and Sec. 3.2, Algorithm 2, in their
 * one-processor form): starting from root r, level[r] = 0 and pred[r] = r; every other
 * vertex reachable from r gets level = its hop distance from r and pred = a neighbour one
 * level closer to r; unreachable vertices keep level = pred = -1. A level-synchronous
 * search (Algorithm 1's while loop) reaches exactly the hop distances, so the oracle is
 * the textbook sequential FIFO-queue BFS: pop u, and for each neighbour v still unvisited
 * (the bitmap test of Algorithm 1) set its visited flag, pred[v] = u, level[v] =
 * level[u] + 1 and push v.
 *
 * The graph is undirected and stored as a symmetric CSR: offsets int64[n + 1] and
 * neighbour ids int32[offsets[n]] (the paper's CSC `col`/`row` pair, Sec. 3.1; for a
 * symmetric matrix CSC and CSR coincide).
 *
 * Parity status: levels are pinned by closed forms and by an independent brute-force
 * relaxation; parents have no unique value (ties are decided by whichever atomic wins on
 * the GPU, Sec. 3.4) and are checked by the tree invariants in oracle_check_tree; m_c is
 * pinned by a closed form on grids and by brute-force component sums.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Sequential FIFO BFS (Algorithm 1 semantics on one processor). Returns the number of
 * reached vertices (including the root), or -1 on bad arguments. */
int64_t oracle_bfs(int64_t n, const int64_t *offsets, const int32_t *cols, int32_t root,
                   int32_t *level, int32_t *pred) {
    if (n < 1 || !offsets || !level || !pred || root < 0 || root >= n) return -1;
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!queue) return -1;
    for (int64_t v = 0; v < n; ++v) {
        level[v] = -1;
        pred[v] = -1;
    }
    int64_t head = 0, tail = 0;
    level[root] = 0;
    pred[root] = root;
    queue[tail++] = root;
    while (head < tail) {
        const int32_t u = queue[head++];
        for (int64_t e = offsets[u]; e < offsets[u + 1]; ++e) {
            const int32_t v = cols[e];
            if (level[v] == -1) {
                level[v] = level[u] + 1;
                pred[v] = u;
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    return tail;
}

/* Edges counted for TEPS (Sec. 4: input edge tuples within the traversed component).
 * With a cleaned symmetric CSR every undirected edge inside the component appears twice,
 * once from each endpoint, so m_c = (sum of degrees of reached vertices) / 2. */
int64_t oracle_component_edges(int64_t n, const int64_t *offsets, const int32_t *level) {
    int64_t twice = 0;
    for (int64_t v = 0; v < n; ++v)
        if (level[v] >= 0) twice += offsets[v + 1] - offsets[v];
    return twice / 2;
}

/* Is (u, v) an entry of the CSR? Rows are sorted ascending, so binary search. */
static int has_edge(const int64_t *offsets, const int32_t *cols, int32_t u, int32_t v) {
    int64_t lo = offsets[u], hi = offsets[u + 1];
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (cols[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo < offsets[u + 1] && cols[lo] == v;
}

/* Checks a BFS result (level, pred) against the oracle's levels level_ref:
 *   1  level[v] != level_ref[v] for some v (levels must be exact; this also makes the
 *      reached set equal to the oracle's component)
 *   2  level[root] != 0 or pred[root] != root
 *   3  pred[v] == -1 differs from level[v] == -1
 *   4  pred[v] out of range, or (pred[v], v) is not a CSR entry
 *   5  level[pred[v]] != level[v] - 1
 * Returns 0 when valid, else the first failing check's code, with the vertex in *bad. */
int oracle_check_tree(int64_t n, const int64_t *offsets, const int32_t *cols, int32_t root,
                      const int32_t *level_ref, const int32_t *level, const int32_t *pred,
                      int64_t *bad) {
    if (bad) *bad = -1;
    if (root < 0 || root >= n) return 2;
    for (int64_t v = 0; v < n; ++v)
        if (level[v] != level_ref[v]) {
            if (bad) *bad = v;
            return 1;
        }
    if (level[root] != 0 || pred[root] != root) {
        if (bad) *bad = root;
        return 2;
    }
    for (int64_t v = 0; v < n; ++v) {
        if (v == root) continue;
        if ((pred[v] == -1) != (level[v] == -1)) {
            if (bad) *bad = v;
            return 3;
        }
        if (level[v] == -1) continue;
        const int32_t p = pred[v];
        if (p < 0 || p >= n || !has_edge(offsets, cols, p, (int32_t)v)) {
            if (bad) *bad = v;
            return 4;
        }
        if (level[p] != level[v] - 1) {
            if (bad) *bad = v;
            return 5;
        }
    }
    return 0;
}

/* Graph500-style level check over every CSR entry (u, v): both endpoints reached or
 * neither, and |level[u] - level[v]| <= 1. Holds for any valid BFS; returns 0 when valid,
 * else 6 with the offending source vertex in *bad. */
int oracle_check_edges(int64_t n, const int64_t *offsets, const int32_t *cols,
                       const int32_t *level, int64_t *bad) {
    if (bad) *bad = -1;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = offsets[u]; e < offsets[u + 1]; ++e) {
            const int32_t v = cols[e];
            const int32_t a = level[u], b = level[v];
            if ((a < 0) != (b < 0) || (a >= 0 && (a - b > 1 || b - a > 1))) {
                if (bad) *bad = u;
                return 6;
            }
        }
    return 0;
}

/* One top-down level (the expansion step of Algorithm 2, with the R = C = 1
 * identities: every destination is local, so dst_verts has one block). For each u in
 * front[0..n_front) in order and each neighbour v of u: if v's visited bit is clear, set
 * it, pred[v] = u, level[v] = lvl and append v to next. bitmap: uint32[ceil(n/32)], bit
 * v % 32 of word v / 32. Returns the number of appended vertices. */
int64_t oracle_expand_level(int64_t n, const int64_t *offsets, const int32_t *cols,
                            const int32_t *front, int64_t n_front, int32_t lvl,
                            uint32_t *bitmap, int32_t *level, int32_t *pred, int32_t *next) {
    (void)n;
    int64_t count = 0;
    for (int64_t k = 0; k < n_front; ++k) {
        const int32_t u = front[k];
        for (int64_t e = offsets[u]; e < offsets[u + 1]; ++e) {
            const int32_t v = cols[e];
            const uint32_t m = 1u << (v % 32);
            if (bitmap[v / 32] & m) continue;
            bitmap[v / 32] |= m;
            pred[v] = u;
            level[v] = lvl;
            next[count++] = v;
        }
    }
    return count;
}
