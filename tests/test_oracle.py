"""Pins for the CPU oracle (CPU only): closed forms, golden hand-worked examples,
brute force on tiny graphs, and planted mistakes that the checkers must catch.

The oracle computes hop distances and a BFS tree (Sec. 2.2 Algorithm 1; Sec. 3.2
Algorithm 2 with R = C = 1) and m_c, the TEPS numerator (Sec. 4)."""
import numpy as np
import pytest

from _graphs import (binary_tree_edges, brute_force_distances, complete_edges, cycle_edges, load_golden,
                     path_edges, random_edges, star_edges)


def _g(graphs_mod, n, src, dst):
    return graphs_mod.from_edges(n, src, dst)


def _run(oracle_mod, g, root):
    lv, pr = oracle_mod.bfs(g.offsets, g.cols, root)
    code, bad = oracle_mod.check_tree(g.offsets, g.cols, root, lv, lv, pr)
    assert code == 0, (oracle_mod.TREE_CODES[code], bad)
    assert oracle_mod.check_edges(g.offsets, g.cols, lv)[0] == 0
    return lv, pr


@pytest.mark.parametrize("n", [1, 2, 7, 100])
def test_path(oracle_mod, graphs_mod, n):
    g = _g(graphs_mod, n, *path_edges(n))
    lv, pr = _run(oracle_mod, g, 0)
    assert np.array_equal(lv, np.arange(n))
    assert np.array_equal(pr, np.maximum(np.arange(n) - 1, 0))  # a path has a unique BFS tree
    mid = n // 2
    lv, _ = _run(oracle_mod, g, mid)
    assert np.array_equal(lv, np.abs(np.arange(n) - mid))


def test_star(oracle_mod, graphs_mod):
    n = 50
    g = _g(graphs_mod, n, *star_edges(n))
    lv, pr = _run(oracle_mod, g, 0)
    assert lv[0] == 0 and np.all(lv[1:] == 1) and np.all(pr[1:] == 0)
    lv, pr = _run(oracle_mod, g, 7)
    expect = np.full(n, 2)
    expect[0], expect[7] = 1, 0
    assert np.array_equal(lv, expect)
    assert pr[0] == 7 and np.all(np.delete(pr, [0, 7]) == 0)


@pytest.mark.parametrize("n", [1, 15, 31, 1000])
def test_complete_binary_tree(oracle_mod, graphs_mod, n):
    g = _g(graphs_mod, n, *binary_tree_edges(n))
    lv, pr = _run(oracle_mod, g, 0)
    i = np.arange(n)
    assert np.array_equal(lv, np.floor(np.log2(i + 1)).astype(np.int32))
    assert np.array_equal(pr[1:], (i[1:] - 1) // 2)


@pytest.mark.parametrize("n", [3, 10, 11])
def test_cycle(oracle_mod, graphs_mod, n):
    g = _g(graphs_mod, n, *cycle_edges(n))
    lv, _ = _run(oracle_mod, g, 0)
    i = np.arange(n)
    assert np.array_equal(lv, np.minimum(i, n - i))


def test_complete_graph(oracle_mod, graphs_mod):
    n = 40
    g = _g(graphs_mod, n, *complete_edges(n))
    lv, pr = _run(oracle_mod, g, 5)
    assert lv[5] == 0 and np.all(np.delete(lv, 5) == 1) and np.all(np.delete(pr, 5) == 5)
    assert oracle_mod.component_edges(g.offsets, lv) == n * (n - 1) // 2


@pytest.mark.parametrize("dims", [(1, 1, 1), (4, 3, 2), (7, 5, 6), (16, 16, 16)])
def test_grid3d_manhattan(oracle_mod, graphs_mod, dims):
    """3D grid: hop distance = Manhattan distance; every vertex is reached and
    m_c = (X-1)YZ + X(Y-1)Z + XY(Z-1)."""
    X, Y, Z = dims
    g = graphs_mod.grid3d(X, Y, Z)
    rng = np.random.default_rng(1)
    ids = np.arange(X * Y * Z)
    x, y, z = ids % X, (ids // X) % Y, ids // (X * Y)
    for root in [0, X * Y * Z - 1, int(rng.integers(0, X * Y * Z))]:
        lv, _ = _run(oracle_mod, g, root)
        rx, ry, rz = root % X, (root // X) % Y, root // (X * Y)
        assert np.array_equal(lv, np.abs(x - rx) + np.abs(y - ry) + np.abs(z - rz))
        assert oracle_mod.component_edges(g.offsets, lv) == (X - 1) * Y * Z + X * (Y - 1) * Z + X * Y * (Z - 1)


def test_disjoint_union(oracle_mod, graphs_mod):
    """Two paths side by side: the other component stays at -1 / -1."""
    s1, d1 = path_edges(10)
    s2, d2 = path_edges(5)
    g = _g(graphs_mod, 15, np.concatenate([s1, s2 + 10]), np.concatenate([d1, d2 + 10]))
    lv, pr = _run(oracle_mod, g, 3)
    assert np.all(lv[10:] == -1) and np.all(pr[10:] == -1)
    assert np.array_equal(lv[:10], np.abs(np.arange(10) - 3))
    assert oracle_mod.component_edges(g.offsets, lv) == 9


def test_isolated_root(oracle_mod, graphs_mod):
    g = _g(graphs_mod, 5, np.array([1], np.int32), np.array([2], np.int32))
    lv, pr = _run(oracle_mod, g, 0)
    assert list(lv) == [0, -1, -1, -1, -1] and list(pr) == [0, -1, -1, -1, -1]
    assert oracle_mod.component_edges(g.offsets, lv) == 0


@pytest.mark.parametrize("name", ["petersen.txt", "two_components.txt"])
def test_golden(oracle_mod, graphs_mod, name):
    fx = load_golden(name)
    g = _g(graphs_mod, fx["n"], fx["src"], fx["dst"])
    lv, _ = _run(oracle_mod, g, fx["root"])
    assert np.array_equal(lv, fx["levels"])
    assert oracle_mod.component_edges(g.offsets, lv) == fx["m_c"]


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_all_pairs(oracle_mod, graphs_mod, seed):
    """Every root of a random tiny multigraph (self-loops and repeats included) against
    fixed-point relaxation on the raw edge list; m_c against a count over the deduplicated
    raw pairs inside the component."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 64))
    m = int(rng.integers(0, 3 * n))
    src, dst = random_edges(n, m, rng)
    g = _g(graphs_mod, n, src, dst)
    dist = brute_force_distances(n, src, dst)
    pairs = {(min(a, b), max(a, b)) for a, b in zip(src.tolist(), dst.tolist()) if a != b}
    for root in range(n):
        lv, _ = _run(oracle_mod, g, root)
        assert np.array_equal(lv, dist[root]), (seed, root)
        reached = lv >= 0
        m_c = sum(1 for a, b in pairs if reached[a])
        assert oracle_mod.component_edges(g.offsets, lv) == m_c


def _planted(oracle_mod, graphs_mod):
    g = graphs_mod.rmat(10, 8, seed=77)
    root = int(graphs_mod.pick_roots(g, 1, 3)[0])
    lv, pr = oracle_mod.bfs(g.offsets, g.cols, root)
    return g, root, lv, pr


def test_checker_catches_wrong_level(oracle_mod, graphs_mod):
    g, root, lv, pr = _planted(oracle_mod, graphs_mod)
    bad = lv.copy()
    v = int(np.flatnonzero(lv == 2)[0])
    bad[v] = 3
    assert oracle_mod.check_tree(g.offsets, g.cols, root, lv, bad, pr)[0] == 1
    assert oracle_mod.check_edges(g.offsets, g.cols, bad)[0] in (0, 6)


def test_checker_catches_root_and_unreached(oracle_mod, graphs_mod):
    g, root, lv, pr = _planted(oracle_mod, graphs_mod)
    bad = pr.copy()
    bad[root] = -1
    assert oracle_mod.check_tree(g.offsets, g.cols, root, lv, lv, bad)[0] == 2
    bad = pr.copy()
    bad[int(np.flatnonzero(lv == 1)[0])] = -1
    assert oracle_mod.check_tree(g.offsets, g.cols, root, lv, lv, bad)[0] == 3


def test_checker_catches_non_edge_parent(oracle_mod, graphs_mod):
    g, root, lv, pr = _planted(oracle_mod, graphs_mod)
    v = int(np.flatnonzero(lv == 2)[0])
    nbrs = set(g.cols[g.offsets[v]:g.offsets[v + 1]].tolist())
    cand = [int(u) for u in np.flatnonzero(lv == 1) if int(u) not in nbrs]
    bad = pr.copy()
    bad[v] = cand[0]
    assert oracle_mod.check_tree(g.offsets, g.cols, root, lv, lv, bad) == (4, v)


def test_checker_catches_same_level_parent(oracle_mod, graphs_mod):
    g, root, lv, pr = _planted(oracle_mod, graphs_mod)
    # an edge between two vertices on the same level
    for v in np.flatnonzero(lv == 2):
        row = g.cols[g.offsets[v]:g.offsets[v + 1]]
        same = row[lv[row] == 2]
        if same.size:
            bad = pr.copy()
            bad[v] = int(same[0])
            assert oracle_mod.check_tree(g.offsets, g.cols, root, lv, lv, bad) == (5, int(v))
            return
    pytest.skip("no same-level edge in this graph")


def test_checker_edges_catches_skipped_level(oracle_mod, graphs_mod):
    g, root, lv, pr = _planted(oracle_mod, graphs_mod)
    bad = lv.copy()
    bad[lv == 2] = 4  # jumps from 1 to 4 across an edge
    assert oracle_mod.check_edges(g.offsets, g.cols, bad)[0] == 6


def test_expand_level_matches_full_search(oracle_mod, graphs_mod):
    """Iterating the one-level expansion from {root} reproduces the search, and the set of
    vertices appended at level L is exactly {v : level[v] = L}."""
    g = graphs_mod.rmat(11, 16, seed=5)
    root = int(graphs_mod.pick_roots(g, 1, 9)[0])
    ref, _ = oracle_mod.bfs(g.offsets, g.cols, root)
    n = g.n
    bitmap = np.zeros((n + 31) // 32, dtype=np.uint32)
    level = np.full(n, -1, dtype=np.int32)
    pred = np.full(n, -1, dtype=np.int32)
    bitmap[root // 32] |= np.uint32(1 << (root % 32))
    level[root], pred[root] = 0, root
    front = np.array([root], dtype=np.int32)
    lvl = 1
    while front.size:
        nxt = oracle_mod.expand_level(g.offsets, g.cols, front, lvl, bitmap, level, pred)
        assert np.array_equal(np.sort(nxt), np.flatnonzero(ref == lvl))
        front, lvl = nxt, lvl + 1
    assert np.array_equal(level, ref)
    assert oracle_mod.check_tree(g.offsets, g.cols, root, ref, level, pred)[0] == 0


def test_expand_level_hand_example(oracle_mod, graphs_mod):
    """Frontier with a zero-degree entry and a repeated vertex; visited targets are skipped."""
    fx = load_golden("two_components.txt")
    g = _g(graphs_mod, fx["n"], fx["src"], fx["dst"])
    n = g.n
    bitmap = np.zeros(1, dtype=np.uint32)
    level = np.full(n, -1, dtype=np.int32)
    pred = np.full(n, -1, dtype=np.int32)
    for v in (0, 1, 2):
        bitmap[0] |= np.uint32(1 << v)
    front = np.array([11, 1, 2, 1], dtype=np.int32)  # 11 has degree 0; 1 appears twice
    nxt = oracle_mod.expand_level(g.offsets, g.cols, front, 2, bitmap, level, pred)
    assert sorted(nxt.tolist()) == [3, 6]
    assert level[3] == 2 and level[6] == 2 and pred[3] == 1 and pred[6] == 2


def test_checker_edges_exact_bounds(oracle_mod, graphs_mod):
    """The edge check's two conditions on their own: a level gap of exactly 2 across an
    edge, and an edge from the root to a vertex marked unreached (gap 1, so only the
    reached-or-neither condition can catch it); valid levels, including an unreached
    component, pass."""
    g = graphs_mod.from_edges(5, np.array([0, 1, 3], np.int32), np.array([1, 2, 4], np.int32))
    ok = np.array([0, 1, 2, -1, -1], np.int32)
    assert oracle_mod.check_edges(g.offsets, g.cols, ok) == (0, -1)
    assert oracle_mod.check_edges(g.offsets, g.cols, np.array([0, 1, 3, -1, -1], np.int32))[0] == 6
    assert oracle_mod.check_edges(g.offsets, g.cols, np.array([0, -1, -1, -1, -1], np.int32)) == (6, 0)
    assert oracle_mod.check_edges(g.offsets, g.cols, np.array([0, 1, 2, 5, -1], np.int32))[0] == 6
