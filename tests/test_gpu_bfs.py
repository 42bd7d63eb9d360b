"""Parity of the CUDA single-source search and of the one-level expansion with the CPU
oracle, through the C ABI. Levels must match bit for bit; parents must pass the BFS-tree
invariants (ties between parents are decided by atomics, Sec. 3.4); the edge count m_c
(Sec. 4) must equal the oracle's."""

import numpy as np
import pytest

from _graphs import (binary_tree_edges, complete_edges, cycle_edges, load_golden, path_edges, random_edges,
                     star_edges)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_1605_gb300 import _build

    _build.build_bfs()
    return torch


def _upload(capi, g, force64=False, shape=None, host_loop=False):
    h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz,
                              capi.BFS_OFFSETS_INT64 | (capi.BFS_KEEP_INT64 if force64 else 0))
    if shape is not None:
        capi.bfs_graph_set_shape(h, capi.BFS_KERNEL_SINGLE, shape)
    if host_loop:
        capi.bfs_graph_set_option(h, capi.BFS_OPT_LOOP, capi.BFS_LOOP_HOST)
    return h


def check_root(capi, oracle, torch, h, g, root, host_out=False):
    if host_out:
        lv = np.empty(g.n, dtype=np.int32)
        pr = np.empty(g.n, dtype=np.int32)
        st = capi.bfs_run(h, root, lv, pr, want_stats=True)
    else:
        dl = torch.empty(g.n, dtype=torch.int32, device="cuda")
        dp = torch.empty(g.n, dtype=torch.int32, device="cuda")
        st = capi.bfs_run(h, root, dl, dp, want_stats=True)
        lv, pr = dl.cpu().numpy(), dp.cpu().numpy()
    ref, _ = oracle.bfs(g.offsets, g.cols, root)
    assert np.array_equal(lv, ref), f"levels differ at {np.flatnonzero(lv != ref)[:10]}"
    code, bad = oracle.check_tree(g.offsets, g.cols, root, ref, lv, pr)
    assert code == 0, (oracle.TREE_CODES[code], bad)
    assert st.edges_traversed == oracle.component_edges(g.offsets, ref)
    assert st.vertices_reached == int((ref >= 0).sum())
    assert st.depth == int(ref.max()) + 1
    return st


FAMILIES = {
    "path": lambda: (5000, *path_edges(5000)),
    "star": lambda: (3000, *star_edges(3000)),
    "tree": lambda: (4095, *binary_tree_edges(4095)),
    "cycle": lambda: (1001, *cycle_edges(1001)),
    "complete": lambda: (90, *complete_edges(90)),
}


@pytest.mark.parametrize("family", sorted(FAMILIES))
@pytest.mark.parametrize("force64", [False, True])
def test_closed_form_families(torch_cuda, oracle_mod, graphs_mod, family, force64):
    from paper_1408_1605_gb300 import capi

    n, s, d = FAMILIES[family]()
    g = graphs_mod.from_edges(n, s, d)
    h = _upload(capi, g, force64)
    try:
        for root in (0, n - 1, n // 3):
            check_root(capi, oracle_mod, torch_cuda, h, g, root)
    finally:
        capi.bfs_graph_destroy(h)


@pytest.mark.parametrize("name", ["petersen.txt", "two_components.txt"])
def test_golden(torch_cuda, oracle_mod, graphs_mod, name):
    from paper_1408_1605_gb300 import capi

    fx = load_golden(name)
    g = graphs_mod.from_edges(fx["n"], fx["src"], fx["dst"])
    h = _upload(capi, g)
    try:
        st = check_root(capi, oracle_mod, torch_cuda, h, g, fx["root"])
        assert st.edges_traversed == fx["m_c"]
        for root in range(fx["n"]):  # isolated and small-component roots too
            check_root(capi, oracle_mod, torch_cuda, h, g, root)
    finally:
        capi.bfs_graph_destroy(h)


def test_grid3d_manhattan(torch_cuda, oracle_mod, graphs_mod):
    from paper_1408_1605_gb300 import capi

    X, Y, Z = 37, 23, 19
    g = graphs_mod.grid3d(X, Y, Z)
    h = _upload(capi, g)
    try:
        for root in (0, X * Y * Z - 1, 7 + X * (11 + Y * 5)):
            check_root(capi, oracle_mod, torch_cuda, h, g, root)
    finally:
        capi.bfs_graph_destroy(h)


@pytest.mark.parametrize("shape", list(range(10)))
@pytest.mark.parametrize("force64", [False, True])
def test_rmat16_all_shapes(torch_cuda, oracle_mod, graphs_mod, shape, force64):
    """R-MAT scale 16, edge factor 16 (the small configuration): 16 seeded roots, every
    compiled expansion shape, int32 and int64 offsets."""
    from paper_1408_1605_gb300 import capi

    g = graphs_mod.rmat(16, 16, seed=graphs_mod.GRAPH_SEED_BASE + 0)
    roots = graphs_mod.pick_roots(g, 16, graphs_mod.root_seed(graphs_mod.GRAPH_SEED_BASE + 0))
    h = _upload(capi, g, force64, shape=shape)
    try:
        for r in roots[: 16 if shape == 7 else 4]:
            check_root(capi, oracle_mod, torch_cuda, h, g, int(r))
    finally:
        capi.bfs_graph_destroy(h)


def test_host_loop_and_host_outputs(torch_cuda, oracle_mod, graphs_mod):
    from paper_1408_1605_gb300 import capi

    g = graphs_mod.rmat(14, 16, seed=3)
    roots = graphs_mod.pick_roots(g, 3, 4)
    for host_loop in (False, True):
        h = _upload(capi, g, host_loop=host_loop)
        try:
            for r in roots:
                check_root(capi, oracle_mod, torch_cuda, h, g, int(r), host_out=True)
                check_root(capi, oracle_mod, torch_cuda, h, g, int(r), host_out=False)
        finally:
            capi.bfs_graph_destroy(h)


def test_uniform_and_random_multigraph(torch_cuda, oracle_mod, graphs_mod):
    from paper_1408_1605_gb300 import capi

    g = graphs_mod.uniform(50000, 200000, seed=8)
    h = _upload(capi, g)
    try:
        for r in graphs_mod.pick_roots(g, 4, 1):
            check_root(capi, oracle_mod, torch_cuda, h, g, int(r))
    finally:
        capi.bfs_graph_destroy(h)
    rng = np.random.default_rng(0)
    for _ in range(5):
        n = int(rng.integers(2, 400))
        s, d = random_edges(n, int(rng.integers(0, 4 * n)), rng)
        g = graphs_mod.from_edges(n, s, d)
        h = _upload(capi, g)
        try:
            for root in rng.integers(0, n, 5):
                check_root(capi, oracle_mod, torch_cuda, h, g, int(root))
        finally:
            capi.bfs_graph_destroy(h)


def test_errors(torch_cuda, graphs_mod):
    from paper_1408_1605_gb300 import capi

    g = graphs_mod.rmat(10, 8, seed=1)
    h = _upload(capi, g)
    lv = torch_cuda.empty(g.n, dtype=torch_cuda.int32, device="cuda")
    try:
        for root in (-1, g.n):
            with pytest.raises(capi.BfsError) as e:
                capi.bfs_run(h, root, lv, lv)
            assert e.value.status == 1
    finally:
        capi.bfs_graph_destroy(h)
    # a column id out of range (no BFS_VALIDATE at create): reported by the search
    off = np.array([0, 1, 2], dtype=np.int32)
    cols = np.array([1, 7], dtype=np.int32)
    h = capi.bfs_graph_create(off, cols, 2, 2, 0)
    try:
        with pytest.raises(capi.BfsError) as e:
            capi.bfs_run(h, 0, lv, lv, want_stats=True)
        assert e.value.status == 2
    finally:
        capi.bfs_graph_destroy(h)


def _expand_state(torch, g, visited, level_of):
    n = g.n
    bitmap = np.zeros((n + 31) // 32, dtype=np.uint32)
    for v in visited:
        bitmap[v // 32] |= np.uint32(1 << (v % 32))
    level = np.full(n, -1, dtype=np.int32)
    pred = np.full(n, -1, dtype=np.int32)
    for v in visited:
        level[v] = level_of
    return bitmap, level, pred


@pytest.mark.parametrize("force64", [False, True])
def test_expand_one_level(torch_cuda, oracle_mod, graphs_mod, force64):
    """One level (scan + mapping + claim + append) against the oracle's one-level step, on
    frontiers with repeated vertices, zero-degree vertices, a hub, and ragged sizes."""
    from paper_1408_1605_gb300 import capi

    torch = torch_cuda
    g = graphs_mod.rmat(15, 16, seed=21)
    deg = g.degrees()
    rng = np.random.default_rng(5)
    zero = np.flatnonzero(deg == 0)
    hub = int(np.argmax(deg))
    h = _upload(capi, g, force64)
    try:
        cases = [
            np.array([hub], dtype=np.int32),
            np.array([hub, hub, int(zero[0]), hub], dtype=np.int32),
            rng.choice(g.n, 1, replace=False).astype(np.int32),
            rng.choice(g.n, 777, replace=False).astype(np.int32),
            np.concatenate([zero[:3000], rng.choice(g.n, 3000)]).astype(np.int32),
            rng.choice(g.n, 20000, replace=False).astype(np.int32),
        ]
        for level, front in enumerate(cases, start=1):
            visited = rng.choice(g.n, g.n // 3, replace=False)
            visited = np.union1d(visited, front)
            bm, lv, pr = _expand_state(torch, g, visited, level - 1)
            ref_bm, ref_lv, ref_pr = bm.copy(), lv.copy(), pr.copy()
            ref_next = oracle_mod.expand_level(g.offsets, g.cols, front, level, ref_bm, ref_lv, ref_pr)
            d_front = torch.from_numpy(front).cuda()
            d_bm = torch.from_numpy(bm.view(np.int32)).cuda()
            d_lv = torch.from_numpy(lv).cuda()
            d_pr = torch.from_numpy(pr).cuda()
            d_next = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
            d_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            capi.bfs_expand(h, d_front, front.size, level, d_bm, d_lv, d_pr, d_next, d_cnt)
            cnt = int(d_cnt.item())
            nxt = d_next[:cnt].cpu().numpy()
            assert cnt == ref_next.size
            assert np.array_equal(np.sort(nxt), np.sort(ref_next))
            assert np.array_equal(d_bm.cpu().numpy().view(np.uint32), ref_bm)
            assert np.array_equal(d_lv.cpu().numpy(), ref_lv)
            got_pr = d_pr.cpu().numpy()
            new = ref_next
            assert np.all(np.delete(got_pr, new) == np.delete(ref_pr, new))
            fset = set(front.tolist())
            for v in new[:5000]:
                p = int(got_pr[v])
                assert p in fset and v in g.cols[g.offsets[p]:g.offsets[p + 1]]
        # empty frontier
        d_cnt = torch.full((1,), 5, dtype=torch.int64, device="cuda")
        capi.bfs_expand(h, None, 0, 3, d_bm, d_lv, d_pr, d_next, d_cnt)
        assert int(d_cnt.item()) == 0
        # out-of-range frontier vertex
        with pytest.raises(capi.BfsError):
            bad = torch.tensor([0, g.n + 5], dtype=torch.int32, device="cuda")
            capi.bfs_expand(h, bad, 2, 1, d_bm, d_lv, d_pr, d_next, d_cnt)
    finally:
        capi.bfs_graph_destroy(h)


@pytest.mark.parametrize("force64", [False, True])
@pytest.mark.parametrize("shape", [1, 7])
def test_expand_one_level_to_bitmap(torch_cuda, oracle_mod, graphs_mod, force64, shape):
    """The expansion that hands over its next frontier as a bitmap (Sec. 5) and the
    warp-centric unpack of that bitmap into a list, against the oracle's one-level step, on
    frontiers with repeated vertices, zero-degree vertices, a hub and ragged sizes, for a
    CTA-tile shape and a warp-tile shape: bitmap bit-exact, list = the same set, each
    vertex once, ascending within runs."""
    from paper_1408_1605_gb300 import capi

    torch = torch_cuda
    g = graphs_mod.rmat(15, 16, seed=21)
    deg = g.degrees()
    rng = np.random.default_rng(6)
    zero = np.flatnonzero(deg == 0)
    hub = int(np.argmax(deg))
    h = _upload(capi, g, force64, shape=shape)
    words = (g.n + 31) // 32
    try:
        cases = [
            np.array([hub], dtype=np.int32),
            np.array([hub, hub, int(zero[0]), hub], dtype=np.int32),
            rng.choice(g.n, 1, replace=False).astype(np.int32),
            rng.choice(g.n, 777, replace=False).astype(np.int32),
            np.concatenate([zero[:3000], rng.choice(g.n, 3000)]).astype(np.int32),
            rng.choice(g.n, 20000, replace=False).astype(np.int32),
        ]
        for level, front in enumerate(cases, start=1):
            visited = np.union1d(rng.choice(g.n, g.n // 3, replace=False), front)
            bm, lv, pr = _expand_state(torch, g, visited, level - 1)
            ref_bm, ref_lv, ref_pr = bm.copy(), lv.copy(), pr.copy()
            ref_next = oracle_mod.expand_level(g.offsets, g.cols, front, level, ref_bm, ref_lv, ref_pr)
            want_bits = np.zeros(words, dtype=np.uint32)
            np.bitwise_or.at(want_bits, ref_next // 32, (np.uint32(1) << (ref_next % 32).astype(np.uint32)))
            d_front = torch.from_numpy(front).cuda()
            d_bm = torch.from_numpy(bm.view(np.int32)).cuda()
            d_lv = torch.from_numpy(lv).cuda()
            d_pr = torch.from_numpy(pr).cuda()
            d_nbm = torch.full((words,), -1, dtype=torch.int32, device="cuda")  # cleared by the call
            d_next = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
            d_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            capi.bfs_expand_bitmap(h, d_front, front.size, level, d_bm, d_lv, d_pr, d_nbm, d_next, d_cnt)
            cnt = int(d_cnt.item())
            assert cnt == ref_next.size
            assert np.array_equal(d_nbm.cpu().numpy().view(np.uint32), want_bits)
            nxt = d_next[:cnt].cpu().numpy()
            assert np.array_equal(np.sort(nxt), np.sort(ref_next))  # each vertex once
            runs = np.flatnonzero(np.diff(nxt) < 0)  # ascending within each unpacked run
            assert runs.size <= max(1, words // 64)
            assert np.array_equal(d_bm.cpu().numpy().view(np.uint32), ref_bm)
            assert np.array_equal(d_lv.cpu().numpy(), ref_lv)
            got_pr = d_pr.cpu().numpy()
            assert np.all(np.delete(got_pr, ref_next) == np.delete(ref_pr, ref_next))
            fset = set(front.tolist())
            for v in ref_next[:5000]:
                p = int(got_pr[v])
                assert p in fset and v in g.cols[g.offsets[p]:g.offsets[p + 1]]
            # the bitmap alone (no list)
            capi.bfs_expand_bitmap(h, d_front, front.size, level, d_bm, d_lv, d_pr, d_nbm, None, d_cnt)
            assert int(d_cnt.item()) == 0 and not d_nbm.any()  # everything was claimed by the first call
        # empty frontier
        d_cnt = torch.full((1,), 5, dtype=torch.int64, device="cuda")
        capi.bfs_expand_bitmap(h, None, 0, 3, d_bm, d_lv, d_pr, d_nbm, d_next, d_cnt)
        assert int(d_cnt.item()) == 0 and not d_nbm.any()
    finally:
        capi.bfs_graph_destroy(h)


FRONTIER_MODES = ("list", "auto", "bitmap")


@pytest.mark.parametrize("loop", ["graph", "persistent", "host"])
@pytest.mark.parametrize("mode", FRONTIER_MODES)
def test_frontier_modes_end_to_end(torch_cuda, oracle_mod, graphs_mod, loop, mode):
    """Whole searches with the list-or-bitmap switch off, automatic and forced on, in every
    level loop, on graphs whose large levels cross the switch (R-MAT, input order and
    relabelled; uniform) and graphs whose levels never do (grid, path, binary tree), with
    both offset widths and CTA-tile and warp-tile shapes: levels equal the oracle's, parents
    valid, m_c equal."""
    from paper_1408_1605_gb300 import capi

    loops = {"graph": capi.BFS_LOOP_GRAPH, "persistent": capi.BFS_LOOP_PERSISTENT, "host": capi.BFS_LOOP_HOST}
    modes = {"list": capi.BFS_FRONTIER_LIST, "auto": capi.BFS_FRONTIER_AUTO, "bitmap": capi.BFS_FRONTIER_BITMAP}
    gs = [(graphs_mod.rmat(17, 16, seed=5), 0), (graphs_mod.rmat(17, 16, seed=5), capi.BFS_RELABEL_DEGREE),
          (graphs_mod.uniform(50000, 400000, seed=9), 0), (graphs_mod.grid3d(23, 19, 17), 0),
          (graphs_mod.from_edges(3000, *path_edges(3000)), 0),
          (graphs_mod.from_edges(4095, *binary_tree_edges(4095)), 0)]
    for i, (g, relabel) in enumerate(gs):
        for force64, shape in ((False, 7), (True, 1)):
            h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64 | relabel
                                      | (capi.BFS_KEEP_INT64 if force64 else 0))
            try:
                capi.bfs_graph_set_shape(h, capi.BFS_KERNEL_SINGLE, shape)
                capi.bfs_graph_set_option(h, capi.BFS_OPT_LOOP, loops[loop])
                capi.bfs_graph_set_option(h, capi.BFS_OPT_FRONTIER, modes[mode])
                assert capi.bfs_graph_get_option(h, capi.BFS_OPT_FRONTIER) == modes[mode]
                roots = graphs_mod.pick_roots(g, 2, 40 + i)
                for r in roots:
                    check_root(capi, oracle_mod, torch_cuda, h, g, int(r))
                    if loop == "persistent":
                        unpacked = capi.bfs_graph_get_option(h, capi.BFS_OPT_UNPACKED_LEVELS)
                        assert (unpacked == 0) if mode == "list" else (unpacked >= 0)
                        if mode == "bitmap" and g.n > 10000:
                            assert unpacked >= 1
            finally:
                capi.bfs_graph_destroy(h)


@pytest.mark.parametrize("scale", [20])
def test_rmat_larger(torch_cuda, oracle_mod, graphs_mod, scale):
    from paper_1408_1605_gb300 import capi

    g = graphs_mod.rmat(scale, 16, seed=99)
    h = _upload(capi, g)
    try:
        for r in graphs_mod.pick_roots(g, 3, 7):
            check_root(capi, oracle_mod, torch_cuda, h, g, int(r))
    finally:
        capi.bfs_graph_destroy(h)
