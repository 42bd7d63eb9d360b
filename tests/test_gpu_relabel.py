"""Graphs created with BFS_RELABEL_DEGREE (stored renumbered by degree, every row sorted):
the renumbering is invisible to callers. Every search mode returns the oracle's levels in
the caller's vertex ids, valid parents and the oracle's m_c: the CUDA-graph, host and
persistent loops, bottom-up levels, int32 and int64 offsets, host outputs, batched waves
and the serving loop."""

import numpy as np
import pytest

from _graphs import binary_tree_edges, load_golden, path_edges, random_edges, star_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_1605_gb300 import _build

    _build.build_bfs()
    return torch


@pytest.fixture(scope="module")
def capi_mod(torch_cuda):
    from paper_1408_1605_gb300 import capi

    return capi


def _create(capi, g, force64=False, host_loop=False):
    h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64 | capi.BFS_RELABEL_DEGREE
                              | (capi.BFS_KEEP_INT64 if force64 else 0))
    if host_loop:
        capi.bfs_graph_set_option(h, capi.BFS_OPT_LOOP, capi.BFS_LOOP_HOST)
    return h


def _families(graphs_mod):
    fams = [graphs_mod.from_edges(3000, *path_edges(3000)), graphs_mod.from_edges(2500, *star_edges(2500)),
            graphs_mod.from_edges(4095, *binary_tree_edges(4095)), graphs_mod.grid3d(19, 13, 9),
            graphs_mod.uniform(20000, 70000, seed=8), graphs_mod.rmat(15, 16, seed=graphs_mod.GRAPH_SEED_BASE)]
    fx = load_golden("two_components.txt")
    fams.append(graphs_mod.from_edges(fx["n"], fx["src"], fx["dst"]))
    rng = np.random.default_rng(31)
    for _ in range(3):
        n = int(rng.integers(2, 400))
        fams.append(graphs_mod.from_edges(n, *random_edges(n, int(rng.integers(0, 4 * n)), rng)))
    return fams


def _check(capi, oracle, torch, h, g, root, host_out=False):
    if host_out:
        lv = np.empty(g.n, np.int32)
        pr = np.empty(g.n, np.int32)
        st = capi.bfs_run(h, root, lv, pr, want_stats=True)
    else:
        dl = torch.empty(g.n, dtype=torch.int32, device="cuda")
        dp = torch.empty(g.n, dtype=torch.int32, device="cuda")
        st = capi.bfs_run(h, root, dl, dp, want_stats=True)
        lv, pr = dl.cpu().numpy(), dp.cpu().numpy()
    ref, _ = oracle.bfs(g.offsets, g.cols, root)
    assert np.array_equal(lv, ref), f"root {root}: levels differ at {np.flatnonzero(lv != ref)[:8]}"
    code, bad = oracle.check_tree(g.offsets, g.cols, root, ref, lv, pr)
    assert code == 0, (oracle.TREE_CODES[code], bad)
    assert st.edges_traversed == oracle.component_edges(g.offsets, ref)
    assert st.vertices_reached == int((ref >= 0).sum()) and st.depth == int(ref.max()) + 1
    return st


# (loop, bottom-up, host loop)
MODES = {"graph": (1, 0, False), "host": (2, 0, True), "persistent-td": (0, 0, False), "persistent-do": (0, 1, False)}


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("force64", [False, True])
def test_single_source_modes(torch_cuda, oracle_mod, graphs_mod, capi_mod, mode, force64):
    capi = capi_mod
    loop, bu, host_loop = MODES[mode]
    rng = np.random.default_rng(5)
    for g in _families(graphs_mod):
        h = _create(capi, g, force64, host_loop)
        try:
            assert capi.bfs_graph_get_option(h, capi.BFS_OPT_RELABELED) == 1
            assert capi.bfs_graph_get_option(h, capi.BFS_OPT_PROBE) == 0
            capi.bfs_graph_set_option(h, capi.BFS_OPT_LOOP, loop)
            capi.bfs_graph_set_option(h, capi.BFS_OPT_BOTTOM_UP, bu)
            for root in sorted({0, g.n - 1, int(rng.integers(0, g.n)), int(np.argmax(g.degrees()))}):
                _check(capi, oracle_mod, torch_cuda, h, g, root)
        finally:
            capi.bfs_graph_destroy(h)


def test_rmat_every_shape_and_probe(torch_cuda, oracle_mod, graphs_mod, capi_mod):
    capi = capi_mod
    g = graphs_mod.rmat(16, 16, seed=graphs_mod.GRAPH_SEED_BASE + 3)
    roots = graphs_mod.pick_roots(g, 4, 99)
    h = _create(capi, g)
    try:
        for probe in (0, 1):
            capi.bfs_graph_set_option(h, capi.BFS_OPT_PROBE, probe)
            for shape in range(capi.bfs_shape_count(capi.BFS_KERNEL_SINGLE)):
                capi.bfs_graph_set_shape(h, capi.BFS_KERNEL_SINGLE, shape)
                for r in roots[:2]:
                    _check(capi, oracle_mod, torch_cuda, h, g, int(r))
        _check(capi, oracle_mod, torch_cuda, h, g, int(roots[2]), host_out=True)
    finally:
        capi.bfs_graph_destroy(h)


def test_batched_waves(torch_cuda, oracle_mod, graphs_mod, capi_mod):
    from test_gpu_batch import check_wave

    capi = capi_mod
    for g in (graphs_mod.rmat(14, 16, seed=77), graphs_mod.grid3d(14, 11, 9), graphs_mod.uniform(9000, 30000, seed=2)):
        rng = np.random.default_rng(g.n)
        for force64 in (False, True):
            h = _create(capi, g, force64)
            try:
                roots = rng.integers(0, g.n, size=64)
                roots[5] = roots[9]  # a repeated root
                check_wave(capi, oracle_mod, torch_cuda, h, g, roots)
                check_wave(capi, oracle_mod, torch_cuda, h, g, roots[:7], host_out=True)
            finally:
                capi.bfs_graph_destroy(h)


def test_serving_results_equal_alone(torch_cuda, oracle_mod, graphs_mod, capi_mod):
    from paper_1408_1605_gb300 import serving

    capi = capi_mod
    gs = [graphs_mod.rmat(14, 16, seed=43), graphs_mod.grid3d(16, 12, 10)]
    handles = [_create(capi, g) for g in gs]
    srv = capi.bfs_serve_create()
    try:
        ids = [capi.bfs_serve_add_graph(srv, h) for h in handles]
        alloc = lambda n: (torch_cuda.empty(n, dtype=torch_cuda.int32, device="cuda"),  # noqa: E731
                           torch_cuda.empty(n, dtype=torch_cuda.int32, device="cuda"))
        res = serving.run_poisson(srv, ids, [g.n for g in gs], 60, rate=3000.0, seed=3, alloc=alloc)
        for q in res.queries:
            g = gs[ids.index(q.graph_id)]
            st = capi.bfs_serve_result(srv, q.ticket)
            lv, pr = q.levels.cpu().numpy(), q.parents.cpu().numpy()
            ref, _ = oracle_mod.bfs(g.offsets, g.cols, q.root)
            assert np.array_equal(lv, ref)
            assert oracle_mod.check_tree(g.offsets, g.cols, q.root, ref, lv, pr)[0] == 0
            assert st.edges_traversed == oracle_mod.component_edges(g.offsets, ref)
    finally:
        capi.bfs_serve_destroy(srv)
        for h in handles:
            capi.bfs_graph_destroy(h)


def test_expand_rejected_and_column_range_reported(torch_cuda, graphs_mod, capi_mod):
    capi = capi_mod
    torch = torch_cuda
    g = graphs_mod.from_edges(64, *path_edges(64))
    h = _create(capi, g)
    try:
        n = g.n
        dev = lambda k: torch.zeros(k, dtype=torch.int32, device="cuda")  # noqa: E731
        with pytest.raises(capi.BfsError) as e:
            capi.bfs_expand(h, dev(1), 1, 1, dev((n + 31) // 32), dev(n), dev(n), dev(n),
                            torch.zeros(1, dtype=torch.int64, device="cuda"))
        assert e.value.status == 1
    finally:
        capi.bfs_graph_destroy(h)
    # an out-of-range column id (not validated at creation) survives the renumbering and
    # is reported by the search
    cols = g.cols.copy()
    cols[5] = g.n + 7
    h = capi.bfs_graph_create(g.offsets, cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64 | capi.BFS_RELABEL_DEGREE)
    try:
        lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
        with pytest.raises(capi.BfsError) as e:
            capi.bfs_run(h, 0, lv, lv.clone(), want_stats=True)
        assert e.value.status == 2
    finally:
        capi.bfs_graph_destroy(h)
