"""The 2D-partitioned search of Sec. 3.2 (Algorithm 2: expand and fold exchanges), Sec. 3.4
(Algorithm 3 with destinations owned by other processor columns) and Sec. 3.5 (the update
kernel), emulated on one GPU over R x C virtual processors: levels equal the oracle's for
every root, parents valid (assembled from sender-column predecessors), on processor grids
1x1, 1x2, 2x1, 2x2, 2x4 and 3x2 (the last pads the vertex count to a multiple of R C)."""
import numpy as np
import pytest

from _graphs import binary_tree_edges, load_golden, path_edges, random_edges

pytestmark = pytest.mark.gpu

GRIDS = [(1, 1), (1, 2), (2, 1), (2, 2), (2, 4), (3, 2)]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_1605_gb300 import _build

    _build.build_bfs()
    return torch


def _graphs(graphs_mod):
    fx = load_golden("two_components.txt")
    src, dst = random_edges(300, 900, np.random.default_rng(4))
    return [graphs_mod.rmat(14, 16, seed=61), graphs_mod.grid3d(11, 9, 7),
            graphs_mod.from_edges(1000, *path_edges(1000)), graphs_mod.from_edges(1023, *binary_tree_edges(1023)),
            graphs_mod.from_edges(fx["n"], fx["src"], fx["dst"]), graphs_mod.from_edges(300, src, dst)]


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("force64", [False, True])
def test_2d_partitioned_search(torch_cuda, oracle_mod, graphs_mod, grid, force64):
    from paper_1408_1605_gb300 import capi

    torch = torch_cuda
    R, C = grid
    for g in _graphs(graphs_mod):
        h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz,
                                  capi.BFS_OFFSETS_INT64 | (capi.BFS_KEEP_INT64 if force64 else 0))
        try:
            lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
            pr = torch.empty(g.n, dtype=torch.int32, device="cuda")
            roots = list(graphs_mod.pick_roots(g, 3, 8)) + [g.n - 1]
            for r in roots:
                capi.bfs_run_2d(h, R, C, int(r), lv, pr)
                ref, _ = oracle_mod.bfs(g.offsets, g.cols, int(r))
                got_l, got_p = lv.cpu().numpy(), pr.cpu().numpy()
                assert np.array_equal(got_l, ref), (grid, g.name, r, np.flatnonzero(got_l != ref)[:8])
                code, bad = oracle_mod.check_tree(g.offsets, g.cols, int(r), ref, got_l, got_p)
                assert code == 0, (grid, g.name, r, oracle_mod.TREE_CODES[code], bad)
        finally:
            capi.bfs_graph_destroy(h)


def test_2d_refusals(torch_cuda, graphs_mod):
    from paper_1408_1605_gb300 import capi

    torch = torch_cuda
    g = graphs_mod.rmat(10, 8, seed=2)
    h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64 | capi.BFS_RELABEL_DEGREE)
    lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
    try:
        with pytest.raises(capi.BfsError, match="own numbering"):
            capi.bfs_run_2d(h, 2, 2, 0, lv, lv)
    finally:
        capi.bfs_graph_destroy(h)
    h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64)
    try:
        for R, C in ((0, 2), (2, 65)):
            with pytest.raises(capi.BfsError) as e:
                capi.bfs_run_2d(h, R, C, 0, lv, lv)
            assert e.value.status == 1
        with pytest.raises(capi.BfsError, match="device memory"):
            capi.bfs_run_2d(h, 2, 2, 0, np.zeros(g.n, np.int32), np.zeros(g.n, np.int32))
    finally:
        capi.bfs_graph_destroy(h)
