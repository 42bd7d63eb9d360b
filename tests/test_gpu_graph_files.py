"""Graphs read from files (the paper's Table 3 inputs come as edge-list files, Sec. 5):
a SNAP-style text edge list and a MatrixMarket coordinate file are written here, loaded
through graphs.load_edge_list, searched through the C ABI with bfs_run and bfs_run_batch,
and compared with the oracle: levels bit-exact for every root, parents valid, m_c equal."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_1605_gb300 import _build

    _build.build_bfs()
    return torch


def _check_graph(capi, oracle, torch, g, roots, flags):
    h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64 | flags)
    try:
        lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
        pr = torch.empty(g.n, dtype=torch.int32, device="cuda")
        refs = []
        for r in roots:
            st = capi.bfs_run(h, int(r), lv, pr, want_stats=True)
            ref, _ = oracle.bfs(g.offsets, g.cols, int(r))
            refs.append(ref)
            got_l, got_p = lv.cpu().numpy(), pr.cpu().numpy()
            assert np.array_equal(got_l, ref)
            code, bad = oracle.check_tree(g.offsets, g.cols, int(r), ref, got_l, got_p)
            assert code == 0, (oracle.TREE_CODES[code], bad)
            assert st.edges_traversed == oracle.component_edges(g.offsets, ref)
        bl = torch.empty((len(roots), g.n), dtype=torch.int32, device="cuda")
        bp = torch.empty((len(roots), g.n), dtype=torch.int32, device="cuda")
        bst = capi.bfs_run_batch(h, roots, bl, bp, want_stats=True)
        L, P = bl.cpu().numpy(), bp.cpu().numpy()
        for b, (r, ref) in enumerate(zip(roots, refs)):
            assert np.array_equal(L[b], ref)
            code, bad = oracle.check_tree(g.offsets, g.cols, int(r), ref, L[b], P[b])
            assert code == 0, (oracle.TREE_CODES[code], bad)
            assert bst[b].edges_traversed == oracle.component_edges(g.offsets, ref)
    finally:
        capi.bfs_graph_destroy(h)


@pytest.mark.parametrize("relabel", [False, True])
def test_text_edge_list_file(torch_cuda, oracle_mod, graphs_mod, tmp_path, relabel):
    from paper_1408_1605_gb300 import capi

    src, dst = graphs_mod.rmat_edges(13, 8, seed=graphs_mod.GRAPH_SEED_BASE + 77)
    rng = np.random.default_rng(5)
    lines = ["# Directed graph (each unordered pair of nodes is saved once)", "# FromNodeId\tToNodeId"]
    for u, v in zip(src.tolist(), dst.tolist()):
        lines.append(f"{u}\t{v}" if rng.integers(0, 3) else f"{u} {v}")
    path = tmp_path / "rmat13.txt"
    path.write_text("\n".join(lines) + "\n")
    g = graphs_mod.load_edge_list(str(path))
    want = graphs_mod.from_edges(int(max(src.max(), dst.max())) + 1, src, dst)
    assert np.array_equal(g.offsets, want.offsets) and np.array_equal(g.cols, want.cols)
    roots = graphs_mod.pick_roots(g, 40, 99)
    _check_graph(capi, oracle_mod, torch_cuda, g, roots,
                 capi.BFS_RELABEL_DEGREE if relabel else 0)


def test_matrix_market_file_compacted(torch_cuda, oracle_mod, graphs_mod, tmp_path):
    from paper_1408_1605_gb300 import capi

    # a 3D grid with a hole of unused ids, as a symmetric pattern matrix (each pair once)
    src, dst = graphs_mod.grid3d_edges(21, 17, 11)
    src = np.where(src >= 1000, src + 500, src)
    dst = np.where(dst >= 1000, dst + 500, dst)
    n = 21 * 17 * 11 + 500
    body = "\n".join(f"{max(u, v) + 1} {min(u, v) + 1}" for u, v in zip(src.tolist(), dst.tolist()))
    path = tmp_path / "grid.mtx"
    path.write_text(f"%%MatrixMarket matrix coordinate pattern symmetric\n% grid with a gap\n{n} {n} {src.size}\n"
                    f"{body}\n")
    g = graphs_mod.load_edge_list(str(path), compact=True)
    assert g.n == 21 * 17 * 11 and g.ids.size == g.n
    roots = graphs_mod.pick_roots(g, 24, 7)
    _check_graph(capi, oracle_mod, torch_cuda, g, roots, 0)
    # closed form on the compacted grid: ids keep their order, so the level is the
    # Manhattan distance between grid coordinates
    h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64)
    try:
        lv = torch_cuda.empty(g.n, dtype=torch_cuda.int32, device="cuda")
        pr = torch_cuda.empty(g.n, dtype=torch_cuda.int32, device="cuda")
        r = int(roots[0])
        capi.bfs_run(h, r, lv, pr)
        ids = np.arange(g.n)
        x, y, z = ids % 21, (ids // 21) % 17, ids // (21 * 17)
        want = np.abs(x - r % 21) + np.abs(y - (r // 21) % 17) + np.abs(z - r // (21 * 17))
        assert np.array_equal(lv.cpu().numpy(), want)
    finally:
        capi.bfs_graph_destroy(h)
