"""Kernel-shape tuning and several graphs searched at once on different streams; results
stay exact after every shape change."""
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


def test_tune_single_and_batch_then_exact(torch_cuda, oracle_mod, graphs_mod):
    from paper_1408_1605_gb300 import capi

    torch = torch_cuda
    g = graphs_mod.rmat(17, 16, seed=8)
    roots = graphs_mod.pick_roots(g, 24, 3)
    h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64)
    try:
        lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
        pr = torch.empty(g.n, dtype=torch.int32, device="cuda")
        best, ms = capi.bfs_tune(h, capi.BFS_KERNEL_SINGLE, roots[:3], lv, pr)
        count = capi.bfs_shape_count(capi.BFS_KERNEL_SINGLE)
        assert len(ms) == 4 * count and all(x > 0 for x in ms)
        assert best == int(np.argmin(ms))
        assert capi.bfs_graph_get_shape(h, capi.BFS_KERNEL_SINGLE) == best % count
        assert capi.bfs_graph_get_option(h, capi.BFS_OPT_LOOP) == (capi.BFS_LOOP_GRAPH if best < count
                                                                  else capi.BFS_LOOP_PERSISTENT)
        assert capi.bfs_graph_get_option(h, capi.BFS_OPT_PERSIST_CTAS) == (
            1 if best >= 3 * count else 2 if best >= 2 * count else 0)
        bl = torch.empty((24, g.n), dtype=torch.int32, device="cuda")
        bp = torch.empty((24, g.n), dtype=torch.int32, device="cuda")
        bbest, bms = capi.bfs_tune(h, capi.BFS_KERNEL_BATCH, roots, bl, bp)
        assert capi.bfs_graph_get_shape(h, capi.BFS_KERNEL_BATCH) == bbest
        for kind in (capi.BFS_KERNEL_SINGLE, capi.BFS_KERNEL_BATCH):
            for s in range(capi.bfs_shape_count(kind)):
                capi.bfs_graph_set_shape(h, kind, s)
                if kind == capi.BFS_KERNEL_SINGLE:
                    capi.bfs_graph_set_option(h, capi.BFS_OPT_LOOP, s % 3)
                r = int(roots[s])
                ref, _ = oracle_mod.bfs(g.offsets, g.cols, r)
                if kind == capi.BFS_KERNEL_SINGLE:
                    capi.bfs_run(h, r, lv, pr)
                    got_l, got_p = lv.cpu().numpy(), pr.cpu().numpy()
                else:
                    capi.bfs_run_batch(h, roots, bl, bp)
                    got_l, got_p = bl[s].cpu().numpy(), bp[s].cpu().numpy()
                assert np.array_equal(got_l, ref), (kind, s)
                assert oracle_mod.check_tree(g.offsets, g.cols, r, ref, got_l, got_p)[0] == 0
    finally:
        capi.bfs_graph_destroy(h)


def test_many_graphs_on_streams(torch_cuda, oracle_mod, graphs_mod):
    """Waves of several graphs of different scales in flight together on four streams."""
    from paper_1408_1605_gb300 import capi

    torch = torch_cuda
    rng = np.random.default_rng(14)
    gs = [graphs_mod.rmat(int(s), 16, seed=100 + i) for i, s in enumerate(rng.integers(10, 15, 8))]
    hs = [capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64) for g in gs]
    streams = [torch.cuda.Stream() for _ in range(4)]
    try:
        outs, rootss = [], []
        for i, (g, h) in enumerate(zip(gs, hs)):
            roots = graphs_mod.pick_roots(g, 64, i)
            st = streams[i % 4]
            with torch.cuda.stream(st):
                lv = torch.empty((roots.size, g.n), dtype=torch.int32, device="cuda")
                pr = torch.empty((roots.size, g.n), dtype=torch.int32, device="cuda")
            capi.bfs_run_batch(h, roots, lv, pr, stream=st)
            outs.append((lv, pr))
            rootss.append(roots)
        torch.cuda.synchronize()
        for g, (lv, pr), roots in zip(gs, outs, rootss):
            L, P = lv.cpu().numpy(), pr.cpu().numpy()
            for b in (0, roots.size // 2, roots.size - 1):
                ref, _ = oracle_mod.bfs(g.offsets, g.cols, int(roots[b]))
                assert np.array_equal(L[b], ref)
                assert oracle_mod.check_tree(g.offsets, g.cols, int(roots[b]), ref, L[b], P[b])[0] == 0
    finally:
        for h in hs:
            capi.bfs_graph_destroy(h)
