"""Serving loop (continuous batching) through the C ABI: every result in a mixed Poisson
load equals the same query run alone (levels bit-exact, parents valid, m_c equal);
admission honours the memory budget; waits time out, cancellation and back-pressure work."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(graphs_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_1605_gb300 import _build, capi

    _build.build_bfs()
    gs = [graphs_mod.rmat(15, 16, seed=41), graphs_mod.grid3d(24, 20, 16), graphs_mod.uniform(30000, 120000, seed=5)]
    handles = [capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64) for g in gs]
    yield torch, capi, gs, handles
    for h in handles:
        capi.bfs_graph_destroy(h)


def _server(capi, handles, **cfg):
    s = capi.bfs_serve_create(**cfg)
    ids = [capi.bfs_serve_add_graph(s, h) for h in handles]
    return s, ids


def _check(oracle, capi, srv, g, q, host):
    st = capi.bfs_serve_result(srv, q.ticket)
    lv = q.levels if host else q.levels.cpu().numpy()
    pr = q.parents if host else q.parents.cpu().numpy()
    ref, _ = oracle.bfs(g.offsets, g.cols, q.root)
    assert np.array_equal(lv, ref), f"root {q.root}: levels differ from the query run alone"
    code, bad = oracle.check_tree(g.offsets, g.cols, q.root, ref, lv, pr)
    assert code == 0, (oracle.TREE_CODES[code], bad)
    assert st.edges_traversed == oracle.component_edges(g.offsets, ref)
    assert st.depth == int(ref.max()) + 1
    # latency (submission to completion) covers the service time (admission to completion)
    assert st.expand_ms >= st.device_ms >= 0.0


@pytest.mark.parametrize("host,lpr", [(False, 1), (False, 0), (True, 3)])
def test_poisson_mix_equals_alone(env, oracle_mod, host, lpr):
    from paper_1408_1605_gb300 import serving

    torch, capi, gs, handles = env
    srv, ids = _server(capi, handles, levels_per_round=lpr)
    try:
        if host:
            alloc = lambda n: (np.empty(n, np.int32), np.empty(n, np.int32))  # noqa: E731
        else:
            alloc = lambda n: (torch.empty(n, dtype=torch.int32, device="cuda"),  # noqa: E731
                               torch.empty(n, dtype=torch.int32, device="cuda"))
        res = serving.run_poisson(srv, ids, [g.n for g in gs], 150, rate=3000.0, seed=7, alloc=alloc)
        for q in res.queries:
            _check(oracle_mod, capi, srv, gs[ids.index(q.graph_id)], q, host)
        rep = capi.bfs_serve_stats(srv)
        assert rep["completed"] == 150 and rep["failed"] == 0
        assert rep["max_concurrent"] > 1  # queries overlapped in waves
        assert 0 < rep["latency_p50_ms"] <= rep["latency_p99_ms"] <= rep["latency_max_ms"]
        assert rep["gteps"] > 0
    finally:
        capi.bfs_serve_destroy(srv)


def test_burst_same_root_and_all_slots(env, oracle_mod):
    """More queries than slots, repeated roots, isolated-root queries."""
    from paper_1408_1605_gb300.serving import Query

    torch, capi, gs, handles = env
    g = gs[0]
    srv, ids = _server(capi, handles[:1], max_wave=8)
    try:
        rng = np.random.default_rng(2)
        iso = np.flatnonzero(g.degrees() == 0)
        roots = list(rng.integers(0, g.n, 30)) + [int(iso[0])] * 3 + [17] * 5
        qs = []
        for r in roots:
            lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
            pr = torch.empty(g.n, dtype=torch.int32, device="cuda")
            q = Query(ids[0], int(r), lv, pr)
            q.ticket = capi.bfs_serve_submit(srv, ids[0], int(r), lv, pr)
            qs.append(q)
        for q in qs:
            capi.bfs_serve_wait(srv, q.ticket, 60000)
            _check(oracle_mod, capi, srv, g, q, host=False)
        assert capi.bfs_serve_stats(srv)["max_concurrent"] <= 8 * 2  # 8 slots x 2 waves per graph
    finally:
        capi.bfs_serve_destroy(srv)


def test_memory_budget_limits_admission(env, oracle_mod):
    """Host-output queries need an 8n-byte staging buffer each; a budget with room for two
    keeps at most two running, and every query still completes correctly."""
    from paper_1408_1605_gb300.serving import Query

    torch, capi, gs, handles = env
    g = gs[0]
    probe, pid = _server(capi, handles[:1])
    base = capi.bfs_serve_stats(probe)["peak_memory_bytes"]
    capi.bfs_serve_destroy(probe)
    cap = base + 2 * 8 * g.n + 1000
    srv, ids = _server(capi, handles[:1], memory_cap_bytes=cap)
    try:
        qs = []
        for r in np.random.default_rng(9).integers(0, g.n, 12):
            q = Query(ids[0], int(r), np.empty(g.n, np.int32), np.empty(g.n, np.int32))
            q.ticket = capi.bfs_serve_submit(srv, ids[0], q.root, q.levels, q.parents)
            qs.append(q)
        for q in qs:
            capi.bfs_serve_wait(srv, q.ticket, 60000)
            _check(oracle_mod, capi, srv, g, q, host=True)
        rep = capi.bfs_serve_stats(srv)
        assert rep["max_concurrent"] <= 2 and rep["peak_memory_bytes"] <= cap
    finally:
        capi.bfs_serve_destroy(srv)


def test_timeout_cancel_and_backpressure(env):
    """A budget with no room for staging blocks host-output queries: wait times out, the
    queue fills (BUSY), cancellation releases them."""
    torch, capi, gs, handles = env
    g = gs[0]
    probe, _ = _server(capi, handles[:1])
    base = capi.bfs_serve_stats(probe)["peak_memory_bytes"]
    capi.bfs_serve_destroy(probe)
    srv, ids = _server(capi, handles[:1], memory_cap_bytes=base + 1000, queue_capacity=2)
    try:
        bufs = [(np.empty(g.n, np.int32), np.empty(g.n, np.int32)) for _ in range(3)]
        t1 = capi.bfs_serve_submit(srv, ids[0], 0, *bufs[0])
        t2 = capi.bfs_serve_submit(srv, ids[0], 1, *bufs[1])
        with pytest.raises(capi.BfsError) as e:
            capi.bfs_serve_submit(srv, ids[0], 2, *bufs[2])
        assert e.value.status == 6  # BUSY
        with pytest.raises(capi.BfsError) as e:
            capi.bfs_serve_wait(srv, t1, 50)
        assert e.value.status == 5  # TIMEOUT
        assert not capi.bfs_serve_poll(srv, t1)
        capi.bfs_serve_cancel(srv, t1)
        capi.bfs_serve_cancel(srv, t2)
        for t in (t1, t2):
            with pytest.raises(capi.BfsError) as e:
                capi.bfs_serve_wait(srv, t, 5000)
            assert e.value.status == 7  # CANCELLED
        rep = capi.bfs_serve_stats(srv)
        assert rep["cancelled"] == 2 and rep["rejected"] == 1
    finally:
        capi.bfs_serve_destroy(srv)


def test_cancel_running_query(env, graphs_mod):
    """A long search (a path: one vertex per level) stops at a level boundary once
    cancelled, or completes first; either way it is reported done."""
    torch, capi, _, _ = env
    from _graphs import path_edges

    n = 200000
    g = graphs_mod.from_edges(n, *path_edges(n))
    h = capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz, capi.BFS_OFFSETS_INT64)
    srv, ids = _server(capi, [h])
    try:
        lv = torch.empty(n, dtype=torch.int32, device="cuda")
        pr = torch.empty(n, dtype=torch.int32, device="cuda")
        t = capi.bfs_serve_submit(srv, ids[0], 0, lv, pr)
        import time

        time.sleep(0.05)
        capi.bfs_serve_cancel(srv, t)
        try:
            capi.bfs_serve_wait(srv, t, 120000)
            status = 0
        except capi.BfsError as e:
            status = e.status
        assert status in (0, 7)
        if status == 7:
            snap = lv.clone()
            time.sleep(0.05)
            assert torch.equal(snap, lv)  # no writes after the cancel was reported
    finally:
        capi.bfs_serve_destroy(srv)
        capi.bfs_graph_destroy(h)


def test_serve_errors(env):
    torch, capi, gs, handles = env
    srv, ids = _server(capi, handles[:1])
    try:
        buf = torch.empty(gs[0].n, dtype=torch.int32, device="cuda")
        with pytest.raises(capi.BfsError) as e:
            capi.bfs_serve_submit(srv, 5, 0, buf, buf)
        assert e.value.status == 8
        with pytest.raises(capi.BfsError) as e:
            capi.bfs_serve_submit(srv, ids[0], gs[0].n, buf, buf)
        assert e.value.status == 1
        t = capi.bfs_serve_submit(srv, ids[0], 0, buf, buf)
        with pytest.raises(capi.BfsError) as e:
            capi.bfs_serve_add_graph(srv, handles[1])
        assert e.value.status == 6
        capi.bfs_serve_wait(srv, t, 60000)
        with pytest.raises(capi.BfsError) as e:
            capi.bfs_serve_wait(srv, 999999, 10)
        assert e.value.status == 8
    finally:
        capi.bfs_serve_destroy(srv)
