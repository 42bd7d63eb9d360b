"""Host side of the serving load driver (CPU only): the seeded Poisson schedule and the
submit loop's handling of back-pressure (BFS_ERR_BUSY) against a fake server."""
import numpy as np
import pytest


def test_poisson_schedule():
    from paper_1408_1605_gb300 import serving

    sizes = [100, 5000, 7]
    a1, g1, r1 = serving.poisson_schedule(20000, 2000.0, sizes, seed=11)
    a2, g2, r2 = serving.poisson_schedule(20000, 2000.0, sizes, seed=11)
    assert np.array_equal(a1, a2) and np.array_equal(g1, g2) and np.array_equal(r1, r2)  # seeded
    assert a1[0] == 0.0 and np.all(np.diff(a1) >= 0)
    gaps = np.diff(a1)
    # exponential gaps at 2000/s: mean 0.5 ms, standard error 0.5 ms / sqrt(20000)
    assert abs(gaps.mean() - 5e-4) < 5 * 5e-4 / np.sqrt(gaps.size)
    assert set(np.unique(g1).tolist()) == {0, 1, 2}
    for g, n in enumerate(sizes):
        assert r1[g1 == g].min() >= 0 and r1[g1 == g].max() < n
    a3, _, _ = serving.poisson_schedule(100, 2000.0, sizes, seed=12)
    assert not np.array_equal(a1[:100], a3)


def test_run_poisson_retries_busy(monkeypatch):
    from paper_1408_1605_gb300 import capi, serving

    submitted, waited = [], []
    busy = {"left": 3}

    def fake_submit(server, graph_id, root, levels, parents):
        if busy["left"]:
            busy["left"] -= 1
            raise capi.BfsError(6, "queue full")
        submitted.append((graph_id, root))
        return len(submitted)

    monkeypatch.setattr(capi, "bfs_serve_submit", fake_submit)
    monkeypatch.setattr(capi, "bfs_serve_wait", lambda server, ticket, timeout_ms: waited.append(ticket))
    alloc = lambda n: (np.empty(n, np.int32), np.empty(n, np.int32))  # noqa: E731
    res = serving.run_poisson(1, [10, 20], [50, 60], 12, rate=1e5, seed=3, alloc=alloc)
    assert res.busy_retries == 3 and len(res.queries) == 12
    assert [q.ticket for q in res.queries] == list(range(1, 13)) and waited == list(range(1, 13))
    _, gsel, roots = serving.poisson_schedule(12, 1e5, [50, 60], 3)
    assert submitted == [([10, 20][g], int(r)) for g, r in zip(gsel, roots)]


def test_run_poisson_other_errors_propagate(monkeypatch):
    from paper_1408_1605_gb300 import capi, serving

    def fake_submit(*a):
        raise capi.BfsError(1, "bad root")

    monkeypatch.setattr(capi, "bfs_serve_submit", fake_submit)
    with pytest.raises(capi.BfsError):
        serving.run_poisson(1, [0], [10], 2, rate=1e5, seed=1,
                            alloc=lambda n: (np.empty(n, np.int32), np.empty(n, np.int32)))
