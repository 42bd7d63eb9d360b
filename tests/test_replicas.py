"""The N > 1 path of bench.py on CPU: replicas only (a single search does not shard without a
per-level exchange). Roots are dealt to ranks disjointly, the whole-job value is the sum of
the ranks' harmonic means and the step time the slowest rank's, gathered once after the
timed region (world size 2, gloo, 127.0.0.1); the reference arm runs on rank 0 only."""
import os
import socket
import types

import numpy as np
import pytest

import bench


def test_replica_roots_disjoint_and_covering():
    pool = np.arange(1000, 1000 + 64 * 4, dtype=np.int32)
    for world in (1, 2, 3, 4):
        parts = [bench.replica_roots(pool, 64, world, r) for r in range(world)]
        assert sorted(np.concatenate(parts).tolist()) == pool[: 64 * world].tolist()
        assert parts[0].tolist() == pool[:64].tolist()  # rank 0 searches the configuration's roots
        for r in range(world):
            assert len(parts[r]) == 64
            for q in range(r + 1, world):
                assert not set(parts[r].tolist()) & set(parts[q].tolist())


def test_aggregate_single_rank_is_identity():
    assert bench.aggregate_replicas(1.5, 2.5, 3.5, 1) == (1.5, 2.5, 3.5)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        hm, e2e, ms = 10.0 * (rank + 1), 1.0 * (rank + 1), 5.0 + 3.0 * rank
        got = bench.aggregate_replicas(hm, e2e, ms, world, device="cpu")
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(" ".join(repr(x) for x in got))
    finally:
        dist.destroy_process_group()


def test_aggregate_gloo_world_size_2(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    if not torch.distributed.is_available() or not torch.distributed.is_gloo_available():
        pytest.skip("gloo backend not available")
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        vals = [float(x) for x in (tmp_path / f"rank{rank}.txt").read_text().split()]
        assert vals == [30.0, 3.0, 8.0]  # sum of values, sum of e2e, max of step times


def test_reference_arm_runs_on_rank_zero_only():
    args = types.SimpleNamespace(steps=4, warmup=1, gpus=2, impl="reference", relabel="auto")
    # rank 1 returns before touching the graph or the oracle
    assert bench.run_reference(args, wl=None, g=None, roots=np.arange(4), rank=1) == 0


def _make_shared_worker(rank, cache_dir, out_dir):
    from paper_1408_1605_gb300.workloads import WORKLOADS

    g = WORKLOADS["rmat-s16-ef16"].make_shared(cache_dir)
    np.save(os.path.join(out_dir, f"off{rank}.npy"), np.asarray(g.offsets))
    np.save(os.path.join(out_dir, f"cols{rank}.npy"), np.asarray(g.cols))


def test_ranks_share_one_generated_graph(tmp_path, graphs_mod):
    """Ranks of a multi-GPU bench run map one saved copy of the graph (generated once, under
    a file lock) instead of generating it each: same arrays as a fresh generation."""
    import multiprocessing as mp

    from paper_1408_1605_gb300.workloads import WORKLOADS

    cache, out = tmp_path / "cache", tmp_path / "out"
    out.mkdir()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_make_shared_worker, args=(r, str(cache), str(out))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    ref = WORKLOADS["rmat-s16-ef16"].make()
    for r in range(2):
        assert np.array_equal(np.load(out / f"off{r}.npy"), ref.offsets)
        assert np.array_equal(np.load(out / f"cols{r}.npy"), ref.cols)
    saved = sorted(p.name for p in cache.iterdir() if p.suffix == ".npy")
    assert len(saved) == 2  # one offsets file, one columns file: a single generation


def test_graph_cache_dir(monkeypatch):
    """The shared graph goes where there is room for it; with no room anywhere each rank
    generates its own copy."""
    from paper_1408_1605_gb300.workloads import WORKLOADS

    wl = WORKLOADS["rmat-s16-ef16"]
    monkeypatch.setenv("GBFS_GRAPH_CACHE", "/some/dir")
    assert bench.graph_cache_dir(wl) == "/some/dir"
    monkeypatch.delenv("GBFS_GRAPH_CACHE")
    full = types.SimpleNamespace(f_bavail=0, f_frsize=4096)
    roomy = types.SimpleNamespace(f_bavail=1 << 30, f_frsize=4096)
    monkeypatch.setattr(bench.os, "statvfs", lambda d: full)
    assert bench.graph_cache_dir(wl) is None
    monkeypatch.setattr(bench.os, "statvfs", lambda d: full if d == "/dev/shm" else roomy)
    got = bench.graph_cache_dir(wl)
    assert got is not None and not got.startswith("/dev/shm")
