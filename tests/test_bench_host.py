"""Host-side pieces of bench.py (CPU only): the harmonic mean over roots, the algorithmic-byte
model of the roofline, the relabelling choice, and the rule that the ncu traffic figure is
reported only for the kernel source and vertex order it was captured on."""
import re
import types

import pytest

import bench


def test_harmonic_mean():
    assert bench.harmonic_mean([1.0, 2.0, 4.0]) == pytest.approx(3 / 1.75)
    assert bench.harmonic_mean([5.0]) == 5.0
    assert bench.harmonic_mean([]) == 0.0
    assert bench.harmonic_mean([1.0, 0.0]) == 0.0  # a failed root is not averaged away


def test_algorithmic_bytes():
    # 2 m_c column ids of 4 B; per reached vertex: offsets pair, queue id + scan value
    # written and read, level and parent
    assert bench.alg_bytes_expand(100, 10, 4) == 8 * 100 + 32 * 10
    assert bench.alg_bytes_expand(100, 10, 8) == 8 * 100 + 48 * 10


def test_use_relabel():
    assert bench.use_relabel("rmat", "auto") and not bench.use_relabel("rmat", "off")
    assert not bench.use_relabel("grid3d", "auto") and bench.use_relabel("grid3d", "on")
    assert not bench.use_relabel("uniform", "auto")


def test_config_names_the_reference_input_order():
    wl = types.SimpleNamespace(name="rmat-s16-ef16", description="d", kind="rmat")
    g = types.SimpleNamespace(n=10, nnz=20)
    ours = types.SimpleNamespace(steps=4, roots=64, impl="ours", relabel="auto", gpus=1)
    ref = types.SimpleNamespace(steps=4, roots=64, impl="reference", relabel="auto", gpus=1)
    assert bench.config_for(wl, g, ours)["vertex_order"].startswith("relabelled")
    assert bench.config_for(wl, g, ref)["vertex_order"].startswith("as generated")


def _traffic_file(tmp_path, h, order, kernel="k_bfs_persistent/shape4"):
    import json

    (tmp_path / "traffic.json").write_text(json.dumps(
        {"kernel_source_hash": h, "entries": {f"rmat-s26-ef16|{order}|{kernel}": {"traffic_per_launch": 2.5e9}}}))


def test_traffic_only_for_matching_source_and_order(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    h = bench.kernel_source_hash()
    _traffic_file(tmp_path, h, "relabelled")
    k = "k_bfs_persistent/shape4"
    assert bench.profiled_traffic("rmat-s26-ef16", True, k) == 2.5e9
    assert bench.profiled_traffic("rmat-s26-ef16", False, k) is None  # other vertex order
    assert bench.profiled_traffic("rmat-s22-ef16", True, k) is None   # workload not profiled
    assert bench.profiled_traffic("rmat-s26-ef16", True, "k_bfs_persistent/shape7") is None  # other shape
    assert bench.profiled_traffic("rmat-s26-ef16", True, "k_expand/shape4") is None   # other kernel
    _traffic_file(tmp_path, "0" * 16, "relabelled")
    assert bench.profiled_traffic("rmat-s26-ef16", True, k) is None   # kernel changed since
    (tmp_path / "traffic.json").write_text("not json")
    assert bench.profiled_traffic("rmat-s26-ef16", True, k) is None


def test_source_hash_ignores_comments():
    a = "int f() {  // one\n  return 1; /* two\n lines */\n}\n"
    b = "int f() {\n\n  return 1;\n}\n// trailing\n"
    assert bench.strip_comments(a) == bench.strip_comments(b)
    assert bench.strip_comments("x = 1;") != bench.strip_comments("x = 2;")


def test_committed_traffic_figures_parse():
    import json
    import os

    path = os.path.join(bench.PROFILES, bench.TRAFFIC_JSON)
    if not os.path.exists(path):
        pytest.skip("no traffic figures committed")
    db = json.load(open(path))
    assert re.fullmatch(r"[0-9a-f]{16}", db["kernel_source_hash"])
    for key, rec in db["entries"].items():
        workload, order, kernel = key.split("|")
        assert order in ("relabelled", "as-generated") and kernel.startswith("k_") and "/shape" in kernel
        assert rec["traffic_per_launch"] > 0
        assert "--clock-control none" in rec["command"]


def test_reference_arm_runs_on_cpu(tmp_path):
    """The reference arm (the CPU oracle, timed) needs no GPU: one JSON line with the
    contract's keys for a small workload."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.abspath(bench.__file__))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                          "rmat-s16-ef16", "--steps", "3", "--warmup", "1"],
                         capture_output=True, text=True, timeout=300, cwd=str(tmp_path))
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GTEPS" and line["value"] > 0
    assert line["steps"] == 3 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["config"]["workload"] == "rmat-s16-ef16"
    assert line["cpu_baseline"]["cpu_model"] and line["cpu_baseline"]["host_cores"] >= 1


def test_reference_arm_on_an_edge_list_file(tmp_path, graphs_mod):
    """bench.py --edge-list runs on a graph read from a text edge list (the form of the
    paper's real-world inputs); the line names the file and says the data is not synthetic."""
    import json
    import os
    import subprocess
    import sys

    import numpy as np

    src, dst = graphs_mod.rmat_edges(12, 16, seed=21)
    path = tmp_path / "toy-graph.txt"
    np.savetxt(path, np.stack([src, dst], 1), fmt="%d", delimiter="\t", header="toy", comments="# ")
    root = os.path.dirname(os.path.abspath(bench.__file__))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--edge-list",
                          str(path), "--steps", "3", "--warmup", "1"],
                         capture_output=True, text=True, timeout=300, cwd=str(tmp_path))
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["config"]["workload"] == "edgelist-toy-graph" and line["data"] == "edge list file (toy-graph.txt)"
    assert line["value"] > 0 and line["steps"] == 3
    assert line["config"]["l2_flush"].startswith("inputs smaller than L2")


def test_l2_note():
    big, small = types.SimpleNamespace(nnz=2_000_000_000, n=1), types.SimpleNamespace(nnz=1000, n=10)
    assert bench.l2_note(big).startswith("inputs larger than L2")
    assert bench.l2_note(small).startswith("inputs smaller than L2")


def test_clock_summary_reads_the_timed_window():
    """Median SM clock and the throttle reasons seen inside the timed window (samples just
    outside it are ignored while the window has any)."""
    cs = bench.ClockSampler(None)
    row = lambda sm, hw="Not Active", cap="Not Active": ["t", str(sm), "2070", "900", "0x0", hw,  # noqa: E731
                                                         "Not Active", "Not Active", cap]
    cs.samples = [(0.5, row(900, hw="Active")), (1.0, row(2070)), (1.1, row(2040, cap="Active")),
                  (1.2, row(2070)), (5.0, row(800))]
    s = bench.ClockSampler.summary(cs, 1.0, 1.2)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples_in_window"] == 3
    cs.samples = [(9.0, row(1500)), (9.1, ["t", "[N/A]"])]  # none inside: all usable samples
    s = cs.summary(1.0, 1.2)
    assert s["sm_mhz"] == 1500.0 and s["samples_in_window"] == 0


def test_load_peaks(tmp_path, monkeypatch):
    import json

    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_peaks()["source"] == "fallback"
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6668.2, "bf16_tflops": 1700}))
    assert bench.load_peaks() == {"hbm_gbs": 6668.2, "source": "measured"}


def test_oracle_checks_catch_planted_mistakes(graphs_mod, oracle_mod):
    """The bench's parity machinery (oracle levels in threads, bounded check queue): the
    oracle's own results pass; a changed level, a parent that is not a neighbour and a
    parent one level too high are each reported for the leg and root they were planted in."""
    import numpy as np

    g = graphs_mod.rmat(12, 16, seed=graphs_mod.GRAPH_SEED_BASE)
    roots = graphs_mod.pick_roots(g, 6, 3)
    checks = bench.OracleChecks(g, threads=3)
    checks.set_ref(int(roots[0]), oracle_mod.bfs(g.offsets, g.cols, int(roots[0]))[0])
    checks.compute(roots)
    for i, r in enumerate(roots):
        lv, pr = oracle_mod.bfs(g.offsets, g.cols, int(r))
        checks.submit("good", i, r, lv, pr)
        bad_l, bad_p = lv.copy(), pr.copy()
        v = int(np.flatnonzero(lv == 2)[0])
        if i % 3 == 0:
            bad_l[v] = 3
        elif i % 3 == 1:
            bad_p[v] = v  # a vertex is not its own neighbour (the builder removes loops)
        else:
            bad_p[v] = int(r)  # the root is at level 0, not 1
        checks.submit("planted", i, r, bad_l, bad_p)
    rep = checks.report()
    checks.close()
    assert rep["good"] == {"roots_checked": 6, "levels_exact": True, "parents_valid": True, "ok": True}
    bad = rep["planted"]
    assert bad["roots_checked"] == 6 and not bad["ok"] and not bad["levels_exact"] and not bad["parents_valid"]
    assert len(bad["failures"]) == 4 and bad["failures"][0]["root"] == int(roots[0])
