#!/usr/bin/env python3
"""Benchmark: harmonic-mean GTEPS of single-source BFS on one GB300, with the achieved
fraction of the HBM roofline, an end-to-end figure through the C ABI with host buffers,
and the CPU oracle timed as a baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

A step is one complete search from one root (init, every level's expansion, level loop
on the device). K steps use K distinct seeded roots. TEPS per root = m_c / device time,
m_c = undirected input edges in the traversed component (Sec. 4 of the paper); the value
is the harmonic mean over roots (Sec. 4: 64 roots, harmonic mean). With --gpus N > 1
(torchrun, one process per GPU) every rank runs its own replica of the graph on its own
roots (no collective on the data path) and the value is the sum of per-rank harmonic
means. Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "harmonic-mean GTEPS over roots (single-source BFS); % of HBM peak"
UNIT = "GTEPS"
PROFILES = os.path.join(ROOT, "profiles")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


def harmonic_mean(xs):
    xs = [x for x in xs]
    return len(xs) / sum(1.0 / x for x in xs) if xs and all(x > 0 for x in xs) else 0.0


def strip_comments(src: str) -> str:
    """C++ source without comments and blank lines (so that comment edits keep the hash)."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def kernel_source_hash() -> str:
    """Identifies the single-source expansion code a traffic capture was taken on."""
    h = hashlib.sha256()
    for f in ("bfs_kernels.cu", "common.cuh", "kernels.h"):
        with open(os.path.join(ROOT, "paper_1408_1605_gb300", "csrc", f)) as fh:
            h.update(strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, relabel: bool):
    """Per-launch DRAM bytes of the expansion kernel from the committed ncu summary, if it
    was taken on the current kernel source and the same vertex order (else None)."""
    path = os.path.join(PROFILES, "k_expand_traffic.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    if not m_hash or m_hash.group(1) != kernel_source_hash():
        return None
    m_order = re.search(r"vertex_order:\s*(\S+)", text)
    if (m_order.group(1) if m_order else "as-generated") != ("relabelled" if relabel else "as-generated"):
        return None
    m = re.search(rf"traffic_per_launch\[{re.escape(workload)}\]:\s*([0-9.eE+]+)", text)
    return float(m.group(1)) if m else None


# ------------------------------------------------------------------------------------------
# clocks sampled with nvidia-smi while the timed region runs

class ClockSampler:
    FIELDS = ["timestamp", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.samples.append((time.time(), [x.strip() for x in line.split(",")]))

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self, t0: float, t1: float) -> dict:
        inside = [s for t, s in self.samples if t0 <= t <= t1 + 0.15]
        used = inside if inside else [s for _, s in self.samples]
        sm, mx, reasons = [], [], set()
        for s in used:
            try:
                sm.append(float(s[1]))
                mx.append(float(s[2]))
            except (ValueError, IndexError):
                continue
            for name, val in zip(self.REASONS, s[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples_in_window": len(inside), "samples": len(used)}


def gpu_smi_id():
    try:
        import torch

        p = torch.cuda.get_device_properties(torch.cuda.current_device())
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return None


# ------------------------------------------------------------------------------------------

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def alg_bytes_expand(m_c: int, n_c: int, off_bytes: int) -> int:
    """Algorithmic HBM bytes of one search's expansion launches: every reached vertex's
    row is read once (2 m_c column ids of 4 B), and per reached vertex its offsets pair,
    its queue entry written and read (id 4 B + scan value), and its level and parent."""
    per_vertex = 2 * off_bytes + (4 + off_bytes) * 2 + 8
    return 8 * m_c + per_vertex * n_c


def graph_cache_dir(wl):
    """Where ranks share a generated graph: $GBFS_GRAPH_CACHE, else /dev/shm or the temp
    directory, whichever has room for twice the graph (None if neither has). A graph read
    from a file is not cached: every rank reads the file."""
    if wl.kind == "edgelist":
        return None
    if os.environ.get("GBFS_GRAPH_CACHE"):
        return os.environ["GBFS_GRAPH_CACHE"]
    import tempfile

    n = 1 << wl.scale if wl.kind in ("rmat", "uniform") else math.prod(wl.dims)
    entries = 2 * wl.edge_factor * n if wl.kind in ("rmat", "uniform") else 6 * n
    need = 2 * (4 * entries + 8 * (n + 1))
    for d in ("/dev/shm", tempfile.gettempdir()):
        try:
            st = os.statvfs(d)
        except OSError:
            continue
        if st.f_bavail * st.f_frsize > need:
            return os.path.join(d, "gbfs_graphs")
    return None


def replica_roots(pool, warmup: int, world: int, rank: int):
    """Each rank is an independent replica (a single search does not shard without a
    per-level exchange): the pool's first warmup x world roots warm the ranks up and the
    rest are dealt round-robin, so the ranks' timed roots are disjoint and cover the pool."""
    return pool[: warmup * world][rank::world], pool[warmup * world:][rank::world]


def aggregate_replicas(hm: float, e2e_hm: float, ms_step: float, world: int, device="cuda"):
    """Whole-job figures of the replica ranks: the sum of their harmonic-mean GTEPS (every
    rank searches its own roots: weak scaling) and the slowest rank's time per step. No data
    path collective; one all_gather of three numbers after the timed region."""
    if world <= 1:
        return hm, e2e_hm, ms_step
    import torch

    t = torch.tensor([hm, e2e_hm, ms_step], dtype=torch.float64, device=device)
    gathered = [torch.zeros_like(t) for _ in range(world)]
    torch.distributed.all_gather(gathered, t)
    return (float(sum(x[0] for x in gathered)), float(sum(x[1] for x in gathered)),
            float(max(x[2] for x in gathered)))


def run_reference(args, wl, g, roots, rank):
    """The reference arm: the CPU oracle as it stands, one thread, on the same graph and
    roots; steps are bounded by a wall-clock budget so the run ends within minutes."""
    import oracle

    if rank != 0:
        return 0
    t0 = time.perf_counter()
    _ = int(g.cols[:: 1 << 12].sum())  # touch the arrays once (warm-up)
    warm_s = time.perf_counter() - t0
    teps, times, used = [], [], 0
    budget = float(os.environ.get("GBFS_REFERENCE_BUDGET_S", "150"))
    t_start = time.perf_counter()
    for r in roots[: args.steps]:
        t = time.perf_counter()
        lv, _ = oracle.bfs(g.offsets, g.cols, int(r))
        dt = time.perf_counter() - t
        m_c = oracle.component_edges(g.offsets, lv)
        teps.append(m_c / dt / 1e9)
        times.append(dt)
        used += 1
        if time.perf_counter() - t_start > budget:
            break
    hm = harmonic_mean(teps)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(hm, 4), "unit": UNIT, "n_gpus": args.gpus,
        "steps": used, "steps_requested": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * sum(times) / max(used, 1), 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i32/i64", "data": data_kind(wl),
        "config": config_for(wl, g, args),
        "cpu_baseline": {"value": round(hm, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{used} of {args.steps} requested roots (wall-clock budget {budget:.0f} s); "
                                   f"warm-up = one strided pass over the CSR ({warm_s:.1f} s)", **host_cpu()},
        "e2e": {"value": round(hm, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def use_relabel(kind: str, mode: str) -> bool:
    """Degree relabelling (BFS_RELABEL_DEGREE) pays on skewed degree distributions (R-MAT);
    on uniform random graphs and grids it was measured slightly slower, so auto leaves them,
    and graphs read from files (not measured) keep their order unless asked."""
    return mode == "on" or (mode == "auto" and kind == "rmat")


def create_graph(capi, g, relabel: bool) -> int:
    return capi.bfs_graph_create(g.offsets, g.cols, g.n, g.nnz,
                                 capi.BFS_OFFSETS_INT64 | (capi.BFS_RELABEL_DEGREE if relabel else 0))


L2_BYTES = 129e6


def l2_note(g) -> str:
    """How the timed searches stand to the L2 cache: the rules ask for inputs larger than
    L2 or a flush between timed iterations; no flush is done, so say which case holds."""
    if 4 * g.nnz > L2_BYTES:
        return "inputs larger than L2 (the column array alone exceeds the 129 MB L2)"
    return "inputs smaller than L2 and not flushed between roots (warm-cache figure)"


def data_kind(wl) -> str:
    return f"edge list file ({os.path.basename(wl.path)})" if wl.kind == "edgelist" else "synthetic"


def config_for(wl, g, args) -> dict:
    return {"workload": wl.name, "description": wl.description, "n_vertices": g.n, "csr_entries": g.nnz,
            "offsets": "int64" if g.nnz > 2**31 - 1 else "int32", "roots": args.steps,
            "vertex_order": "as generated (the oracle's input)" if args.impl == "reference"
            else "relabelled by degree at graph creation" if use_relabel(wl.kind, args.relabel) else "as generated",
            "l2_flush": l2_note(g),
            "parallelism": f"replicas x{args.gpus}"}


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rmat-s26-ef16")
    ap.add_argument("--edge-list", default="",
                    help="run on a graph read from this file (text edge list or MatrixMarket) instead of --workload")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=16)
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-waves", type=int, default=0,
                    help="64-root waves in the batched leg (default: 4 on R-MAT s22, i.e. 256 roots; else 1)")
    ap.add_argument("--no-direction", action="store_true")
    ap.add_argument("--mode", default="single", choices=["single", "serve", "multigraph"])
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--serve-rates", default="2000,5000,10000,20000,50000")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--serve-levels-per-round", type=int, default=0)
    ap.add_argument("--relabel", default="auto", choices=["auto", "on", "off"],
                    help="BFS_RELABEL_DEGREE at graph creation (auto: R-MAT graphs only)")
    args = ap.parse_args()
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "multigraph":
        return run_multigraph(args)
    args.warmup = max(args.warmup, 0)

    from paper_1408_1605_gb300.workloads import WORKLOADS

    if args.edge_list:
        from paper_1408_1605_gb300.workloads import edge_list_workload

        wl = edge_list_workload(args.edge_list)
    else:
        wl = WORKLOADS[args.workload]
    args.grid_dims = wl.dims if wl.kind == "grid3d" else None
    rank, world, local_rank = dist_env()
    t = time.perf_counter()
    cache = graph_cache_dir(wl) if (world > 1 or os.environ.get("GBFS_GRAPH_CACHE")) else None
    g = None
    if cache:  # one generation per node, not per rank: ranks share the saved graph
        try:
            g = wl.make_shared(cache)
        except OSError as e:
            log(f"[bench] shared graph cache unusable ({e}); generating in this process")
    if g is None:
        g = wl.make()
    log(f"[bench] {wl.name}: n={g.n} nnz={g.nnz} prepared in {time.perf_counter() - t:.1f}s")
    pool = wl.pick_roots(g, max(64, (args.warmup + args.steps) * world))
    if pool.size == 0:
        raise SystemExit("graph has no vertex with degree > 0")
    import numpy as np

    need = (args.warmup + args.steps) * world
    pool = np.resize(pool, need) if pool.size < need else pool[:need]
    if args.impl == "reference":
        _, timed_roots = replica_roots(pool, args.warmup, world, rank)
        return run_reference(args, wl, g, timed_roots, rank)

    import torch

    from paper_1408_1605_gb300 import capi

    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    warm_roots, timed_roots = replica_roots(pool, args.warmup, world, rank)

    t = time.perf_counter()
    relabel = use_relabel(wl.kind, args.relabel)
    h = create_graph(capi, g, relabel)
    tune_class = wl.kind + ("-relabel" if relabel else "")
    log(f"[bench] upload{' + relabel' if relabel else ''} {time.perf_counter() - t:.1f}s")
    off_bytes = 8 if g.nnz > 2**31 - 1 else 4
    lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
    pr = torch.empty(g.n, dtype=torch.int32, device="cuda")
    shapes = {}
    if not args.no_autotune:
        from paper_1408_1605_gb300 import autotune

        tune_roots = pool[: max(3, min(len(pool), 3))]
        rec = autotune.apply_or_tune(h, capi.BFS_KERNEL_SINGLE, tune_class, g.n, tune_roots, lv, pr)
        shapes["single"] = {"shape": rec["shape"], **rec["shape_info"], "cached": rec["cached"],
                            "loop": ["persistent", "graph", "host"][rec.get("loop", 1)],
                            "persist_ctas_per_sm": rec.get("persist_ctas", 0)}
        log(f"[bench] single-source shape {shapes['single']} ms per shape {rec.get('ms')}")
    for r in warm_roots:
        capi.bfs_run(h, int(r), lv, pr, want_stats=True)
    torch.cuda.synchronize()

    sampler = ClockSampler(gpu_smi_id())
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    w0 = time.time()
    ev0.record()
    for r in timed_roots:
        st = capi.bfs_run(h, int(r), lv, pr, want_stats=True)
        stats.append(st.as_dict())
    ev1.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    w1 = time.time()
    time.sleep(0.2)
    sampler.stop()
    clocks = sampler.summary(w0, w1)
    elapsed_ms = ev0.elapsed_time(ev1)

    teps = [s["edges_traversed"] / (s["device_ms"] * 1e-3) / 1e9 for s in stats]
    hm = harmonic_mean(teps)
    total_bytes = sum(alg_bytes_expand(s["edges_traversed"], s["vertices_reached"], off_bytes) for s in stats)
    expand_ms = sum(s["expand_ms"] for s in stats)
    launches_expand = sum(s["depth"] for s in stats)
    launches = sum(s["depth"] + 1 for s in stats)
    achieved = total_bytes / (expand_ms * 1e-3) / 1e9

    # end to end through the C ABI with host (pinned) outputs: device->host copy of the
    # levels and parents inside the timed region, the root passed in as the step's input
    e2e_roots = timed_roots[: max(1, min(args.e2e_steps, len(timed_roots)))]
    hl = torch.empty(g.n, dtype=torch.int32, pin_memory=True)
    hp = torch.empty(g.n, dtype=torch.int32, pin_memory=True)
    capi.bfs_run(h, int(e2e_roots[0]), hl, hp)
    e2e_teps = []
    for r in e2e_roots:
        t = time.perf_counter()
        st = capi.bfs_run(h, int(r), hl, hp, want_stats=True)
        dt = time.perf_counter() - t
        e2e_teps.append(st.edges_traversed / dt / 1e9)
    e2e_hm = harmonic_mean(e2e_teps)

    direction = None
    if not args.no_direction:
        direction = direction_leg(h, g, timed_roots, stats, wl, args, lv, pr)

    batched = None
    if not args.no_batched:
        waves = args.batch_waves or (4 if wl.name == "rmat-s22-ef16" else 1)
        if waves * 64 <= len(timed_roots):
            broots, bstats = timed_roots[: waves * 64], stats[: waves * 64]
        else:  # more roots than the timed ones: same seeded draw, single-source times taken here
            broots = wl.pick_roots(g, waves * 64)
            bstats = [capi.bfs_run(h, int(r), lv, pr, want_stats=True).as_dict() for r in broots]
        batched = batched_leg(h, g, broots, bstats, None if args.no_autotune else tune_class, shapes)

    # aggregate over replicas: sum of per-rank harmonic means; time = max over ranks
    value, e2e_hm, ms_step = aggregate_replicas(hm, e2e_hm, elapsed_ms / max(len(stats), 1), world)

    parity, cpu_baseline = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        parity, cpu_baseline = cpu_leg(args, g, h, timed_roots, lv, pr)

    if rank == 0:
        peaks = load_peaks()
        traffic = profiled_traffic(wl.name, relabel)
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": len(stats),
            "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "i32/i64", "data": data_kind(wl),
            "config": dict(config_for(wl, g, args), shapes=shapes),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                         "kernel": "k_expand", "launches": launches_expand,
                         "peak_source": peaks["source"],
                         "alg_bytes_per_launch": round(total_bytes / max(launches_expand, 1))},
            "e2e": {"value": round(e2e_hm, 3), "unit": UNIT, "h2d_bytes_per_step": 4,
                    "d2h_bytes_per_step": 8 * g.n + 72, "steps": len(e2e_roots)},
            "gpu_launches": launches,
            "clocks": clocks,
            "detail": {"mean_device_ms": round(sum(s["device_ms"] for s in stats) / len(stats), 4),
                       "mean_expand_ms": round(expand_ms / len(stats), 4),
                       "mean_depth": round(launches_expand / len(stats), 2),
                       "mean_m_c": round(sum(s["edges_traversed"] for s in stats) / len(stats)),
                       "min_gteps": round(min(teps), 3), "max_gteps": round(max(teps), 3)},
        }
        if direction is not None:
            line["direction_optimizing"] = direction
        if batched is not None:
            line["batched"] = batched
        if parity is not None:
            line["parity"] = parity
        if cpu_baseline is not None:
            line["cpu_baseline"] = cpu_baseline
        print(json.dumps(line), flush=True)
    capi.bfs_graph_destroy(h)
    if world > 1:
        torch.distributed.destroy_process_group()
    if parity is not None and not parity["ok"]:
        return 1
    return 0


def direction_leg(h, g, roots, single_stats, wl, args, lv, pr):
    """The same roots with bottom-up levels allowed (persistent loop, Beamer's switching):
    harmonic-mean GTEPS, levels checked exact against the top-down results on sampled roots."""
    import numpy as np

    from paper_1408_1605_gb300 import capi

    saved = (capi.bfs_graph_get_option(h, capi.BFS_OPT_LOOP), capi.bfs_graph_get_option(h, capi.BFS_OPT_BOTTOM_UP),
             capi.bfs_graph_get_shape(h, capi.BFS_KERNEL_SINGLE),
             capi.bfs_graph_get_option(h, capi.BFS_OPT_PERSIST_CTAS))
    capi.bfs_graph_set_option(h, capi.BFS_OPT_BOTTOM_UP, 1)
    shape_ms = None
    if not args.no_autotune:
        best, shape_ms = capi.bfs_tune(h, capi.BFS_KERNEL_SINGLE, roots[:3], lv, pr)
    else:
        capi.bfs_graph_set_option(h, capi.BFS_OPT_LOOP, capi.BFS_LOOP_PERSISTENT)
    shape = capi.bfs_graph_get_shape(h, capi.BFS_KERNEL_SINGLE)
    for r in roots[:3]:
        capi.bfs_run(h, int(r), lv, pr, want_stats=True)
    st = [capi.bfs_run(h, int(r), lv, pr, want_stats=True).as_dict() for r in roots]
    teps = [s["edges_traversed"] / (s["device_ms"] * 1e-3) / 1e9 for s in st]
    # parity: levels identical to the top-down search on a few roots (which the oracle checks)
    import torch

    import oracle

    ok, parents_ok = True, True
    tl = torch.empty_like(lv)
    tp = torch.empty_like(pr)
    for i, r in enumerate(roots[:4]):
        capi.bfs_run(h, int(r), lv, pr)
        capi.bfs_graph_set_option(h, capi.BFS_OPT_BOTTOM_UP, 0)
        capi.bfs_run(h, int(r), tl, tp)
        capi.bfs_graph_set_option(h, capi.BFS_OPT_BOTTOM_UP, 1)
        ok &= bool(torch.equal(lv, tl))
        if i == 0:  # parents of the bottom-up search: valid BFS tree for the (oracle-checked) levels
            ref = tl.cpu().numpy()
            code, _ = oracle.check_tree(g.offsets, g.cols, int(r), ref, lv.cpu().numpy(), pr.cpu().numpy())
            parents_ok = code == 0
    capi.bfs_graph_set_option(h, capi.BFS_OPT_LOOP, saved[0])
    capi.bfs_graph_set_option(h, capi.BFS_OPT_BOTTOM_UP, saved[1])
    capi.bfs_graph_set_shape(h, capi.BFS_KERNEL_SINGLE, saved[2])
    capi.bfs_graph_set_option(h, capi.BFS_OPT_PERSIST_CTAS, saved[3])
    return {"value": round(harmonic_mean(teps), 3), "unit": UNIT, "steps": len(st), "shape": shape,
            "mean_device_ms": round(sum(s["device_ms"] for s in st) / len(st), 4),
            "mean_bottom_up_levels": round(sum(s["bottom_up_levels"] for s in st) / len(st), 2),
            "levels_equal_top_down_on_roots": 4, "levels_equal": ok, "parents_valid": parents_ok,
            "note": "same BFS (levels identical, parents valid); large levels run bottom-up (Beamer direction switching)"}


def batched_leg(h, g, roots, single_stats, graph_class=None, shapes=None):
    """The same roots as 64-root waves (bfs_run_batch): aggregate GTEPS of the waves against
    the aggregate of the single-source searches of exactly these roots (sum m_c / sum time
    for both)."""
    import torch

    from paper_1408_1605_gb300 import capi

    wave = 64
    k = min(wave, len(roots))
    lv = torch.empty((k, g.n), dtype=torch.int32, device="cuda")
    pr = torch.empty((k, g.n), dtype=torch.int32, device="cuda")
    if graph_class is not None:
        from paper_1408_1605_gb300 import autotune

        rec = autotune.apply_or_tune(h, capi.BFS_KERNEL_BATCH, graph_class, g.n, roots[:k], lv, pr)
        if shapes is not None:
            shapes["batch"] = {"shape": rec["shape"], **rec["shape_info"], "cached": rec["cached"]}
        log(f"[bench] batch shape {rec['shape']} ms per shape {rec.get('ms')}")
    capi.bfs_run_batch(h, roots[:k], lv, pr, want_stats=True)  # warm-up (buffers, graph)
    edges, ms, waves = 0, 0.0, 0
    for i in range(0, len(roots), wave):
        part = roots[i:i + wave]
        st = capi.bfs_run_batch(h, part, lv[: len(part)], pr[: len(part)], want_stats=True)
        edges += sum(s.edges_traversed for s in st)
        ms += st[0].device_ms
        waves += 1
    single_agg = sum(s["edges_traversed"] for s in single_stats) / (sum(s["device_ms"] for s in single_stats) * 1e-3)
    agg = edges / (ms * 1e-3)
    # the same waves with bottom-up levels allowed (BFS_OPT_BOTTOM_UP applies to waves too)
    saved_bu = capi.bfs_graph_get_option(h, capi.BFS_OPT_BOTTOM_UP)
    capi.bfs_graph_set_option(h, capi.BFS_OPT_BOTTOM_UP, 1)
    capi.bfs_run_batch(h, roots[:k], lv, pr, want_stats=True)  # warm-up (new wave loop)
    edges_do, ms_do, bu_levels = 0, 0.0, 0
    for i in range(0, len(roots), wave):
        part = roots[i:i + wave]
        st = capi.bfs_run_batch(h, part, lv[: len(part)], pr[: len(part)], want_stats=True)
        edges_do += sum(s.edges_traversed for s in st)
        ms_do += st[0].device_ms
        bu_levels += st[0].bottom_up_levels
    capi.bfs_graph_set_option(h, capi.BFS_OPT_BOTTOM_UP, saved_bu)
    agg_do = edges_do / (ms_do * 1e-3)
    del lv, pr
    torch.cuda.empty_cache()
    assert len(single_stats) == len(roots)
    return {"waves": waves, "roots_per_wave": wave, "roots": len(roots), "aggregate_gteps": round(agg / 1e9, 3),
            "single_source_aggregate_gteps": round(single_agg / 1e9, 3), "ratio": round(agg / single_agg, 3),
            "ms_per_wave": round(ms / waves, 3),
            "direction_optimizing": {"aggregate_gteps": round(agg_do / 1e9, 3),
                                     "ratio_vs_single_top_down": round(agg_do / single_agg, 3),
                                     "ms_per_wave": round(ms_do / waves, 3),
                                     "bottom_up_levels_per_wave": round(bu_levels / waves, 2)}}


def run_serve(args) -> int:
    """Serving workload: four resident graphs (R-MAT s20 and s24, grid 192^3, uniform 2^23
    vertices of mean degree 8), queries with seeded uniform roots arriving as a Poisson
    process, admitted into up-to-64-slot waves per graph. One JSON line with p50 / p99
    latency and aggregate GTEPS per offered rate."""
    import numpy as np
    import torch

    from paper_1408_1605_gb300 import capi, serving
    from paper_1408_1605_gb300.workloads import WORKLOADS

    rank, world, local_rank = dist_env()
    torch.cuda.set_device(local_rank)
    names = ["rmat-s20-ef16", "rmat-s24-ef16", "grid3d-192", "uniform-n8M-deg8"]
    gs, hs = [], []
    for nm in names:
        t = time.perf_counter()
        g = WORKLOADS[nm].make()
        gs.append(g)
        hs.append(create_graph(capi, g, use_relabel(WORKLOADS[nm].kind, args.relabel)))
        log(f"[serve] {nm}: n={g.n} nnz={g.nnz} ({time.perf_counter() - t:.1f}s)")
    n_buf = 96  # output buffers per graph, reused once their query completes
    pools = [[(torch.empty(g.n, dtype=torch.int32, device="cuda"), torch.empty(g.n, dtype=torch.int32, device="cuda"))
              for _ in range(n_buf)] for g in gs]
    results = []
    for rate in [float(x) for x in args.serve_rates.split(",")]:
        srv = capi.bfs_serve_create(memory_cap_bytes=64 << 30, levels_per_round=args.serve_levels_per_round)
        ids = [capi.bfs_serve_add_graph(srv, h) for h in hs]
        nq = int(min(4000, max(200, rate * args.serve_seconds)))
        arrivals, gsel, roots = serving.poisson_schedule(nq, rate, [g.n for g in gs], seed=20140806 + 4)
        in_use = [[None] * n_buf for _ in gs]
        nxt = [0] * len(gs)
        tickets = []
        t0 = time.perf_counter()
        for i in range(nq):
            target = t0 + arrivals[i]
            while time.perf_counter() < target:
                pass
            gi = int(gsel[i])
            j = nxt[gi]
            nxt[gi] = (j + 1) % n_buf
            if in_use[gi][j] is not None:  # buffer still owned by an earlier query
                capi.bfs_serve_wait(srv, in_use[gi][j], 600000)
            lv, pr = pools[gi][j]
            tk = capi.bfs_serve_submit(srv, ids[gi], int(roots[i]), lv, pr)
            in_use[gi][j] = tk
            tickets.append(tk)
        for tk in tickets:
            capi.bfs_serve_wait(srv, tk, 600000)
        offered = time.perf_counter() - t0
        rep = capi.bfs_serve_stats(srv)
        capi.bfs_serve_destroy(srv)
        results.append({"offered_qps": rate, "queries": nq, "achieved_qps": round(nq / offered, 1),
                        "p50_ms": round(rep["latency_p50_ms"], 3), "p99_ms": round(rep["latency_p99_ms"], 3),
                        "mean_ms": round(rep["latency_mean_ms"], 3), "gteps": round(rep["gteps"], 3),
                        "max_concurrent": rep["max_concurrent"], "levels": rep["levels"]})
        log(f"[serve] rate {rate:.0f}: {results[-1]}")
    for h in hs:
        capi.bfs_graph_destroy(h)
    if rank == 0:
        best = max(r["gteps"] for r in results)
        print(json.dumps({"metric": "serving: p50/p99 latency and aggregate GTEPS under Poisson load",
                          "mode": "serve", "value": best, "unit": "GTEPS", "n_gpus": world,
                          "higher_is_better": True, "data": "synthetic", "dtype": "i32/i64",
                          "config": {"workload": "serve: rmat-s20, rmat-s24, grid3d-192, uniform-n8M-deg8",
                                     "roots": "seeded uniform per graph", "wave": 64,
                                     "levels_per_round": args.serve_levels_per_round or 8,
                                     "memory_cap_bytes": 64 << 30,
                                     "relabel": args.relabel},
                          "rates": results}), flush=True)
    return 0


def run_multigraph(args) -> int:
    """Uneven batch: 32 R-MAT graphs (edge factor 16) with scales drawn uniformly from 14 to
    20 (seeded), 64 roots each, one 64-root wave per graph; every wave is a CUDA-graph level
    loop, the waves of different graphs run on four streams at once, and each graph's batch
    shape comes from the autotuner (cached per scale). Aggregate GTEPS = sum of m_c over all
    roots / device time of the whole set."""
    import numpy as np
    import torch

    import oracle
    from paper_1408_1605_gb300 import autotune, capi, graphs

    rank, world, local_rank = dist_env()
    torch.cuda.set_device(local_rank)
    rng = np.random.default_rng(20140806 + 3)
    scales = rng.integers(14, 21, 32)
    gs, hs, roots, outs = [], [], [], []
    t = time.perf_counter()
    for i, sc in enumerate(scales):
        g = graphs.rmat(int(sc), 16, seed=20140806 + 300 + i)
        h = create_graph(capi, g, use_relabel("rmat", args.relabel))
        r = graphs.pick_roots(g, 64, graphs.root_seed(20140806 + 300 + i))
        lv = torch.empty((r.size, g.n), dtype=torch.int32, device="cuda")
        pr = torch.empty((r.size, g.n), dtype=torch.int32, device="cuda")
        gs.append(g), hs.append(h), roots.append(r), outs.append((lv, pr))
    log(f"[multigraph] 32 graphs, scales {sorted(scales.tolist())}, built in {time.perf_counter() - t:.1f}s")
    chosen = {}
    for g, h, r, (lv, pr) in zip(gs, hs, roots, outs):
        rec = autotune.apply_or_tune(h, capi.BFS_KERNEL_BATCH, "rmat" + ("-relabel" if use_relabel("rmat", args.relabel)
                                                                         else ""), g.n, r, lv, pr)
        chosen[int(round(np.log2(g.n)))] = rec["shape"]
    streams = [torch.cuda.Stream() for _ in range(4)]

    def one_pass(want_stats):
        sts = []
        for i, (h, r, (lv, pr)) in enumerate(zip(hs, roots, outs)):
            st = capi.bfs_run_batch(h, r, lv, pr, stream=streams[i % 4], want_stats=want_stats)
            sts.append(st)
        return sts

    stats = one_pass(True)  # warm-up, and the per-root m_c
    edges = sum(s.edges_traversed for st in stats for s in st)
    for _ in range(max(args.warmup - 1, 0)):
        one_pass(False)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    main = torch.cuda.current_stream()
    times = []
    for _ in range(max(1, args.steps)):
        ev0.record(main)
        for s in streams:
            s.wait_event(ev0)
        one_pass(False)
        for s in streams:
            e = torch.cuda.Event()
            e.record(s)
            main.wait_event(e)
        ev1.record(main)
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1))
    ms = float(np.median(times))
    # parity on sampled roots of four graphs
    ok, checked = True, 0
    for i in (0, 10, 20, 31):
        L, P = outs[i][0].cpu().numpy(), outs[i][1].cpu().numpy()
        for b in (0, 63):
            ref, _ = oracle.bfs(gs[i].offsets, gs[i].cols, int(roots[i][b]))
            ok &= bool(np.array_equal(L[b], ref))
            ok &= oracle.check_tree(gs[i].offsets, gs[i].cols, int(roots[i][b]), ref, L[b], P[b])[0] == 0
            checked += 1
    for h in hs:
        capi.bfs_graph_destroy(h)
    if rank == 0:
        print(json.dumps({"metric": "aggregate GTEPS, 32 uneven R-MAT graphs x 64 roots (batched waves)",
                          "mode": "multigraph", "value": round(edges / (ms * 1e-3) / 1e9, 3), "unit": "GTEPS",
                          "n_gpus": world, "steps": len(times), "warmup": args.warmup,
                          "ms_per_step": round(ms, 3), "higher_is_better": True, "data": "synthetic",
                          "dtype": "i32/i64",
                          "config": {"workload": "32 R-MAT graphs, scales U{14..20}, EF16, 64 roots each",
                                     "scales": sorted(int(x) for x in scales), "streams": 4,
                                     "batch_shape_per_scale": chosen,
                                     "vertex_order": "relabelled by degree" if use_relabel("rmat", args.relabel)
                                     else "as generated"},
                          "parity": {"roots_checked": checked, "ok": ok}}), flush=True)
    return 0 if ok else 1


def host_cpu() -> dict:
    """The host the oracle is timed on: CPU model (x86 'model name', else the Arm part
    number) and the number of cores present (the oracle uses one)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
        m = re.search(r"^model name\s*:\s*(.+)$", info, re.M) or re.search(r"^CPU part\s*:\s*(\S+)", info, re.M)
        model = m.group(1).strip() if m else None
    except OSError:
        pass
    import platform

    return {"cpu_model": model or platform.machine(), "host_cores": os.cpu_count()}


def cpu_leg(args, g, h, roots, lv, pr):
    """Oracle timed single-threaded on a bounded sample of the timed roots; the GPU result
    for the same roots is checked against it (levels exact, parents valid)."""
    import numpy as np

    import oracle
    from paper_1408_1605_gb300 import capi

    teps, checked, exact_all, valid_all, used = [], 0, True, True, 0
    t_all = time.perf_counter()
    for r in roots:
        t = time.perf_counter()
        ref, _ = oracle.bfs(g.offsets, g.cols, int(r))
        dt = time.perf_counter() - t
        m_c = oracle.component_edges(g.offsets, ref)
        teps.append(m_c / dt / 1e9)
        used += 1
        capi.bfs_run(h, int(r), lv, pr, want_stats=True)
        got_l, got_p = lv.cpu().numpy(), pr.cpu().numpy()
        exact_all &= bool(np.array_equal(got_l, ref))
        code, _ = oracle.check_tree(g.offsets, g.cols, int(r), ref, got_l, got_p)
        valid_all &= code == 0
        checked += 1
        if time.perf_counter() - t_all > args.cpu_budget_s:
            break
    parity = {"roots_checked": checked, "levels_exact": exact_all, "parents_valid": valid_all,
              "ok": exact_all and valid_all}
    dims = getattr(args, "grid_dims", None)
    if dims:
        # full-size closed form on more roots: level = Manhattan distance on the grid
        X, Y, Z = dims
        ids = np.arange(g.n, dtype=np.int64)
        x, y, z = ids % X, (ids // X) % Y, ids // (X * Y)
        closed_ok, n_closed = True, 0
        for r in roots[:8]:
            capi.bfs_run(h, int(r), lv, pr)
            rx, ry, rz = int(r) % X, (int(r) // X) % Y, int(r) // (X * Y)
            want = np.abs(x - rx) + np.abs(y - ry) + np.abs(z - rz)
            closed_ok &= bool(np.array_equal(lv.cpu().numpy(), want))
            n_closed += 1
        parity["closed_form_roots"] = n_closed
        parity["closed_form_ok"] = closed_ok
        parity["ok"] = parity["ok"] and closed_ok
    cpu = {"value": round(harmonic_mean(teps), 4), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{used} of the {len(roots)} timed roots, full searches on the same graph", **host_cpu()}
    return parity, cpu


if __name__ == "__main__":
    sys.exit(main())
