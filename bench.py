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


TRAFFIC_JSON = "traffic.json"


def profiled_traffic(workload: str, relabel: bool, kernel: str):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu figures
    (profiles/traffic.json), if they were taken on the current kernel source and the same
    vertex order (else None: the kernel changed since the counters were read)."""
    path = os.path.join(PROFILES, TRAFFIC_JSON)
    try:
        with open(path) as f:
            db = json.load(f)
    except (OSError, ValueError):
        return None
    if db.get("kernel_source_hash") != kernel_source_hash():
        return None
    order = "relabelled" if relabel else "as-generated"
    rec = db.get("entries", {}).get(f"{workload}|{order}|{kernel}")
    return float(rec["traffic_per_launch"]) if rec else None


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


def replica_roots(pool, per_rank: int, world: int, rank: int):
    """Each rank is an independent replica (a single search does not shard without a
    per-level exchange) and searches its own per_rank roots: rank r takes the r-th slice of
    one seeded draw of per_rank x world distinct roots, so the ranks' roots are disjoint and
    rank 0's are the configuration's roots (weak scaling: the work per rank is fixed)."""
    return pool[rank * per_rank:(rank + 1) * per_rank]


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
    roots. Each step is a bounded sample of the GPU arm's step (one search, from the next of
    the same roots, instead of one from each), and the steps are bounded by a wall-clock
    budget so that the run ends within minutes."""
    import oracle

    if rank != 0:
        return 0
    t0 = time.perf_counter()
    _ = int(g.cols[:: 1 << 12].sum())  # touch the arrays once (warm-up)
    warm_s = time.perf_counter() - t0
    teps, times, used = [], [], 0
    budget = float(os.environ.get("GBFS_REFERENCE_BUDGET_S", "150"))
    t_start = time.perf_counter()
    for i in range(args.steps):
        r = roots[i % len(roots)]
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
        "vs_baseline": None, "dtype": "i32", "data": data_kind(wl),
        "config": dict(config_for(wl, g, args), step="one oracle search (a bounded sample of the GPU step)"),
        "cpu_baseline": {"value": round(hm, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{used} of {args.steps} requested steps, one search each from the timed roots in order "
                                   f"(wall-clock budget {budget:.0f} s); "
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
            "offsets": "int64" if g.nnz > 2**31 - 1 else "int32", "roots": args.roots,
            "step": f"one search from each of the {args.roots} roots",
            "vertex_order": "as generated (the oracle's input)" if args.impl == "reference"
            else "relabelled by degree at graph creation" if use_relabel(wl.kind, args.relabel) else "as generated",
            "l2_flush": l2_note(g),
            "parallelism": f"replicas x{args.gpus}"}


def teps_of(s: dict) -> float:
    return s["edges_traversed"] / (s["device_ms"] * 1e-3) / 1e9


class DeviceSlots:
    """Per-root output buffers [k][n] on the device, so that every result a leg produced
    can be checked against the oracle after the timed region. With too little free device
    memory a leg keeps no slots and its results are checked by searching again."""

    def __init__(self, k: int, n: int, want: bool = True, reserve: int = 8 << 30):
        import torch

        self.lv = self.pr = None
        if not want:
            return
        free, _ = torch.cuda.mem_get_info()
        if 2 * 4 * k * n + reserve <= free:
            self.lv = torch.empty((k, n), dtype=torch.int32, device="cuda")
            self.pr = torch.empty((k, n), dtype=torch.int32, device="cuda")

    @property
    def kept(self) -> bool:
        return self.lv is not None

    def release(self):
        self.lv = self.pr = None


def single_pass(capi, h, roots, lv, pr, slots=None):
    """One step: a search from each root (slot i receives root i's result when kept)."""
    out = []
    for i, r in enumerate(roots):
        dl, dp = (slots.lv[i], slots.pr[i]) if slots is not None and slots.kept else (lv, pr)
        out.append(capi.bfs_run(h, int(r), dl, dp, want_stats=True).as_dict())
    return out


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10,
                    help="timed steps; a step is one search from each of the workload's roots (64)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rmat-s26-ef16")
    ap.add_argument("--edge-list", default="",
                    help="run on a graph read from this file (text edge list or MatrixMarket) instead of --workload")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--roots", type=int, default=0, help="roots per step (default: the workload's, 64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity", action="store_true", help="skip the oracle checks of every result")
    ap.add_argument("--parity-threads", type=int, default=0, help="threads of the oracle checks (default: cores)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-batched-config", action="store_true",
                    help="skip the R-MAT scale-22 leg of 256 roots in 4 batched waves")
    ap.add_argument("--batch-waves", type=int, default=1, help="64-root waves in the batched leg")
    ap.add_argument("--no-wide", action="store_true",
                    help="skip the leg on R-MAT s26 edge factor 17 (more than 2^31 - 1 CSR entries: 64-bit offsets)")
    ap.add_argument("--no-direction", action="store_true")
    ap.add_argument("--no-frontier-bitmap", action="store_true",
                    help="skip the leg that times the same searches with the list-or-bitmap frontier switch")
    ap.add_argument("--mode", default="single", choices=["single", "serve", "multigraph"])
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--loop", default="", choices=["", "persistent", "graph", "host"],
                    help="level loop of single-source searches (default: the tuner's choice)")
    ap.add_argument("--shape", type=int, default=-1, help="single-source expansion shape (default: the tuner's)")
    ap.add_argument("--batch-shape", type=int, default=-1,
                    help="batched expansion shape (default: the tuner's; with --no-autotune, the library's)")
    ap.add_argument("--serve-rates", default="2000,5000,10000,20000,50000")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--serve-levels-per-round", type=int, default=0)
    ap.add_argument("--serve-cohort-wait-us", type=int, default=0,
                    help="idle wave's wait for a fuller cohort while a sibling runs (0: library default)")
    ap.add_argument("--relabel", default="auto", choices=["auto", "on", "off"],
                    help="BFS_RELABEL_DEGREE at graph creation (auto: R-MAT graphs only)")
    args = ap.parse_args()
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "multigraph":
        return run_multigraph(args)
    args.warmup = max(args.warmup, 0)
    args.steps = max(args.steps, 1)

    from paper_1408_1605_gb300.workloads import WORKLOADS

    if args.edge_list:
        from paper_1408_1605_gb300.workloads import edge_list_workload

        wl = edge_list_workload(args.edge_list)
    else:
        wl = WORKLOADS[args.workload]
    args.roots = args.roots or wl.roots
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
    import numpy as np

    pool = wl.pick_roots(g, args.roots * world)
    if pool.size == 0:
        raise SystemExit("graph has no vertex with degree > 0")
    if pool.size < args.roots * world:  # fewer distinct roots than asked: repeat the draw
        pool = np.resize(pool, args.roots * world)
    roots = replica_roots(pool, args.roots, world, rank)
    if args.impl == "reference":
        return run_reference(args, wl, g, roots, rank)

    import torch

    from paper_1408_1605_gb300 import capi

    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    t = time.perf_counter()
    relabel = use_relabel(wl.kind, args.relabel)
    h = create_graph(capi, g, relabel)
    tune_class = wl.kind + ("-relabel" if relabel else "")
    log(f"[bench] upload{' + relabel' if relabel else ''} {time.perf_counter() - t:.1f}s")
    off_bytes = 8 if g.nnz > 2**31 - 1 else 4
    lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
    pr = torch.empty(g.n, dtype=torch.int32, device="cuda")
    shapes = {"single": single_shape(capi, h, args, tune_class, g, roots, lv, pr)}
    if args.batch_shape >= 0:
        capi.bfs_graph_set_shape(h, capi.BFS_KERNEL_BATCH, args.batch_shape)

    args.keep = rank == 0 and world == 1 and not args.no_parity  # results kept for the oracle checks
    slots = DeviceSlots(len(roots), g.n, args.keep)
    for _ in range(args.warmup):
        single_pass(capi, h, roots, lv, pr)
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
    for _ in range(args.steps):
        stats.extend(single_pass(capi, h, roots, lv, pr, slots))
    ev1.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    w1 = time.time()
    time.sleep(0.2)
    sampler.stop()
    clocks = sampler.summary(w0, w1)
    elapsed_ms = ev0.elapsed_time(ev1)

    hm = harmonic_mean([teps_of(s) for s in stats])
    loop = shapes["single"]["loop"]
    kernel = "k_bfs_persistent" if loop == "persistent" else "k_expand"
    kernel_key = f"{kernel}/shape{shapes['single']['shape']}"  # traffic figures are per compiled shape
    total_bytes = sum(alg_bytes_expand(s["edges_traversed"], s["vertices_reached"], off_bytes) for s in stats)
    expand_ms = sum(s["expand_ms"] for s in stats)
    levels_run = sum(s["depth"] for s in stats)
    launches_kernel = len(stats) if loop == "persistent" else levels_run
    gpu_launches = 2 * len(stats) if loop == "persistent" else levels_run + len(stats)
    achieved = total_bytes / (expand_ms * 1e-3) / 1e9
    last = stats[-len(roots):]  # the last step: the results kept in the slots

    # end to end through the C ABI with host (pinned) outputs: device->host copy of the
    # levels and parents inside the timed region, the root passed in as the step's input
    hl = torch.empty(g.n, dtype=torch.int32, pin_memory=True)
    hp = torch.empty(g.n, dtype=torch.int32, pin_memory=True)
    capi.bfs_run(h, int(roots[0]), hl, hp)
    e2e_teps = []
    for r in roots:
        t = time.perf_counter()
        st = capi.bfs_run(h, int(r), hl, hp, want_stats=True)
        dt = time.perf_counter() - t
        e2e_teps.append(st.edges_traversed / dt / 1e9)
    e2e_hm = harmonic_mean(e2e_teps)
    del hl, hp

    bitmap_leg = None
    if not args.no_frontier_bitmap:
        bitmap_leg = frontier_bitmap_leg(capi, h, g, roots, args, lv, pr, hm)

    direction = None
    if not args.no_direction:
        direction = direction_leg(capi, h, g, roots, args, lv, pr)

    batched = None
    if not args.no_batched:
        k = min(64 * max(args.batch_waves, 1), len(roots))
        tune_batch = not args.no_autotune and args.batch_shape < 0
        batched = batched_leg(capi, h, g, roots[:k], last[:k], tune_class if tune_batch else None, shapes,
                              args.keep)

    # aggregate over replicas: sum of per-rank harmonic means; time = max over ranks
    value, e2e_hm, ms_step = aggregate_replicas(hm, e2e_hm, elapsed_ms / args.steps, world)

    parity, cpu_baseline, batched_config = None, None, None
    if rank == 0 and world == 1:
        checks = None if args.no_parity else OracleChecks(g, args.parity_threads)
        if not args.no_cpu_baseline:
            cpu_baseline = cpu_baseline_leg(g, roots, checks)
        if checks is not None:
            parity = parity_leg(capi, h, g, roots, checks, slots, lv, pr, direction, batched, args, bitmap_leg)
            checks.close()
    for leg in (direction, batched, bitmap_leg):  # release the kept outputs
        for key in ("_slots", "_slots_do", "_options"):
            if leg is not None:
                leg.pop(key, None)
    del slots
    wide = None
    if rank == 0 and world == 1 and not args.no_batched_config and not args.no_batched \
            and wl.name != "rmat-s22-ef16":
        capi.bfs_graph_destroy(h)
        h = None
        torch.cuda.empty_cache()
        batched_config = batched_config_leg(capi, args)
    if rank == 0 and world == 1 and not args.no_wide and wl.name == "rmat-s26-ef16":
        if h is not None:
            capi.bfs_graph_destroy(h)
            h = None
        torch.cuda.empty_cache()
        wide = wide_offsets_leg(capi, args)

    if rank == 0:
        peaks = load_peaks()
        traffic = profiled_traffic(wl.name, relabel, kernel_key)
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "i32", "data": data_kind(wl),
            "config": dict(config_for(wl, g, args), shapes=shapes),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": round(achieved / peaks["hbm_gbs"], 4),
                         "traffic": round(traffic) if traffic else None,
                         "kernel": kernel, "shape": shapes["single"]["shape"], "launches": launches_kernel,
                         "levels": levels_run,
                         "peak_source": peaks["source"],
                         "alg_bytes_per_launch": round(total_bytes / max(launches_kernel, 1))},
            "e2e": {"value": round(e2e_hm, 3), "unit": UNIT, "h2d_bytes_per_step": 4 * len(roots),
                    "d2h_bytes_per_step": (8 * g.n + 72) * len(roots), "searches": len(roots),
                    "timing": "wall clock around each bfs_run call with pinned host outputs"},
            "gpu_launches": gpu_launches,
            "clocks": clocks,
            "detail": {"searches_timed": len(stats),
                       "mean_device_ms": round(sum(s["device_ms"] for s in stats) / len(stats), 4),
                       "mean_expand_ms": round(expand_ms / len(stats), 4),
                       "mean_depth": round(levels_run / len(stats), 2),
                       "mean_m_c": round(sum(s["edges_traversed"] for s in stats) / len(stats)),
                       "min_gteps": round(min(teps_of(s) for s in stats), 3),
                       "max_gteps": round(max(teps_of(s) for s in stats), 3)},
        }
        if bitmap_leg is not None:
            line["frontier_bitmap"] = bitmap_leg
        if direction is not None:
            line["direction_optimizing"] = direction
        if batched is not None:
            line["batched"] = batched
        if batched_config is not None:
            line["batched_rmat_s22_4x64"] = batched_config
        if wide is not None:
            line["wide_offsets_rmat_s26_ef17"] = wide
        if parity is not None:
            line["parity"] = parity
        if cpu_baseline is not None:
            line["cpu_baseline"] = cpu_baseline
        print(json.dumps(line), flush=True)
    if h is not None:
        capi.bfs_graph_destroy(h)
    if world > 1:
        torch.distributed.destroy_process_group()
    ok = (parity is None or parity["ok"]) and (batched_config is None or batched_config.get("parity_ok", True)) \
        and (wide is None or wide.get("parity_ok", True))
    return 0 if ok else 1


def single_shape(capi, h, args, tune_class, g, roots, lv, pr) -> dict:
    """The single-source loop mode and shape: the tuner's (cached per GPU, graph class and
    scale), or the ones given on the command line."""
    loops = {"persistent": capi.BFS_LOOP_PERSISTENT, "graph": capi.BFS_LOOP_GRAPH, "host": capi.BFS_LOOP_HOST}
    names = {v: k for k, v in loops.items()}
    if not args.no_autotune and not args.loop and args.shape < 0:
        from paper_1408_1605_gb300 import autotune

        rec = autotune.apply_or_tune(h, capi.BFS_KERNEL_SINGLE, tune_class, g.n, roots[:3], lv, pr)
        out = {"shape": rec["shape"], **rec["shape_info"], "cached": rec["cached"],
               "loop": names[rec.get("loop", 1)], "persist_ctas_per_sm": rec.get("persist_ctas", 0)}
        log(f"[bench] single-source shape {out} ms per shape {rec.get('ms')}")
        return out
    if args.loop:
        capi.bfs_graph_set_option(h, capi.BFS_OPT_LOOP, loops[args.loop])
    if args.shape >= 0:
        capi.bfs_graph_set_shape(h, capi.BFS_KERNEL_SINGLE, args.shape)
    shape = capi.bfs_graph_get_shape(h, capi.BFS_KERNEL_SINGLE)
    return {"shape": shape, **capi.bfs_shape_info(capi.BFS_KERNEL_SINGLE, shape), "cached": False,
            "loop": names[capi.bfs_graph_get_option(h, capi.BFS_OPT_LOOP)],
            "persist_ctas_per_sm": capi.bfs_graph_get_option(h, capi.BFS_OPT_PERSIST_CTAS)}


def frontier_bitmap_leg(capi, h, g, roots, args, lv, pr, list_hm) -> dict:
    """The same searches (same loop and shape) with the list-or-bitmap switch of the
    paper's Sec. 5 (BFS_FRONTIER_AUTO): a level whose next frontier would hold more than
    n / 32 ids hands it over as a bitmap, unpacked in vertex order. Reports whether it pays
    against the list-only figure; each root's result is kept for the oracle checks."""
    capi.bfs_graph_set_option(h, capi.BFS_OPT_FRONTIER, capi.BFS_FRONTIER_AUTO)
    try:
        single_pass(capi, h, roots[:3], lv, pr)
        slots = DeviceSlots(len(roots), g.n, args.keep)
        st = single_pass(capi, h, roots, lv, pr, slots)
        unpacked = capi.bfs_graph_get_option(h, capi.BFS_OPT_UNPACKED_LEVELS)
    finally:
        capi.bfs_graph_set_option(h, capi.BFS_OPT_FRONTIER, capi.BFS_FRONTIER_LIST)
    hm = harmonic_mean([teps_of(s) for s in st])
    return {"value": round(hm, 3), "unit": UNIT, "searches": len(st), "mode": "auto (list while <= n/32 ids)",
            "mean_device_ms": round(sum(s["device_ms"] for s in st) / len(st), 4),
            "unpacked_levels_last_search": unpacked, "vs_list": round(hm / list_hm, 3) if list_hm else None,
            "pays": bool(list_hm and hm > list_hm), "_slots": slots}


def direction_leg(capi, h, g, roots, args, lv, pr):
    """The same roots with bottom-up levels allowed (persistent loop, Beamer's switching):
    harmonic-mean GTEPS over the roots; each root's result is kept for the oracle checks."""
    saved = (capi.bfs_graph_get_option(h, capi.BFS_OPT_LOOP), capi.bfs_graph_get_option(h, capi.BFS_OPT_BOTTOM_UP),
             capi.bfs_graph_get_shape(h, capi.BFS_KERNEL_SINGLE),
             capi.bfs_graph_get_option(h, capi.BFS_OPT_PERSIST_CTAS))
    capi.bfs_graph_set_option(h, capi.BFS_OPT_BOTTOM_UP, 1)
    if not args.no_autotune:
        capi.bfs_tune(h, capi.BFS_KERNEL_SINGLE, roots[:3], lv, pr)
    else:
        capi.bfs_graph_set_option(h, capi.BFS_OPT_LOOP, capi.BFS_LOOP_PERSISTENT)
    shape = capi.bfs_graph_get_shape(h, capi.BFS_KERNEL_SINGLE)
    single_pass(capi, h, roots[:3], lv, pr)
    slots = DeviceSlots(len(roots), g.n, args.keep)
    st = single_pass(capi, h, roots, lv, pr, slots)
    out = {"value": round(harmonic_mean([teps_of(s) for s in st]), 3), "unit": UNIT, "searches": len(st),
           "shape": shape, "mean_device_ms": round(sum(s["device_ms"] for s in st) / len(st), 4),
           "mean_bottom_up_levels": round(sum(s["bottom_up_levels"] for s in st) / len(st), 2),
           "note": "same BFS (levels identical, parents valid); large levels run bottom-up "
                   "(Beamer direction switching); the TEPS numerator is m_c as for the top-down search",
           "_slots": slots,
           "_options": (capi.bfs_graph_get_option(h, capi.BFS_OPT_LOOP), 1, shape,
                        capi.bfs_graph_get_option(h, capi.BFS_OPT_PERSIST_CTAS))}
    restore_options(capi, h, saved)
    return out


def restore_options(capi, h, saved):
    capi.bfs_graph_set_option(h, capi.BFS_OPT_LOOP, saved[0])
    capi.bfs_graph_set_option(h, capi.BFS_OPT_BOTTOM_UP, saved[1])
    capi.bfs_graph_set_shape(h, capi.BFS_KERNEL_SINGLE, saved[2])
    capi.bfs_graph_set_option(h, capi.BFS_OPT_PERSIST_CTAS, saved[3])


def run_waves(capi, h, roots, lv, pr, wave=64):
    """Device ms and edges of the roots run as consecutive waves of up to 64 roots; wave i
    writes rows [64 i, 64 i + len) of lv / pr."""
    edges, ms, bu, waves = 0, 0.0, 0, 0
    diag = {"loop_ms": 0.0, "levels": 0, "overflow_records": 0}
    for i in range(0, len(roots), wave):
        part = roots[i:i + wave]
        st = capi.bfs_run_batch(h, part, lv[i:i + len(part)], pr[i:i + len(part)], want_stats=True)
        edges += sum(s.edges_traversed for s in st)
        ms += st[0].device_ms
        bu += st[0].bottom_up_levels
        waves += 1
        diag["loop_ms"] += st[0].expand_ms
        diag["levels"] += capi.bfs_graph_get_option(h, capi.BFS_OPT_WAVE_LEVELS)
        diag["overflow_records"] += capi.bfs_graph_get_option(h, capi.BFS_OPT_WAVE_OVERFLOW)
    run_waves.last = {k: round(v / max(waves, 1), 3) for k, v in diag.items()}  # per wave
    return edges, ms, bu, waves


def batched_leg(capi, h, g, roots, single_stats, graph_class=None, shapes=None, keep=True):
    """The same roots as 64-root waves (bfs_run_batch): aggregate GTEPS of the waves against
    the aggregate of the single-source searches of exactly these roots (sum m_c / sum time
    for both), top-down and with bottom-up levels allowed. The waves' outputs stay on the
    device for the oracle checks (those of the bottom-up waves only if there is room for a
    second set; else the bottom-up waves overwrite them and only theirs are checked)."""
    import torch

    k = min(64, len(roots))
    lv = torch.empty((len(roots), g.n), dtype=torch.int32, device="cuda")
    pr = torch.empty((len(roots), g.n), dtype=torch.int32, device="cuda")
    if graph_class is not None:
        from paper_1408_1605_gb300 import autotune

        rec = autotune.apply_or_tune(h, capi.BFS_KERNEL_BATCH, graph_class, g.n, roots[:k], lv[:k], pr[:k])
        if shapes is not None:
            shapes["batch"] = {"shape": rec["shape"], **rec["shape_info"], "cached": rec["cached"]}
        log(f"[bench] batch shape {rec['shape']} ms per shape {rec.get('ms')}")
    capi.bfs_run_batch(h, roots[:k], lv[:k], pr[:k], want_stats=True)  # warm-up (buffers, graph)
    edges, ms, _, waves = run_waves(capi, h, roots, lv, pr)
    per_wave = run_waves.last
    single_agg = sum(s["edges_traversed"] for s in single_stats) / (sum(s["device_ms"] for s in single_stats) * 1e-3)
    agg = edges / (ms * 1e-3)
    slots = DeviceSlots(0, 0, False)
    slots.lv, slots.pr = lv, pr
    # the same waves with bottom-up levels allowed (BFS_OPT_BOTTOM_UP applies to waves too)
    saved_bu = capi.bfs_graph_get_option(h, capi.BFS_OPT_BOTTOM_UP)
    capi.bfs_graph_set_option(h, capi.BFS_OPT_BOTTOM_UP, 1)
    slots_do = DeviceSlots(len(roots), g.n, keep)
    if not slots_do.kept:
        slots_do, slots = slots, None
    capi.bfs_run_batch(h, roots[:k], slots_do.lv[:k], slots_do.pr[:k], want_stats=True)  # warm-up (new loop)
    edges_do, ms_do, bu_levels, _ = run_waves(capi, h, roots, slots_do.lv, slots_do.pr)
    per_wave_do = run_waves.last
    capi.bfs_graph_set_option(h, capi.BFS_OPT_BOTTOM_UP, saved_bu)
    agg_do = edges_do / (ms_do * 1e-3)
    assert len(single_stats) == len(roots)
    return {"waves": waves, "roots_per_wave": 64, "roots": len(roots), "aggregate_gteps": round(agg / 1e9, 3),
            "single_source_aggregate_gteps": round(single_agg / 1e9, 3), "ratio": round(agg / single_agg, 3),
            "ms_per_wave": round(ms / waves, 3), "per_wave": per_wave,
            "direction_optimizing": {"aggregate_gteps": round(agg_do / 1e9, 3),
                                     "ratio_vs_single_top_down": round(agg_do / single_agg, 3),
                                     "ms_per_wave": round(ms_do / waves, 3),
                                     "bottom_up_levels_per_wave": round(bu_levels / waves, 2),
                                     "per_wave": per_wave_do},
            "_slots": slots, "_slots_do": slots_do}


def wide_offsets_leg(capi, args, n_roots: int = 4) -> dict:
    """R-MAT scale 26 with edge factor 17: the cleaned graph has more than 2^31 - 1 CSR
    entries, so the library keeps 64-bit row offsets, frontier scan values and tile
    descriptors. A few seeded roots run single-source and as one batched wave, with the
    same tuned shapes as the scale-26 edge-factor-16 graph; every result is checked against
    the oracle."""
    import torch

    from paper_1408_1605_gb300.workloads import WORKLOADS

    wl = WORKLOADS["rmat-s26-ef17"]
    t = time.perf_counter()
    g = wl.make()
    roots = wl.pick_roots(g, n_roots)
    relabel = use_relabel(wl.kind, args.relabel)
    h = create_graph(capi, g, relabel)
    log(f"[bench] wide offsets {wl.name}: n={g.n} nnz={g.nnz} ({time.perf_counter() - t:.1f}s)")
    try:
        lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
        pr = torch.empty(g.n, dtype=torch.int32, device="cuda")
        sub = argparse.Namespace(**vars(args))
        tune_class = wl.kind + ("-relabel" if relabel else "")
        single = single_shape(capi, h, sub, tune_class, g, roots, lv, pr)
        single_pass(capi, h, roots[:1], lv, pr)
        slots = DeviceSlots(len(roots), g.n, not args.no_parity)
        stats = single_pass(capi, h, roots, lv, pr, slots)
        res = {"n_vertices": g.n, "csr_entries": g.nnz, "offsets": "int64" if g.nnz > 2**31 - 1 else "int32",
               "roots": len(roots), "single_source_hm_gteps": round(harmonic_mean([teps_of(s) for s in stats]), 3),
               "mean_device_ms": round(sum(s["device_ms"] for s in stats) / len(stats), 3), "single_shape": single}
        bl = torch.empty((len(roots), g.n), dtype=torch.int32, device="cuda")
        bp = torch.empty((len(roots), g.n), dtype=torch.int32, device="cuda")
        bst = capi.bfs_run_batch(h, roots, bl, bp, want_stats=True)
        res["batched_wave_ms"] = round(bst[0].device_ms, 3)
        if not args.no_parity:
            checks = OracleChecks(g, args.parity_threads)
            checks.compute(roots)
            for i, r in enumerate(roots):
                checks.submit("single", i, r, *fetch(capi, h, r, slots, i, lv, pr))
                checks.submit("batched", i, r, bl[i].cpu().numpy(), bp[i].cpu().numpy())
            rep = checks.report()
            checks.close()
            res["parity"] = rep
            res["parity_ok"] = all(v["ok"] for v in rep.values())
        del slots, bl, bp
        return res
    finally:
        capi.bfs_graph_destroy(h)
        torch.cuda.empty_cache()


def batched_config_leg(capi, args) -> dict:
    """The batched configuration of the benchmark: R-MAT scale 22 (edge factor 16), 256
    seeded roots run as 4 waves of 64, against single-source searches of the same 256 roots
    on the same GPU; every root's result of both forms is checked against the oracle."""
    import numpy as np
    import torch

    from paper_1408_1605_gb300.workloads import WORKLOADS

    wl = WORKLOADS["rmat-s22-ef16"]
    t = time.perf_counter()
    g = wl.make()
    roots = wl.pick_roots(g, 256)
    relabel = use_relabel(wl.kind, args.relabel)
    h = create_graph(capi, g, relabel)
    log(f"[bench] batched configuration {wl.name}: n={g.n} nnz={g.nnz}, 256 roots ({time.perf_counter() - t:.1f}s)")
    try:
        lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
        pr = torch.empty(g.n, dtype=torch.int32, device="cuda")
        sub = argparse.Namespace(**vars(args))
        tune_class = wl.kind + ("-relabel" if relabel else "")
        single = single_shape(capi, h, sub, tune_class, g, roots, lv, pr)
        single_pass(capi, h, roots[:8], lv, pr)
        slots = DeviceSlots(len(roots), g.n, not args.no_parity)
        stats = single_pass(capi, h, roots, lv, pr, slots)
        shapes = {"single": single}
        res = batched_leg(capi, h, g, roots, stats, None if args.no_autotune else tune_class, shapes,
                          not args.no_parity)
        res["shapes"] = shapes
        res["single_source_hm_gteps"] = round(harmonic_mean([teps_of(s) for s in stats]), 3)
        if not args.no_parity:
            checks = OracleChecks(g, args.parity_threads)
            checks.compute(roots)
            for i, r in enumerate(roots):
                checks.submit("single", i, r, *fetch(capi, h, r, slots, i, lv, pr))
            for leg, key in (("batched", "_slots"), ("batched_bottom_up", "_slots_do")):
                sl = res.get(key)
                if sl is None:
                    continue
                for i, r in enumerate(roots):
                    checks.submit(leg, i, r, sl.lv[i].cpu().numpy(), sl.pr[i].cpu().numpy())
            rep = checks.report()
            checks.close()
            res["parity"] = rep
            res["parity_ok"] = all(v["ok"] for v in rep.values())
        res.pop("_slots", None)
        res.pop("_slots_do", None)
        del slots
        return res
    finally:
        capi.bfs_graph_destroy(h)
        torch.cuda.empty_cache()


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
    batch_shapes = {}
    for nm in names:
        t = time.perf_counter()
        wl = WORKLOADS[nm]
        g = wl.make()
        gs.append(g)
        relabel = use_relabel(wl.kind, args.relabel)
        h = create_graph(capi, g, relabel)
        hs.append(h)
        if not args.no_autotune:
            # the waves take the graph's batch shape when the graph is added to a server:
            # tune it first (one 64-root wave per shape, cached per graph class and scale)
            from paper_1408_1605_gb300 import autotune

            roots = np.asarray(wl.pick_roots(g, 64), dtype=np.int32)
            lv = torch.empty((roots.size, g.n), dtype=torch.int32, device="cuda")
            pr = torch.empty((roots.size, g.n), dtype=torch.int32, device="cuda")
            rec = autotune.apply_or_tune(h, capi.BFS_KERNEL_BATCH, wl.kind + ("-relabel" if relabel else ""), g.n,
                                         roots, lv, pr)
            batch_shapes[nm] = rec["shape"]
            del lv, pr
            torch.cuda.empty_cache()
        log(f"[serve] {nm}: n={g.n} nnz={g.nnz} ({time.perf_counter() - t:.1f}s)")
    n_buf = 96  # output buffers per graph, reused once their query completes
    pools = [[(torch.empty(g.n, dtype=torch.int32, device="cuda"), torch.empty(g.n, dtype=torch.int32, device="cuda"))
              for _ in range(n_buf)] for g in gs]
    results = []
    for rate in [float(x) for x in args.serve_rates.split(",")]:
        srv = capi.bfs_serve_create(memory_cap_bytes=64 << 30, levels_per_round=args.serve_levels_per_round,
                                    cohort_wait_us=args.serve_cohort_wait_us)
        ids = [capi.bfs_serve_add_graph(srv, h) for h in hs]
        nq = int(min(4000, max(200, rate * args.serve_seconds)))
        arrivals, gsel, roots = serving.poisson_schedule(nq, rate, [g.n for g in gs], seed=20140806 + 4)
        in_use = [[None] * n_buf for _ in gs]
        nxt = [0] * len(gs)
        tickets = []
        sampler = ClockSampler(gpu_smi_id())  # SM clocks and throttle reasons while this rate runs
        sampler.start()
        time.sleep(0.3)
        w0 = time.time()
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
        w1 = time.time()
        time.sleep(0.2)
        sampler.stop()
        rep = capi.bfs_serve_stats(srv)
        # per graph: latency (submission to completion) and service time (admission to completion)
        lat = [[] for _ in gs]
        svc = [[] for _ in gs]
        for i, tk in enumerate(tickets):
            st = capi.bfs_serve_result(srv, tk)
            lat[int(gsel[i])].append(st.expand_ms)
            svc[int(gsel[i])].append(st.device_ms)
        capi.bfs_serve_destroy(srv)
        per_graph = {names[gi]: {"queries": len(lat[gi]),
                                 "p50_ms": round(float(np.percentile(lat[gi], 50)), 2),
                                 "p99_ms": round(float(np.percentile(lat[gi], 99)), 2),
                                 "service_mean_ms": round(float(np.mean(svc[gi])), 2)}
                     for gi in range(len(gs)) if lat[gi]}
        results.append({"offered_qps": rate, "queries": nq, "achieved_qps": round(nq / offered, 1),
                        "p50_ms": round(rep["latency_p50_ms"], 3), "p99_ms": round(rep["latency_p99_ms"], 3),
                        "mean_ms": round(rep["latency_mean_ms"], 3), "gteps": round(rep["gteps"], 3),
                        "max_concurrent": rep["max_concurrent"], "levels": rep["levels"],
                        "per_graph": per_graph, "clocks": sampler.summary(w0, w1)})
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
                                     "cohort_wait_us": args.serve_cohort_wait_us or "mean cohort duration",
                                     "memory_cap_bytes": 64 << 30,
                                     "relabel": args.relabel, "batch_shapes": batch_shapes},
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


class OracleChecks:
    """Every GPU result checked against the oracle, outside the timed regions. The oracle's
    levels of each root are computed once, in threads: the oracle is a C library whose calls
    release the GIL, so the checks use the host's cores (these are correctness runs; the CPU
    baseline's timing comes from separate single-threaded runs). A result passes when its
    levels equal the oracle's and its parents form a valid BFS tree for them
    (oracle.check_tree: root, parent edges in the graph, parent one level up). Results wait
    for a free thread in a bounded queue, so at most a few full-size arrays are held."""

    def __init__(self, g, threads: int = 0):
        import concurrent.futures as cf

        self.g = g
        self.threads = threads or min(os.cpu_count() or 1, 32)
        self.pool = cf.ThreadPoolExecutor(self.threads)
        self.refs = {}
        self.futs = []
        self.sem = threading.BoundedSemaphore(self.threads + 2)

    @staticmethod
    def compact(lv):
        import numpy as np

        top = int(lv.max()) if lv.size else 0
        return lv.astype(np.int8) if top < 127 else lv.astype(np.int16) if top < 32767 else lv

    def set_ref(self, root, lv):
        self.refs[int(root)] = self.compact(lv)

    def compute(self, roots):
        import oracle

        todo = [r for r in dict.fromkeys(int(x) for x in roots) if r not in self.refs]

        def one(r):
            lv, _ = oracle.bfs(self.g.offsets, self.g.cols, r)
            return r, self.compact(lv)

        for r, c in self.pool.map(one, todo):
            self.refs[r] = c

    def submit(self, leg: str, i: int, root, levels, parents):
        import numpy as np

        import oracle

        self.sem.acquire()
        root = int(root)

        def job():
            try:
                ref = self.refs[root].astype(np.int32)
                exact = bool(np.array_equal(levels, ref))
                code, bad = oracle.check_tree(self.g.offsets, self.g.cols, root, ref, levels, parents)
                return leg, i, root, exact, code, bad
            finally:
                self.sem.release()

        self.futs.append(self.pool.submit(job))

    def report(self) -> dict:
        import oracle

        out = {}
        for f in self.futs:
            leg, i, root, exact, code, bad = f.result()
            rec = out.setdefault(leg, {"roots_checked": 0, "levels_exact": True, "parents_valid": True,
                                       "failures": []})
            rec["roots_checked"] += 1
            rec["levels_exact"] &= exact
            rec["parents_valid"] &= code == 0
            if (not exact or code) and len(rec["failures"]) < 4:
                rec["failures"].append({"slot": i, "root": root, "code": oracle.TREE_CODES[code], "vertex": bad})
        self.futs = []
        for rec in out.values():
            rec["ok"] = rec["levels_exact"] and rec["parents_valid"]
            if not rec["failures"]:
                del rec["failures"]
        return out

    def close(self):
        self.pool.shutdown(wait=True)


def fetch(capi, h, root, slots, i, lv, pr):
    """Host copies of root i's result: from its slot, or from a new search."""
    if slots is not None and slots.kept:
        return slots.lv[i].cpu().numpy(), slots.pr[i].cpu().numpy()
    capi.bfs_run(h, int(root), lv, pr)
    return lv.cpu().numpy(), pr.cpu().numpy()


def cpu_baseline_leg(g, roots, checks, budget_s: float = 15.0) -> dict:
    """The oracle timed single-threaded (monotonic clock around each call) on a bounded
    sample of the timed roots: roots in order until the budget is spent, at least one. Its
    levels serve the checks of those roots."""
    import oracle

    teps = []
    t_all = time.perf_counter()
    for r in roots:
        t = time.perf_counter()
        lv, _ = oracle.bfs(g.offsets, g.cols, int(r))
        dt = time.perf_counter() - t
        teps.append(oracle.component_edges(g.offsets, lv) / dt / 1e9)
        if checks is not None:
            checks.set_ref(r, lv)
        if time.perf_counter() - t_all > budget_s:
            break
    return {"value": round(harmonic_mean(teps), 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{len(teps)} of the {len(roots)} timed roots, one full search each on the same graph, "
                      "one thread", **host_cpu()}


def parity_leg(capi, h, g, roots, checks, slots, lv, pr, direction, batched, args, bitmap_leg=None) -> dict:
    """Every timed root's result against the oracle: the top-down searches of the last timed
    step, the direction-optimizing searches and the batched waves' slots (all kept on the
    device), plus, on 3D grids, levels equal to the Manhattan distance on sampled roots."""
    import numpy as np

    t = time.perf_counter()
    checks.compute(roots)
    log(f"[bench] oracle levels of {len(roots)} roots in {time.perf_counter() - t:.1f}s "
        f"({checks.threads} threads)")
    for i, r in enumerate(roots):
        checks.submit("single_source", i, r, *fetch(capi, h, r, slots, i, lv, pr))
    if bitmap_leg is not None:
        sl = bitmap_leg.get("_slots")
        if sl is not None and sl.kept:
            for i, r in enumerate(roots):
                checks.submit("frontier_bitmap", i, r, *fetch(capi, h, r, sl, i, lv, pr))
    if direction is not None:
        sl = direction.get("_slots")
        if sl is None or not sl.kept:
            saved = (capi.bfs_graph_get_option(h, capi.BFS_OPT_LOOP),
                     capi.bfs_graph_get_option(h, capi.BFS_OPT_BOTTOM_UP),
                     capi.bfs_graph_get_shape(h, capi.BFS_KERNEL_SINGLE),
                     capi.bfs_graph_get_option(h, capi.BFS_OPT_PERSIST_CTAS))
            restore_options(capi, h, direction["_options"])
        for i, r in enumerate(roots):
            checks.submit("direction_optimizing", i, r, *fetch(capi, h, r, sl, i, lv, pr))
        if sl is None or not sl.kept:
            restore_options(capi, h, saved)
    if batched is not None:
        for leg, key in (("batched", "_slots"), ("batched_bottom_up", "_slots_do")):
            sl = batched.get(key)
            if sl is None:
                continue
            for i in range(sl.lv.shape[0]):
                checks.submit(leg, i, roots[i], sl.lv[i].cpu().numpy(), sl.pr[i].cpu().numpy())
    rep = checks.report()
    log(f"[bench] parity checks done in {time.perf_counter() - t:.1f}s")
    parity = {"legs": rep, "roots_checked": len(roots), "ok": all(v["ok"] for v in rep.values())}
    dims = getattr(args, "grid_dims", None)
    if dims:
        # full-size closed form: level = Manhattan distance on the grid
        X, Y, Z = dims
        ids = np.arange(g.n, dtype=np.int64)
        x, y, z = ids % X, (ids // X) % Y, ids // (X * Y)
        closed_ok, n_closed = True, 0
        for i, r in enumerate(roots[:8]):
            got, _ = fetch(capi, h, r, slots, i, lv, pr)
            rx, ry, rz = int(r) % X, (int(r) // X) % Y, int(r) // (X * Y)
            want = np.abs(x - rx) + np.abs(y - ry) + np.abs(z - rz)
            closed_ok &= bool(np.array_equal(got, want))
            n_closed += 1
        parity["closed_form_roots"] = n_closed
        parity["closed_form_ok"] = closed_ok
        parity["ok"] = parity["ok"] and closed_ok
    return parity


if __name__ == "__main__":
    sys.exit(main())
