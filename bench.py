#!/usr/bin/env python
"""Benchmark of the graph-kNN path: BFS-kNN GTEPS and fraction of HBM peak.

Workload (one step): the full all-pairs form (GUMAP, Algorithm 1: BFS from
every vertex, kNN in (distance, id) order, UMAP weights, fuzzy union, sorted
COO) with k = 15 on two seeded synthetic graphs shaped like the paper's
scale-free and dense inputs: Barabasi-Albert n = 20,000 with 5 edges per new
vertex (seed 1) and G(n = 5,000, p = 0.1) (seed 2). All sources, so both
graphs' complete outputs are produced every step.

Work unit (Graph500 convention, as for the paper's O(nm) analysis of the
all-pairs form): per source, the undirected edges of its connected
component. GTEPS = work / device time.

value: device time (CUDA events on the launching stream) with the graphs
  resident in HBM; L2 is flushed (512 MB write) before every timed step and
  each step is timed on its own.
e2e: the same metric through the public API from pinned host buffers:
  gumap_knn_create (H2D copy + validation), gumap_knn_run, D2H copy of
  idx/dist/w, gumap_knn_destroy, wall-clock per step.
--impl reference: the CPU oracle (test infrastructure) on a bounded sample
  of the same sources, same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

T_START = time.perf_counter()
ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

K_NEIGHBOURS = 15
METRIC = "BFS-kNN GTEPS (full all-pairs form, k=15) and % of HBM peak"
WORKLOAD = ("full-APSP GUMAP kNN + UMAP weights + fuzzy union + sorted COO, k=15, all sources, on "
            "BA n=20000 m0=5 seed 1 and G(n=5000, p=0.1) seed 2")
PARTIAL_METRIC = "BFS-kNN GTEPS (partial form, k=15 and 50) and % of HBM peak"
PARTIAL_WORKLOAD = ("partial-BFS SL-GUMAP kNN + UMAP weights + fuzzy union + sorted COO, all sources, k=15 and "
                    "k=50, on BA n=1000000 m0=4 seed 3 and the 1000x1000 grid")
FLUSH_BYTES = 512 << 20
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "msbfs_kernel_traffic.json")
KERNEL_SRCS = [os.path.join(ROOT, "paper_2509_19703_gb300", "csrc", "msbfs.cu")]


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="bounded oracle sample budget")
    p.add_argument("--only", choices=["ba20k", "er5k", "ba1m-k15", "ba1m-k50", "grid1m-k15", "grid1m-k50"],
                   default=None,
                   help="run one graph of the workload (config2: ba20k, er5k; partial: ba1m-k15 ... grid1m-k50) "
                        "for profiler captures; not a bench line")
    p.add_argument("--engine", choices=["tuned", "msbfs"], default="tuned",
                   help="headline workload: the autotuner's engine (default), or the MS-BFS kernel with the "
                        "autotuner's other settings (for profiler captures, under which the tuner's timings "
                        "are distorted)")
    p.add_argument("--frontier-build", choices=["tuned", "thread", "warp", "group"], default="tuned",
                   help="partial workload: the frontier engine's merge, autotuned (default) or forced "
                        "(for profiler captures)")
    p.add_argument("--workload", choices=["config2", "partial", "batch", "serve"], default="config2",
                   help="config2: the headline line; partial: the partial form on the 1,000,000-vertex "
                        "graphs; batch: the 2000-graph batching comparison; serve: the request-stream "
                        "latency sweep")
    p.add_argument("--batch-graphs", type=int, default=2000)
    p.add_argument("--serve-requests", type=int, default=10000)
    p.add_argument("--serve-n-cap", type=int, default=200000)
    p.add_argument("--serve-rates", type=float, nargs="*", default=[0.25, 0.5, 0.75, 0.9, 1.0, 1.2])
    p.add_argument("--serve-batch-vertices", type=int, default=0,
                   help="server option max_batch_vertices (0: the library's default)")
    p.add_argument("--no-extras", action="store_true",
                   help="headline line only: skip the summaries of the other workloads (config 1, partial form, "
                        "batching, serving, quality metrics, spectral layout)")
    return p.parse_args()


def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(ms: float, world: int, device: str = "cpu") -> float:
    """The step time of the whole job: the slowest rank's (replicas run the
    same step on every GPU; the value counts the work of all ranks)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(work_per_rank: int, world: int, ms: float) -> float:
    """Whole-job GTEPS: every rank's work over the slowest rank's time."""
    return world * work_per_rank / (ms * 1e-3) / 1e9


def build_graphs(only=None):
    from paper_2509_19703_gb300 import graphgen as gg
    makers = {"ba20k": gg.config_ba20k, "er5k": gg.config_er5k}
    return [m() for name, m in makers.items() if only in (None, name)]


def component_work(g):
    """Per-source work of the full form: undirected edges of the source's component."""
    import numpy as np
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    A = sp.csr_matrix((np.ones(g.nnz, dtype=np.int8), g.col, g.row_ptr), shape=(g.n, g.n))
    ncomp, lab = connected_components(A, directed=False)
    edges = np.bincount(np.repeat(lab, np.diff(g.row_ptr)), minlength=ncomp) // 2
    return edges[lab].astype(np.int64)  # per source


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.tmp = None

    def start(self):
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                          "-lms", "50", "-i", str(self.dev)], stdout=self.tmp,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.strip() for r in self.tmp.read().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                smax = max(smax, float(f[2].split()[0]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- helpers

def measured_peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_sha():
    """sha256 of the MS-BFS kernel's source with comments and whitespace
    removed, so an edit of a comment does not void a traffic record taken on
    the same code."""
    code = ""
    for path in KERNEL_SRCS:
        with open(path) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        code += re.sub(r"\s+", "", src)
    return hashlib.sha256(code.encode()).hexdigest()


def recorded_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; otherwise None."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_code_sha256") != kernel_sha():
        return None
    return rec.get("dram_bytes_per_launch")


def recorded_l2():
    """L2 throughput (% of peak) per launch from the committed ncu summary, if
    it was taken on the current kernel source; otherwise None."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_code_sha256") != kernel_sha():
        return None
    return rec.get("l2_throughput_pct_of_peak")


def msbfs_alg_bytes(g, block_bits, level_sum, launches):
    """Algorithmic bytes of the MS-BFS launches: per level the frontier,
    visited and next bitsets once each (3 n S / 8 = 12 n W bytes, W = S / 32)
    plus the CSR once (4 (n + 1) + 4 nnz); per launch the clearing of the
    visited and next bitsets (8 n W bytes). The gathers of neighbour
    frontier rows are served from L2 and are not counted."""
    W = block_bits // 32
    per_level = 12 * g.n * W + 4 * (g.n + 1) + 4 * g.nnz
    return level_sum * per_level + launches * 8 * g.n * W


def partial_work(g, idx, dist):
    """Traversal work of the partial form per source, from its kNN list:
    (adjacency entries scanned, rows expanded). The expanded vertices are the
    source and every vertex closer than D_s, the distance of the list's last
    entry: fewer than k vertices lie closer than D_s, so all of them are in
    the list. A padded list (the component ran out) expands its whole
    component. Sources are 0..n-1 in row order."""
    import numpy as np
    deg = np.diff(g.row_ptr).astype(np.int64)
    d = np.asarray(dist).view(np.uint16) if np.asarray(dist).dtype == np.int16 else np.asarray(dist)
    idx = np.asarray(idx)
    inner = (d < d[:, -1:]) & (idx >= 0)
    listed = np.where(inner, deg[np.where(idx >= 0, idx, 0)], 0).sum(axis=1)
    return deg[: idx.shape[0]] + listed, 1 + inner.sum(axis=1).astype(np.int64)


def frontier_alg_bytes(entries, rows, k):
    """Algorithmic bytes of one frontier-engine launch (partial form, one warp
    per source): per expanded row its two row_ptr words and its adjacency
    (4 bytes per entry), per source the k ids and distances written (6 k)."""
    return int(8 * int(rows.sum()) + 4 * int(entries.sum()) + 6 * k * len(rows))


def coo_alg_bytes(n, k, nnz):
    """Algorithmic bytes of one COO build (gumap_knn_run with union weights):
    every slot's id and weight read once (8 n k), every entry's column and
    weight written once (8 nnz), the row offsets written (8 n)."""
    return 8 * n * k + 8 * nnz + 8 * n


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_union_rows(g, k, mode, rows):
    """The oracle's lists, distances and union weights of the given rows, for
    the CPU-baseline legs' parity figures. Only oracle functions compute: the
    lists of the rows and of every vertex they list, the FP64 weights of
    those lists, and the union weight of each slot of the rows, whose reverse
    weight comes from the target's list (so the targets' rows are enough)."""
    import numpy as np

    import oracle
    knn = oracle.knn_full if mode == "full" else oracle.knn_partial
    rows = np.asarray(rows, dtype=np.int32)
    idx_r, _ = knn(g, k, sources=rows)
    verts = np.unique(np.concatenate([rows, idx_r[idx_r >= 0]])).astype(np.int32)
    idx_v, dist_v = knn(g, k, sources=verts)
    _, _, a_v = oracle.smooth_knn(dist_v)
    pos = np.full(g.n, -1, dtype=np.int32)
    pos[verts] = np.arange(len(verts), dtype=np.int32)
    # compact ids; ids outside `verts` appear only in targets' rows, where no lookup of a row's slot reads them
    idx_c = np.where(idx_v >= 0, pos[np.maximum(idx_v, 0)], -1).astype(np.int32)
    w_c = oracle.slot_union(idx_c, a_v)
    sel = pos[rows]
    return idx_v[sel], dist_v[sel], w_c[sel]


def sampled_parity(g, k, mode, idx, dist, w, rows):
    """Rows of the GPU's output against the oracle's: (rows whose ids or
    distances differ, max |w_gpu - w_oracle|)."""
    import numpy as np
    ri, rd, rw = oracle_union_rows(g, k, mode, rows)
    gi, gd, gw = idx[rows], dist[rows], w[rows].astype(np.float64)
    bad = int(np.sum(np.any(gi != ri, axis=1) | np.any(gd != rd, axis=1)))
    return bad, float(np.max(np.abs(gw - rw))) if rw.size else 0.0


def oracle_sample(graphs, works, budget_s):
    """Time the CPU oracle (full BFS per source, (dist, id) sort, FP64
    weights) on seeded source samples, scaled to the GPU's per-graph time
    share; returns (GTEPS, description)."""
    import numpy as np
    import oracle
    total_work, total_t, parts = 0, 0.0, []
    per_graph = budget_s / len(graphs)
    for g, w in zip(graphs, works):
        rng = np.random.default_rng(1234)
        order = rng.permutation(g.n).astype(np.int32)
        t0 = time.perf_counter()
        done = 0
        chunk = 16
        while done < g.n and time.perf_counter() - t0 < per_graph:
            src = order[done:done + chunk]
            _, dist = oracle.knn_full(g, K_NEIGHBOURS, sources=src)
            oracle.smooth_knn(dist)
            done += len(src)
        dt = time.perf_counter() - t0
        total_work += int(w[order[:done]].sum())
        total_t += dt
        parts.append(f"{done} of {g.n} sources of {g.name}")
    return total_work / total_t / 1e9, "; ".join(parts) + " (seeded random order, 1 thread)", total_t


def _oracle_worker(job):
    """One process of the all-core oracle sample: its share of each graph's
    seeded source order for `budget` seconds per graph. Returns (work,
    busy seconds, sources done per graph)."""
    import oracle
    graphs, works, shares, budget = job
    work, busy, done_per = 0, 0.0, []
    for g, w, src in zip(graphs, works, shares):
        t0 = time.perf_counter()
        done = 0
        while done < len(src) and time.perf_counter() - t0 < budget:
            chunk = src[done:done + 16]
            _, dist = oracle.knn_full(g, K_NEIGHBOURS, sources=chunk)
            oracle.smooth_knn(dist)
            done += len(chunk)
        busy += time.perf_counter() - t0
        work += int(w[src[:done]].sum())
        done_per.append(done)
    return work, busy, done_per


def _oracle_worker_to_queue(job, q):
    try:
        q.put(("ok", _oracle_worker(job)))
    except Exception as e:  # reported to the parent instead of a result
        q.put(("error", f"{type(e).__name__}: {e}"))


def oracle_sample_all_cores(graphs, works, budget_s, procs):
    """The oracle sample of oracle_sample spread over `procs` processes
    (spawned, so no CUDA state is inherited): process p takes every procs-th
    source of the same seeded order. GTEPS = all processes' work / the
    longest busy time. Raises if a process fails or does not report within
    a generous deadline; every process is ended before returning."""
    import multiprocessing as mp
    import queue

    import numpy as np
    orders = [np.random.default_rng(1234).permutation(g.n).astype(np.int32) for g in graphs]
    jobs = [(graphs, works, [o[p::procs] for o in orders], budget_s / len(graphs)) for p in range(procs)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    workers = [ctx.Process(target=_oracle_worker_to_queue, args=(job, q), daemon=True) for job in jobs]
    res = []
    try:
        for w in workers:
            w.start()
        deadline = time.monotonic() + 2 * budget_s + 120.0
        for _ in workers:
            try:
                status, r = q.get(timeout=max(0.1, deadline - time.monotonic()))
            except queue.Empty:
                raise TimeoutError("an oracle process did not report in time") from None
            if status != "ok":
                raise RuntimeError(r)
            res.append(r)
    finally:
        for w in workers:
            w.join(timeout=5)
            if w.is_alive():
                w.terminate()
                w.join(timeout=5)
    work = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    done = [sum(r[2][i] for r in res) for i in range(len(graphs))]
    desc = "; ".join(f"{d} of {g.n} sources of {g.name}" for d, g in zip(done, graphs))
    return work / busy / 1e9, f"{desc} (seeded random order, {procs} processes)"


# ---------------------------------------------------------------- arms

def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    graphs = build_graphs(args.only)
    works = [component_work(g) for g in graphs]
    budget = max(0.2, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    vals, busys = [], []
    desc = ""
    for i in range(args.warmup + args.steps):
        v, desc, busy = oracle_sample(graphs, works, budget)
        if i >= args.warmup:
            vals.append(v)
            busys.append(busy)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(busys) * 1e3,
            "budget_ms_per_step": budget * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32/f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "k": K_NEIGHBOURS},
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": f"each step: {desc}, about {budget:.0f} s"},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


PARTIAL_RUN_NAMES = {"ba1m-k15": (0, 15), "ba1m-k50": (0, 50), "grid1m-k15": (1, 15), "grid1m-k50": (1, 50)}


def partial_runs(only=None):
    from paper_2509_19703_gb300 import graphgen as gg
    if only in PARTIAL_RUN_NAMES:
        which, k = PARTIAL_RUN_NAMES[only]
        return [((gg.config_ba1m, gg.config_grid1m)[which](), k)]
    graphs = [gg.config_ba1m(), gg.config_grid1m()]
    return [(g, k) for g in graphs for k in (15, 50)]


def run_reference_partial(args):
    """The reference arm of the partial workload: the oracle's partial BFS
    (with its own scan count as the work) and FP64 weights on a seeded
    source sample of each (graph, k), one thread."""
    import numpy as np

    import oracle
    rank, _, _ = dist_info()
    if rank != 0:
        return
    runs = partial_runs()
    budget = max(0.2, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    vals, parts, busys = [], [], []
    for i in range(args.warmup + args.steps):
        work, busy, parts = 0, 0.0, []
        for g, k in runs:
            order = np.random.default_rng(1234).permutation(g.n).astype(np.int32)
            done, t0 = 0, time.perf_counter()
            while done < g.n and time.perf_counter() - t0 < budget / len(runs):
                _, dist, w = oracle.knn_partial(g, k, sources=order[done:done + 1024], return_work=True)
                oracle.smooth_knn(dist)
                work += int(w.sum())
                done += len(w)
            busy += time.perf_counter() - t0
            parts.append(f"{done} of {g.n} sources of {g.name} at k={k}")
        if i >= args.warmup:
            vals.append(work / 2 / busy / 1e9)
            busys.append(busy)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": PARTIAL_METRIC, "value": value, "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(busys) * 1e3,
            "budget_ms_per_step": budget * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32/f64", "data": "synthetic",
            "config": {"workload": PARTIAL_WORKLOAD},
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": f"each step: {'; '.join(parts)}, about {budget:.0f} s"},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2509_19703_gb300 import gumap

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    graphs = build_graphs(args.only)
    works = [component_work(g) for g in graphs]
    work_per_step = int(sum(int(w.sum()) for w in works))
    kgs = [gumap.KnnGraph.from_graph(g, K_NEIGHBOURS, mode=gumap.FULL) for g in graphs]
    tuned = [kg.autotune() for kg in kgs]  # engine settings timed on each graph, before any timed step
    if args.engine == "msbfs":
        for kg in kgs:
            kg.set_option(gumap.OPT_ENGINE, gumap.ENGINE_MSBFS)
    for kg in kgs:
        kg.set_option(gumap.OPT_PROFILE, 1)
    outs = [kg.alloc_outputs(g.n) for kg, g in zip(kgs, graphs)]
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        for kg, o in zip(kgs, outs):
            kg.run(out=o)
    for kg in kgs:
        kg.check()
        kg.reset_stats()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for s in range(args.steps):
        flush.fill_(s & 0xFF)
        torch.cuda.nvtx.range_push("timed_step")  # lets a profiler select the timed launches (ncu --nvtx)
        ev[s][0].record(stream)
        for kg, o in zip(kgs, outs):
            kg.run(out=o)
        ev[s][1].record(stream)
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    ms = max_over_ranks(ms, world, device="cuda")
    for kg in kgs:
        kg.check()
    stats = [kg.stats() for kg in kgs]
    value = job_value(work_per_step, world, ms)

    # roofline of the dominant kernel (the MS-BFS launches)
    alg = sum(msbfs_alg_bytes(g, st["block_bits"], st["bfs_level_sum"], st["bfs_launches"])
              for g, st in zip(graphs, stats))
    bfs_ms = sum(st["bfs_ms"] for st in stats)
    launches = sum(st["bfs_launches"] for st in stats)
    peak, peak_kind = measured_peak_gbs()
    achieved = alg / (bfs_ms * 1e-3) / 1e9 if bfs_ms > 0 else 0.0
    traffic = recorded_traffic()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if peak else None,
                "traffic": traffic, "peak_source": peak_kind,
                "l2_throughput_pct_of_peak": recorded_l2(),
                "kernel": "msbfs_kernel", "launches": launches,
                "avg_launch_ms": bfs_ms / launches if launches else None,
                "alg_bytes_per_launch": alg / launches if launches else None,
                "kernel_share_of_step": (bfs_ms / args.steps) / ms if ms else None,
                "phase_ms_per_step": {ph: sum(st[f"bfs_{ph}_ms"] for st in stats) / args.steps
                                      for ph in ("init", "pull", "extract")}}
    gpu_launches = sum(st["kernel_launches"] for st in stats)

    # end to end through the public API from pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        pinned = []
        h2d = d2h = 0
        for g in graphs:
            rp = torch.from_numpy(g.row_ptr).pin_memory()
            col = torch.from_numpy(g.col).pin_memory()
            pinned.append((rp, col))
            h2d += rp.numel() * 4 + col.numel() * 4
        host_out = [dict(idx=torch.empty((g.n, K_NEIGHBOURS), dtype=torch.int32).pin_memory(),
                         dist=torch.empty((g.n, K_NEIGHBOURS), dtype=torch.int16).pin_memory(),
                         w=torch.empty((g.n, K_NEIGHBOURS), dtype=torch.float32).pin_memory()) for g in graphs]
        d2h = sum(o[key].numel() * o[key].element_size() for o in host_out for key in o)
        times = []
        for s in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for g, (rp, col), ho, o in zip(graphs, pinned, host_out, outs):
                drp = rp.to("cuda", non_blocking=True)
                dcol = col.to("cuda", non_blocking=True)
                h = gumap.gumap_knn_create(drp, dcol, g.n, g.nnz, K_NEIGHBOURS, gumap.FULL, gumap.CSR_ON_DEVICE)
                gumap.gumap_knn_run(h, None, g.n, o["idx"], o["dist"], o["w"])
                for key in ("idx", "dist", "w"):
                    ho[key].copy_(o[key], non_blocking=True)
                torch.cuda.synchronize()
                gumap.gumap_knn_destroy(h)
            dt = time.perf_counter() - t0
            if s > 0:
                times.append(dt)
        e2e_t = statistics.median(times)
        e2e = {"value": world * work_per_step / e2e_t / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_t * 1e3, "timing": "wall clock, median"}

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc, _ = oracle_sample(graphs, works, args.cpu_seconds)
        cpu = {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": desc}
        # parity of the timed run's rows on a seeded sample: ids and distances exact, weights vs FP64
        bad, dw = 0, 0.0
        for g, o in zip(graphs, outs):
            rows = np.random.default_rng(4321).choice(g.n, size=min(g.n, 200), replace=False).astype(np.int32)
            b, e = sampled_parity(g, K_NEIGHBOURS, "full", o["idx"].cpu().numpy(), gumap.dist_u16(o["dist"]),
                                  o["w"].cpu().numpy(), rows)
            bad, dw = bad + b, max(dw, e)
        cpu["parity"] = {"rows_checked": sum(min(g.n, 200) for g in graphs), "rows_differing": bad,
                         "max_abs_dw": dw}
        procs = min(cpu_cores(), 64)
        if procs > 1:
            try:
                v, desc = oracle_sample_all_cores(graphs, works, args.cpu_seconds / 2, procs)
                cpu_all = {"value": v, "unit": "GTEPS", "cores": procs, "kind": "oracle", "sample": desc}
            except Exception as e:  # a reported baseline only: never lose the bench line over it
                cpu_all = {"unavailable": f"{type(e).__name__}: {e}"}

    for kg in kgs:
        kg.close()
    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras = run_extras(args)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32 bitsets / f32 weights", "data": "synthetic",
                "config": {"workload": WORKLOAD, "k": K_NEIGHBOURS,
                           "graphs": [{"name": g.name, "n": g.n, "m": g.m} for g in graphs],
                           "work_edges_per_step": work_per_step, "parallelism": f"replicas x{world}",
                           "l2": "flushed (512 MB write) before each timed step",
                           "block_bits": [st["block_bits"] for st in stats],
                           "levels_max": [st["levels_max"] for st in stats],
                           "autotuned": [{key: t[key] for key in ("engine", "state_bytes", "pull_width", "heavy_mult",
                                                                   "ctas_per_sm", "stage", "direction", "best_ms",
                                                                   "default_ms")}
                                         for t in tuned]},
                "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "e2e": e2e,
                "gpu_launches": gpu_launches, "clocks": clocks}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batch_workload(args, emit=True):
    """Batching (the 2000-graph mix, k = 15): graphs/s of one persistent
    launch per step (gumap_batch_create) against one handle and one run per
    graph on the same GPU and stream. Returns its JSON line (printed when
    emit)."""
    import torch

    from paper_2509_19703_gb300 import graphgen as gg
    from paper_2509_19703_gb300 import gumap

    torch.cuda.set_device(0)
    items = gg.batch_mix(count=args.batch_graphs, base_seed=4)
    graphs = [it.graph for it in items]
    modes = [gumap.FULL if it.mode == "full" else gumap.PARTIAL for it in items]
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def timed(fn, steps):
        ts = []
        for s in range(steps):
            flush.fill_(s & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    kb, offs = gumap.KnnGraph.batch(graphs, K_NEIGHBOURS, modes)
    tuned = kb.autotune()  # the widest unit (source-block width), timed before any timed step
    kb.set_option(gumap.OPT_PROFILE, 1)
    out = kb.alloc_outputs(kb.n)
    for _ in range(args.warmup):
        kb.run(out=out)
    kb.check()
    kb.reset_stats()
    ms_batch = timed(lambda: kb.run(out=out), args.steps)
    st = kb.stats()
    kb.check()
    kb.close()
    # roofline of the batched engine: its units' bytes on the per-level model of
    # the bit-parallel BFS (the bitset rows live in shared memory here) over its
    # own launch time
    peak, peak_kind = measured_peak_gbs()
    bfs_ms = st["bfs_ms"] / max(1, st["bfs_launches"])
    model = st["batch_model_bytes"] / max(1, st["bfs_launches"])
    achieved = model / (bfs_ms * 1e-3) / 1e9 if bfs_ms > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if peak else None, "traffic": None, "peak_source": peak_kind,
                "kernel": "batch_kernel", "avg_launch_ms": bfs_ms, "model_bytes_per_launch": model,
                "kernel_share_of_step": bfs_ms / ms_batch if ms_batch else None,
                "model": "per unit and level 12 n W (frontier, visited, next rows; shared memory here) + the "
                         "graph's CSR 4 (n + 1) + 4 nnz"}
    parity, cpu = None, None
    if not args.no_cpu_baseline:  # a seeded sample of the graphs against the oracle (all rows of each)
        import numpy as np

        import oracle
        idx = out["idx"].cpu().numpy()
        dist = gumap.dist_u16(out["dist"])
        w = out["w"].cpu().numpy().astype(np.float64)
        small = [i for i, g in enumerate(graphs) if g.n <= 6000]  # graphs the oracle finishes in about a second
        pick = np.random.default_rng(44).choice(small, size=min(len(small), 40), replace=False)
        bad, dw, busy = 0, 0.0, 0.0
        for gi in pick:
            g, m = graphs[gi], items[gi].mode
            t0 = time.perf_counter()
            ref = oracle.knn_pipeline(g, K_NEIGHBOURS, m)
            busy += time.perf_counter() - t0
            lo, hi = int(offs[gi]), int(offs[gi + 1])
            li = np.where(idx[lo:hi] >= 0, idx[lo:hi] - lo, -1)
            bad += int(np.sum(np.any(li != ref["idx"], axis=1) | np.any(dist[lo:hi] != ref["dist"], axis=1)))
            dw = max(dw, float(np.max(np.abs(w[lo:hi] - ref["w"]))))
        parity = {"graphs_checked": len(pick), "rows_differing": bad, "max_abs_dw": dw}
        cpu = {"value": len(pick) / busy, "unit": "graphs/s", "cores": 1, "kind": "oracle",
               "sample": f"{len(pick)} seeded graphs of the mix with n <= 6000, every source (1 thread)"}

    singles = [gumap.KnnGraph.from_graph(g, K_NEIGHBOURS, mode=m) for g, m in zip(graphs, modes)]
    souts = [s.alloc_outputs(g.n) for s, g in zip(singles, graphs)]

    def run_all():
        for s, o in zip(singles, souts):
            s.run(out=o)

    for _ in range(max(1, args.warmup // 2)):
        run_all()
    ms_single = timed(run_all, max(1, min(args.steps, 5)))
    for s in singles:
        s.check()
        s.close()
    n_total = sum(g.n for g in graphs)
    line = {"metric": "batched graphs/s (2000-graph mix, k=15) vs one launch per graph",
            "value": len(graphs) / (ms_batch * 1e-3), "unit": "graphs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_batch, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32 bitsets / f32 weights", "data": "synthetic",
            "config": {"workload": "config 4: 2000 seeded graphs, n log-uniform in [100, 20000], grid / BA 2..8 / "
                                   "G(n,p) mean degree 4..40 / random tree, full or partial 50/50, k=15",
                       "graphs": len(graphs), "vertices": n_total, "units": st["n_blocks"],
                       "autotuned": {key: tuned[key] for key in ("batch_width", "best_ms", "default_ms")},
                       "l2": "flushed (512 MB write) before each timed step"},
            "one_launch_per_graph": {"graphs_per_s": len(graphs) / (ms_single * 1e-3), "ms_per_step": ms_single},
            "speedup_vs_one_launch_per_graph": ms_single / ms_batch,
            "roofline": roofline, "parity": parity, "cpu_baseline": cpu,
            "gpu_launches": st["kernel_launches"]}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_partial_workload(args, emit=True):
    """Partial form (SL-GUMAP, Algorithm 4) on the two 1,000,000-vertex
    graphs at k = 15 and k = 50: one step runs gumap_knn_run (kNN lists,
    weights, union, sorted COO, all sources) for each (graph, k). Work per
    source: the adjacency entries of the vertices it expands (closer than
    the distance of its k-th neighbour) / 2, counted from the lists.
    Returns its JSON line (printed when emit)."""
    import numpy as np
    import torch

    from paper_2509_19703_gb300 import gumap

    torch.cuda.set_device(0)
    runs = partial_runs(args.only)
    graphs = []
    for g, _ in runs:
        if not any(g is h for h in graphs):
            graphs.append(g)
    kgs = [gumap.KnnGraph.from_graph(g, k, mode=gumap.PARTIAL) for g, k in runs]
    if args.frontier_build == "tuned":
        tuned = [kg.autotune() for kg in kgs]
    else:  # a forced merge build, for profiler captures: no tuning runs
        build = {"thread": gumap.FRONTIER_THREAD, "warp": gumap.FRONTIER_WARP,
                 "group": gumap.FRONTIER_GROUP}[args.frontier_build]
        for kg in kgs:
            kg.set_option(gumap.OPT_ENGINE, gumap.ENGINE_FRONTIER)
            kg.set_option(gumap.OPT_FRONTIER_BUILD, build)
        tuned = [{"engine": gumap.ENGINE_FRONTIER, "state_bytes": 0, "frontier_build": build, "best_ms": None,
                  "default_ms": None} for _ in kgs]
    for kg in kgs:
        kg.set_option(gumap.OPT_PROFILE, 1)
    outs = [kg.alloc_outputs(g.n) for kg, (g, _) in zip(kgs, runs)]
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        for kg, o in zip(kgs, outs):
            kg.run(out=o)
    for kg in kgs:
        kg.check()
        kg.reset_stats()
    torch.cuda.synchronize()

    sampler = ClockSampler(0)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for s in range(args.steps):
        flush.fill_(s & 0xFF)
        torch.cuda.nvtx.range_push("timed_step")
        ev[s][0].record(stream)
        for kg, o in zip(kgs, outs):
            kg.run(out=o)
        ev[s][1].record(stream)
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    for kg in kgs:
        kg.check()
    stats = [kg.stats() for kg in kgs]

    # work and algorithmic bytes from the lists (identical every step)
    per_run = []
    for (g, k), o, st, kg in zip(runs, outs, stats, kgs):
        entries, rows = partial_work(g, o["idx"].cpu().numpy(), gumap.dist_u16(o["dist"]))
        nnz = int(kg.coo()[0].numel())
        engine_bytes = (frontier_alg_bytes(entries, rows, k) if st["engine"] == gumap.ENGINE_FRONTIER
                        else msbfs_alg_bytes(g, st["block_bits"], st["bfs_level_sum"] // args.steps,
                                             st["bfs_launches"] // args.steps))
        per_run.append({"graph": g.name, "n": g.n, "m": g.m, "k": k, "engine": st["engine"],
                        "work_edges": int(entries.sum()) // 2, "entries": entries, "rows": rows,
                        "coo_nnz": nnz, "engine_alg_bytes": engine_bytes, "coo_alg_bytes": coo_alg_bytes(g.n, k, nnz),
                        "engine_ms": st["bfs_ms"] / args.steps, "weights_ms": st["weights_ms"] / args.steps,
                        "coo_ms": st["sort_ms"] / args.steps,
                        "engine_launches": st["bfs_launches"] // args.steps,
                        "coo_launches": st["sort_launches"] // args.steps})
    work_per_step = sum(r["work_edges"] for r in per_run)
    value = work_per_step / (ms * 1e-3) / 1e9
    stage_ms = {key: sum(r[key] for r in per_run) for key in ("engine_ms", "weights_ms", "coo_ms")}

    # roofline of the BFS engine (the partial BFS of Algorithm 4); the other
    # stages' model fractions beside it
    peak, peak_kind = measured_peak_gbs()
    t_ms = stage_ms["engine_ms"]
    alg = sum(r["engine_alg_bytes"] for r in per_run)
    launches = sum(r["engine_launches"] for r in per_run)
    achieved = alg / (t_ms * 1e-3) / 1e9 if t_ms > 0 else 0.0
    coo_alg = sum(r["coo_alg_bytes"] for r in per_run)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if peak else None, "traffic": None, "peak_source": peak_kind,
                "kernel": "BFS engine (frontier kernels, merge build per graph by the autotuner)",
                "launches_per_step": launches, "alg_bytes_per_step": alg,
                "avg_launch_ms": t_ms / launches if launches else None,
                "kernel_share_of_step": t_ms / ms if ms else None,
                "stage_ms_per_step": stage_ms,
                "coo_stage": {"alg_bytes_per_step": coo_alg,
                              "achieved_gbs": coo_alg / (stage_ms["coo_ms"] * 1e-3) / 1e9 if stage_ms["coo_ms"] else None}}
    gpu_launches = sum(st["kernel_launches"] for st in stats)

    e2e = None
    if args.e2e_steps > 0:
        pinned = {}
        for g in graphs:
            pinned[g.name] = (torch.from_numpy(g.row_ptr).pin_memory(), torch.from_numpy(g.col).pin_memory())
        host_out = [dict(idx=torch.empty((g.n, k), dtype=torch.int32).pin_memory(),
                         dist=torch.empty((g.n, k), dtype=torch.int16).pin_memory(),
                         w=torch.empty((g.n, k), dtype=torch.float32).pin_memory()) for g, k in runs]
        h2d = sum(pinned[g.name][0].numel() * 4 + pinned[g.name][1].numel() * 4 for g, _ in runs)
        d2h = sum(o[key].numel() * o[key].element_size() for o in host_out for key in o)
        times = []
        for s in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for (g, k), ho, o in zip(runs, host_out, outs):
                rp, col = pinned[g.name]
                drp = rp.to("cuda", non_blocking=True)
                dcol = col.to("cuda", non_blocking=True)
                h = gumap.gumap_knn_create(drp, dcol, g.n, g.nnz, k, gumap.PARTIAL, gumap.CSR_ON_DEVICE)
                gumap.gumap_knn_run(h, None, g.n, o["idx"], o["dist"], o["w"])
                for key in ("idx", "dist", "w"):
                    ho[key].copy_(o[key], non_blocking=True)
                torch.cuda.synchronize()
                gumap.gumap_knn_destroy(h)
            if s > 0:
                times.append(time.perf_counter() - t0)
        e2e_t = statistics.median(times)
        e2e = {"value": work_per_step / e2e_t / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_t * 1e3, "timing": "wall clock, median"}

    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        total_work, total_t, parts = 0, 0.0, []
        for r, (g, k) in zip(per_run, runs):
            order = np.random.default_rng(1234).permutation(g.n).astype(np.int32)
            done, t0 = 0, time.perf_counter()
            while done < g.n and time.perf_counter() - t0 < args.cpu_seconds / len(runs):
                src = order[done:done + 4096]
                _, dist, work = oracle.knn_partial(g, k, sources=src, return_work=True)
                oracle.smooth_knn(dist)
                if not np.array_equal(work, r["entries"][src]):
                    raise RuntimeError(f"{g.name} k={k}: work counted from the lists differs from the oracle's")
                total_work += int(work.sum())
                done += len(src)
            total_t += time.perf_counter() - t0
            parts.append(f"{done} of {g.n} sources of {g.name} at k={k}")
        cpu = {"value": total_work / 2 / total_t / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
               "sample": "; ".join(parts) + " (seeded random order, partial BFS + FP64 weights, 1 thread)"}
        # parity of the timed runs' rows on a seeded sample of each (graph, k)
        bad, dw, checked = 0, 0.0, 0
        for (g, k), o in zip(runs, outs):
            rows = np.random.default_rng(4322).choice(g.n, size=200, replace=False).astype(np.int32)
            b, e = sampled_parity(g, k, "partial", o["idx"].cpu().numpy(), gumap.dist_u16(o["dist"]),
                                  o["w"].cpu().numpy(), rows)
            bad, dw, checked = bad + b, max(dw, e), checked + len(rows)
        cpu["parity"] = {"rows_checked": checked, "rows_differing": bad, "max_abs_dw": dw}

    for r in per_run:
        r.pop("entries")
        r.pop("rows")
    line = {"metric": PARTIAL_METRIC, "value": value,
            "unit": "GTEPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32 ids / u16 distances / f32 weights", "data": "synthetic",
            "config": {"workload": PARTIAL_WORKLOAD,
                       "work_edges_per_step": work_per_step, "runs": per_run,
                       "l2": "flushed (512 MB write) before each timed step",
                       "autotuned": [{key: t[key] for key in ("engine", "state_bytes", "frontier_build", "best_ms",
                                                               "default_ms")}
                                     for t in tuned]},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
            "clocks": clocks}
    if emit:
        print(json.dumps(line), flush=True)
    for kg in kgs:
        kg.close()
    return line


def serve_requests(count, seed, n_cap):
    """Config 5 request stream: n lognormal (median 5000, sigma_ln 1.0) clamped
    to [64, n_cap]; BA (4 edges per vertex) / grid / G(n, p) (mean degree 10)
    in thirds; 70 % partial, 30 % full; k uniform in {15, 30}."""
    import math

    from paper_2509_19703_gb300 import graphgen as gg
    u = gg.uniform(seed, 5 * count)
    out = []
    for i in range(count):
        u1, u2, u3, u4, u5 = u[5 * i:5 * i + 5]
        z = math.sqrt(-2.0 * math.log(max(u1, 1e-300))) * math.cos(2.0 * math.pi * u2)  # Box-Muller
        n = int(min(max(5000.0 * math.exp(z), 64), n_cap))
        kind = min(int(u3 * 3), 2)
        s = seed * 10**6 + i
        if kind == 0:
            g = gg.barabasi_albert(n, 4, s)
        elif kind == 1:
            w = max(2, int(round(math.sqrt(n))))
            g = gg.grid(w, max(2, int(round(n / w))))
        else:
            g = gg.gnp(n, min(1.0, 10.0 / n), s)
        k = 15 if u4 < 0.5 else 30
        out.append((g, min(k, g.n - 1), 1 if u5 < 0.7 else 0))  # 1 = partial
    return out


def run_serve_workload(args, emit=True):
    """Serving: a Poisson stream of config-5 requests through gumap_server_*;
    saturated graphs/s, then p50/p99 latency (submit to completion, server
    clock) at offered rates around saturation, overall and per request class
    (graphs that a batched launch takes, n <= 27,000, or larger ones that run
    alone; partial or full form); against the same requests run one handle at
    a time. A seeded sample of the saturated run's results is read back and
    compared with the oracle. Returns its JSON line (printed when emit)."""
    import numpy as np
    import torch

    from paper_2509_19703_gb300 import gumap

    torch.cuda.set_device(0)
    t_stage = [time.perf_counter()]

    def stage(name):
        t = time.perf_counter()
        print(f"[bench] serve {name}: {t - t_stage[0]:.1f} s", file=sys.stderr, flush=True)
        t_stage[0] = t

    reqs = serve_requests(args.serve_requests, 5, args.serve_n_cap)
    stage("requests generated")
    budget = 64 << 30
    small_n = 27000

    def cls(g, m):
        return ("small" if g.n <= small_n else "large") + ("_partial" if m == gumap.PARTIAL else "_full")

    def pct(x, q):
        return float(np.percentile(np.asarray(x), q) * 1e3) if len(x) else None

    def run_stream(rate, sub, check=()):
        """Submit `sub` with Poisson gaps at `rate` (0: all at once), taking
        every finished result back (and releasing it) while submitting, as a
        client does; latency is submit to completion on the server clock."""
        tc = [time.perf_counter()]
        marks = []

        def mark(name):
            t = time.perf_counter()
            marks.append(f"{name} {t - tc[0]:.1f}")
            tc[0] = t

        s = gumap.gumap_server_create(0, budget, max_batch_vertices=args.serve_batch_vertices)
        mark("create")
        rng = np.random.default_rng(55)
        gaps = rng.exponential(1.0 / rate, size=len(sub)) if rate else np.zeros(len(sub))
        lat, t_first, t_last, batched = [], None, 0.0, []
        by_cls = {}
        rows = {}
        pending = {}

        def take(i, rid, r):
            nonlocal t_first, t_last
            lat.append(r["t_done"] - r["t_submit"])
            by_cls.setdefault(cls(sub[i][0], sub[i][2]), []).append(r["t_done"] - r["t_submit"])
            t_first = r["t_submit"] if t_first is None else min(t_first, r["t_submit"])
            t_last = max(t_last, r["t_done"])
            batched.append(r["batch_graphs"])
            if i in check:
                g, k, _ = sub[i]
                o = dict(idx=torch.empty((g.n, k), dtype=torch.int32, device="cuda"),
                         dist=torch.empty((g.n, k), dtype=torch.int16, device="cuda"),
                         w=torch.empty((g.n, k), dtype=torch.float32, device="cuda"))
                gumap.gumap_serve_read(s, rid, o["idx"], o["dist"], o["w"])
                torch.cuda.synchronize()
                rows[i] = (o["idx"].cpu().numpy(), gumap.dist_u16(o["dist"]), o["w"].cpu().numpy())
            gumap.gumap_serve_release(s, rid)

        cursor = [0]

        def drain():
            # poll a round-robin slice of the pending requests (bounded work per call)
            keys = list(pending)
            if not keys:
                return
            start = cursor[0] % len(keys)
            for i in (keys[start:] + keys[:start])[:32]:
                st, r = gumap.gumap_serve_poll(s, pending[i])
                if st == gumap.PENDING:
                    continue
                assert st == gumap.OK, gumap.gumap_status_string(st)
                take(i, pending.pop(i), r)
            cursor[0] = start + 32

        t_next = time.perf_counter()
        for i, ((g, k, m), gap) in enumerate(zip(sub, gaps)):
            t_next += gap
            while time.perf_counter() < t_next:
                drain()
            while True:
                try:
                    pending[i] = gumap.gumap_serve_submit(s, g.row_ptr, g.col, g.n, g.nnz, k, m)
                    break
                except gumap.GumapError as e:
                    if e.status != gumap.ERR_AGAIN:
                        raise
                    drain()
        mark("submit")
        for i in list(pending):
            st, r = gumap.gumap_serve_wait(s, pending[i], 600.0)
            assert st == gumap.OK, gumap.gumap_status_string(st)
            take(i, pending.pop(i), r)
        mark("wait")
        stats = gumap.gumap_server_get_stats(s)
        gumap.gumap_server_destroy(s)
        mark("destroy")
        print(f"[bench] serve stream rate {rate:.1f}/s: " + ", ".join(marks) + " s", file=sys.stderr, flush=True)
        res = {"graphs_per_s": len(lat) / (t_last - t_first), "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
               "launches": stats["launches"], "mean_graphs_per_launch": float(np.mean(batched)),
               "arena_peak_gb": stats["arena_peak_bytes"] / 2**30,
               "by_class": {c: {"requests": len(v), "p50_ms": pct(v, 50), "p99_ms": pct(v, 99)}
                            for c, v in sorted(by_cls.items())}}
        return res, rows

    run_stream(0, reqs[:500])  # warm-up (module loading, allocator)
    stage("warm-up stream")
    check = set()
    if not args.no_cpu_baseline:  # a seeded sample of graphs small enough for the oracle's full BFS
        cand = [i for i, (g, _, _) in enumerate(reqs) if g.n <= 3000]
        check = set(int(i) for i in np.random.default_rng(56).choice(cand, size=min(len(cand), 40), replace=False))
    sat, rows = run_stream(0, reqs, check)
    stage("saturated stream")
    points = []
    for frac in args.serve_rates:
        p, _ = run_stream(frac * sat["graphs_per_s"], reqs)
        p["offered_rate_frac"] = frac
        points.append(p)
        stage(f"stream at {frac} of saturation")
    parity = None
    if check:
        import oracle
        bad, dw = 0, 0.0
        for i, (gi, gd, gw) in rows.items():
            g, k, m = reqs[i]
            ref = oracle.knn_pipeline(g, k, "partial" if m == gumap.PARTIAL else "full")
            bad += int(np.sum(np.any(gi != ref["idx"], axis=1) | np.any(gd != ref["dist"], axis=1)))
            dw = max(dw, float(np.max(np.abs(gw.astype(np.float64) - ref["w"]))))
        parity = {"requests_checked": len(rows), "rows_differing": bad, "max_abs_dw": dw}
    stage("oracle parity")

    # baseline: the same requests, one handle and one synchronous run each;
    # each one's time alone gives the service time of its class
    t0 = time.perf_counter()
    alone = {}
    for g, k, m in reqs:
        t1 = time.perf_counter()
        with gumap.KnnGraph.from_graph(g, k, mode=m) as kg:
            kg.run()
            kg.check()
        alone.setdefault(cls(g, m), []).append(time.perf_counter() - t1)
    single = len(reqs) / (time.perf_counter() - t0)
    stage("one handle per request")
    alone_ms = {c: {"p50_ms": pct(v, 50), "p99_ms": pct(v, 99), "max_ms": max(v) * 1e3}
                for c, v in sorted(alone.items())}
    classes = {}
    for g, _, m in reqs:
        classes[cls(g, m)] = classes.get(cls(g, m), 0) + 1
    line = {"metric": "served graphs/s with p50/p99 latency (config-5 request stream)",
            "value": sat["graphs_per_s"], "unit": "graphs/s", "n_gpus": 1, "steps": len(reqs), "warmup": 1,
            "ms_per_step": 1e3 / sat["graphs_per_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32 bitsets / f32 weights", "data": "synthetic",
            "config": {"workload": "config 5: Poisson stream, n lognormal median 5000 sigma_ln 1.0 clamped "
                                   f"[64, {args.serve_n_cap}], BA/grid/G(n,p) thirds, 70% partial / 30% full, "
                                   "k in {15, 30}, 64 GiB budget", "requests": len(reqs),
                       "max_batch_vertices": args.serve_batch_vertices or "library default",
                       "vertices": int(sum(g.n for g, _, _ in reqs)), "classes": classes},
            "saturated": sat, "latency_sweep": points, "parity": parity,
            "one_handle_per_request_graphs_per_s": single, "alone_ms_by_class": alone_ms,
            "speedup_vs_one_handle_per_request": sat["graphs_per_s"] / single}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def event_ms(fn, reps=20, warm=3):
    """Median device time of fn() on the current stream (CUDA events)."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def config1_summary(args):
    """Config 1: the 32 x 32 grid, full form, k = 15, every source, weights,
    union and COO through gumap_knn_run, after the autotuner; the default
    engine beside it; every row against the oracle."""
    import numpy as np

    from paper_2509_19703_gb300 import graphgen as gg
    from paper_2509_19703_gb300 import gumap
    g = gg.grid(32, 32)
    kg = gumap.KnnGraph.from_graph(g, K_NEIGHBOURS, mode=gumap.FULL)
    out = kg.alloc_outputs(g.n)
    default_ms = event_ms(lambda: kg.run(out=out))
    tuned = kg.autotune()
    ms = event_ms(lambda: kg.run(out=out), reps=50)
    kg.check()
    res = {"workload": "grid 32x32 (n=1024, m=1984), full form, k=15, all sources, weights + union + sorted COO",
           "ms_per_run": ms, "default_engine_ms_per_run": default_ms,
           "gteps": 1024 * 1984 / (ms * 1e-3) / 1e9,
           "autotuned": {key: tuned[key] for key in ("engine", "batch_width", "best_ms")}}
    # the same runs replayed from a captured CUDA graph (GUMAP_OPT_GRAPH, on a
    # stream of their own); the parity check below reads a replayed run's rows
    try:
        import torch
        side = torch.cuda.Stream()
        kg.set_option(gumap.OPT_GRAPH, 1)
        with torch.cuda.stream(side):
            graph_ms = event_ms(lambda: kg.run(out=out), reps=50)
        torch.cuda.synchronize()
        kg.check()
        res["graph_replay"] = {"ms_per_run": graph_ms, "replays": kg.stats()["graph_replays"]}
    except Exception as e:  # reported, not fatal: the line above stands without it
        res["graph_replay"] = {"error": str(e)[:200]}
    if not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        ref = oracle.knn_pipeline(g, K_NEIGHBOURS, "full")
        busy = time.perf_counter() - t0
        res["cpu_baseline"] = {"ms_per_run": busy * 1e3, "gteps": 1024 * 1984 / busy / 1e9, "cores": 1,
                               "kind": "oracle", "sample": "the whole graph, every source (1 thread)"}
        idx, dist = out["idx"].cpu().numpy(), gumap.dist_u16(out["dist"])
        res["parity"] = {"rows_checked": g.n,
                         "rows_differing": int(np.sum(np.any(idx != ref["idx"], axis=1) |
                                                      np.any(dist != ref["dist"], axis=1))),
                         "max_abs_dw": float(np.max(np.abs(out["w"].cpu().numpy().astype(np.float64) - ref["w"])))}
    kg.close()
    return res


def quality_summary(args):
    """Quality metrics (Section 4.1.3) of a seeded drawing of each headline
    graph: neighbourhood preservation (r = 2) and stress, device time; the
    oracle on a seeded sample of vertices, timed, and compared."""
    import numpy as np
    import torch

    from paper_2509_19703_gb300 import gumap
    res = {}
    for g in build_graphs(None):
        X = np.random.default_rng(9).standard_normal((g.n, 2)).astype(np.float32)
        Xd = torch.as_tensor(X, device="cuda")
        kg = gumap.KnnGraph.from_graph(g, K_NEIGHBOURS, mode=gumap.FULL)
        got = {}

        def np_run():
            got["np"] = kg.quality_np(Xd, 2)

        def st_run():
            got["st"] = kg.quality_stress(Xd)

        np_ms = event_ms(np_run, reps=5, warm=1)
        st_ms = event_ms(st_run, reps=5, warm=1)
        kg.check()
        r = {"n": g.n, "np_ms": np_ms, "np_vertices_per_s": g.n / (np_ms * 1e-3),
             "np": float(got["np"][2].item()), "stress_ms": st_ms,
             "stress_pairs_per_s": g.n * (g.n - 1) / (st_ms * 1e-3), "stress": float(got["st"][0].item())}
        if not args.no_cpu_baseline:
            import oracle
            sample = np.random.default_rng(10).choice(g.n, size=20, replace=False).astype(np.int32)
            t0 = time.perf_counter()
            rc, ri, _ = oracle.np_metric(g, X, 2, vertices=sample)
            t_np = time.perf_counter() - t0
            t0 = time.perf_counter()
            _, rr = oracle.stress(g, X, vertices=sample)
            t_st = time.perf_counter() - t0
            c, inter = got["np"][0].cpu().numpy(), got["np"][1].cpu().numpy()
            rows = got["st"][1].cpu().numpy()
            r["cpu_baseline"] = {"kind": "oracle", "cores": 1, "sample": f"{len(sample)} seeded vertices",
                                 "np_vertices_per_s": len(sample) / t_np,
                                 "stress_pairs_per_s": len(sample) * (g.n - 1) / t_st}
            r["parity"] = {"np_counts_equal": bool(np.array_equal(c[sample], rc) and np.array_equal(inter[sample], ri)),
                           "stress_rows_max_rel_err": float(np.max(np.abs(rows[sample] - rr) / np.abs(rr)))}
        res[g.name] = r
        kg.close()
    return res


def spectral_summary(args):
    """Spectral layout (2 coordinates) of the headline graphs' union kNN
    graphs after a full-form run: device time, Lanczos steps, residual; the
    oracle's dense eigensolve timed on a smaller union graph (grid 40 x 40),
    where both are compared."""
    import numpy as np
    import torch

    from paper_2509_19703_gb300 import graphgen as gg
    from paper_2509_19703_gb300 import gumap
    res = {}
    for g in build_graphs(None) + [gg.grid(40, 40)]:
        kg = gumap.KnnGraph.from_graph(g, K_NEIGHBOURS, mode=gumap.FULL)
        kg.run()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        X, mu, info = kg.spectral_layout(2)
        ms = (time.perf_counter() - t0) * 1e3
        r = {"n": g.n, "ms": ms, "mu": mu.tolist(), **info}
        if g.n <= 2000 and not args.no_cpu_baseline:
            from oracle import spectral
            row, col, w = kg.coo()
            row, col, w = row.cpu().numpy(), col.cpu().numpy(), w.cpu().numpy().astype(np.float64)
            t0 = time.perf_counter()
            Xr, mur = spectral.spectral_layout(g.n, row, col, w, 2)
            r["cpu_baseline"] = {"kind": "oracle", "cores": 1, "ms": (time.perf_counter() - t0) * 1e3,
                                 "sample": "the whole graph (dense FP64 eigensolve)"}
            Xg = X.cpu().numpy().astype(np.float64)
            r["parity"] = {"max_abs_dmu": float(np.max(np.abs(mu - mur))),
                           "max_abs_dx_up_to_sign": float(max(min(np.max(np.abs(Xg[:, c] - Xr[:, c])),
                                                                  np.max(np.abs(Xg[:, c] + Xr[:, c])))
                                                              for c in range(2)))}
        res[g.name] = r
        kg.close()
    return res


def summary_of(line, keys):
    return {key: line.get(key) for key in keys}


def run_extras(args):
    """Summaries of the other workloads for the headline line (each also has
    its own --workload line): config 1, the partial form (config 3), batching
    (config 4), serving (config 5), the quality metrics and the spectral
    layout."""
    import copy
    out = {}
    wall = {"headline": round(time.perf_counter() - T_START, 1)}
    print(f"[bench] headline: {wall['headline']:.1f} s", file=sys.stderr, flush=True)
    t0 = time.perf_counter()

    def lap(name):
        nonlocal t0
        t1 = time.perf_counter()
        wall[name] = round(t1 - t0, 1)
        print(f"[bench] {name}: {t1 - t0:.1f} s", file=sys.stderr, flush=True)
        t0 = t1

    out["config1"] = config1_summary(args)
    lap("config1")
    pa = copy.copy(args)
    pa.steps, pa.warmup, pa.e2e_steps, pa.cpu_seconds, pa.only, pa.frontier_build = 10, 3, 2, 4.0, None, "tuned"
    line = run_partial_workload(pa, emit=False)
    out["partial_form"] = summary_of(line, ("metric", "value", "unit", "ms_per_step", "roofline", "cpu_baseline",
                                            "e2e", "gpu_launches", "clocks"))
    out["partial_form"]["stage_ms_per_step"] = line["roofline"]["stage_ms_per_step"]
    lap("partial_form")
    ba = copy.copy(args)
    ba.steps, ba.warmup, ba.batch_graphs = 3, 1, 2000
    line = run_batch_workload(ba, emit=False)
    out["batched"] = summary_of(line, ("metric", "value", "unit", "ms_per_step", "one_launch_per_graph",
                                       "speedup_vs_one_launch_per_graph", "roofline", "parity", "cpu_baseline",
                                       "gpu_launches"))
    lap("batched")
    sa = copy.copy(args)
    # a shorter stream keeps the default run within minutes (the 10,000-request
    # stream with its six rates is `--workload serve`)
    sa.serve_requests = min(args.serve_requests, 3000)
    sa.serve_rates = [0.25, 0.5, 0.9]
    line = run_serve_workload(sa, emit=False)
    out["served"] = summary_of(line, ("metric", "value", "unit", "saturated", "latency_sweep", "parity",
                                      "one_handle_per_request_graphs_per_s", "speedup_vs_one_handle_per_request",
                                      "alone_ms_by_class"))
    out["served"]["requests"] = line["config"]["requests"]
    lap("served")
    out["quality_metrics"] = quality_summary(args)
    lap("quality_metrics")
    out["spectral_layout"] = spectral_summary(args)
    lap("spectral_layout")
    out["wall_s"] = wall
    return out


def main():
    args = parse_args()
    if args.impl == "reference" and args.workload in ("batch", "serve"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the full-form and partial-form "
                                                              "workloads; batch and serve compare against one launch "
                                                              "per graph on the GPU instead"}), flush=True)
    elif args.impl == "reference" and args.workload == "partial":
        run_reference_partial(args)
    elif args.workload == "serve":
        run_serve_workload(args)
    elif args.workload == "partial":
        run_partial_workload(args)
    elif args.workload == "batch":
        run_batch_workload(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
