"""Benchmark: SlimSell BFS-SpMV on one GB300 (GTEPS and fraction of HBM roofline).

Workload (default): undirected Kronecker graph, scale 22, edgefactor 16,
initiator (0.57, 0.19, 0.19, 0.05), cleaned and label-permuted (seed 1); 64
seeded roots run one at a time for each of the four semirings (tropical, real
with fp32 values, boolean, sel-max); C = 32, sigma = n, SlimWork on, SlimChunk
width 1024; every run produces int32 distances and parents (DP for the
non-sel-max semirings).  A step is all 256 runs.

Prints ONE JSON line.  `--impl reference` times the CPU oracle (the plain CSR
semiring BFS) on the host cores instead, on a bounded sample of the same
workload.  Under torchrun every rank runs its own 64 roots (weak scaling, no
data-path collective; the graph is replicated).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402

METRIC = "GTEPS and % of HBM roofline per semiring, batched+learned vs plain single-source"
SEMIRINGS = ["tropical", "real", "boolean", "selmax"]
SR_ID = {"tropical": 0, "real": 1, "boolean": 2, "selmax": 3}
# bytes per vertex of the gathered frontier vector and of the per-row frontier write
FRONTIER_BYTES = {"tropical": 4.0, "real": 4.0, "boolean": 0.125, "selmax": 4.0}
FRONTIER_WRITE = {"tropical": 0.0, "real": 4.0, "boolean": 0.125, "selmax": 4.0}

# DRAM traffic per k_pull launch measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum, mean over the 49 tropical iterations of the first 7
# roots of this workload; the host-driven loop's idle launches, queued past the
# end of a run, are left out; taken with --clock-control none), keyed by the hash
# of the kernel sources it was taken on; reported as null once those sources change.
NCU_TRAFFIC = {"53fa510bf09a0bd2": 241.2e6}
KERNEL_SOURCES = ["ss_bfs.cu", "ss_device.cuh", "ss_common.cuh"]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2010_09913_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def iteration_bytes(it, sr: str, n: int, C: int) -> float:
    """Algorithmic bytes of one pull iteration (SlimSell slots, chunk tables,
    own-row state, discoveries, one pass over the gathered frontier vector)."""
    rows = C * it.active_chunks
    b = 4.0 * it.slots                      # col slots of processed chunks (incl. padding)
    b += 8.0 * it.active_chunks             # cs / cl
    b += rows * (4.0 + FRONTIER_WRITE[sr])  # own-row level read + frontier write
    b += it.frontier * (4.0 + 4.0)          # level write + degree read of new vertices
    if sr == "selmax":
        b += it.frontier * 4.0              # parent write
    b += n * FRONTIER_BYTES[sr]             # gathered frontier vector, once (L2-served)
    return b


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, index: int):
        self.proc = None
        import tempfile
        out_dir = os.environ.get("SS_CLOCKS_DIR") or tempfile.gettempdir()  # raw samples kept there
        self.path = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            return parse_clocks(f)


def parse_clocks(lines):
    """Median SM clock, the largest max clock, the sample count and the throttle
    reasons seen Active, from nvidia-smi's csv,noheader,nounits lines of
    index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
    hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap; None without samples."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
            "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("SS_BENCH_GLOO") is None else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x: float, device=None) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, x: float, device=None) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def _oracle_warm(_):
    import oracle  # the import and library load, outside the timed batches
    oracle.build()
    time.sleep(0.2)  # hold this worker so that every worker gets one
    return 0


def _oracle_task(task):
    """One oracle run in a worker process: (edges reached, seconds).  kind
    "queue": the serial queue BFS plus the max-id parent pass (the CPU
    baseline); kind "semiring": the plain CSR semiring BFS of that semiring."""
    path, root, sr, kind = task
    import oracle
    row_ptr = np.load(os.path.join(path, "row_ptr.npy"), mmap_mode="r")
    col = np.load(os.path.join(path, "col.npy"), mmap_mode="r")
    t0 = time.perf_counter()
    if kind == "queue":
        dist = oracle.bfs_queue(row_ptr, col, int(root))
        oracle.dp(row_ptr, col, dist, int(root))
    else:
        dist = oracle.bfs_semiring(row_ptr, col, int(root), sr)[0]
    dt = time.perf_counter() - t0
    return oracle.reached_edges(row_ptr, dist), dt


class OraclePool:
    """The oracle run on the host cores, one serial run per worker process
    (spawned, so no CUDA state is inherited); the CSR goes to the workers
    through memory-mapped files."""

    def __init__(self, g, workers: int):
        import multiprocessing as mp
        import tempfile
        import oracle
        oracle.build()
        self.dir = tempfile.mkdtemp(prefix="ss_oracle_")
        np.save(os.path.join(self.dir, "row_ptr.npy"), np.asarray(g.row_ptr))
        np.save(os.path.join(self.dir, "col.npy"), np.asarray(g.col))
        self.workers = max(1, workers)
        self.pool = mp.get_context("spawn").Pool(self.workers)
        self.pool.map(_oracle_warm, range(self.workers), chunksize=1)

    def run_for(self, tasks, cpu_seconds: float, kind: str = "queue", per_batch: int | None = None):
        """Run tasks in batches of `per_batch` (default: one per worker) until
        the CPU seconds spent reach `cpu_seconds` (at least one batch):
        (edges, wall seconds, cpu seconds, runs)."""
        per_batch = self.workers if per_batch is None else max(1, min(per_batch, self.workers))
        edges, wall, cpu, runs, i = 0, 0.0, 0.0, 0, 0
        while runs == 0 or (cpu < cpu_seconds and runs < 1_000_000):  # tasks cycle
            batch = [tasks[(i + j) % len(tasks)] for j in range(per_batch)]
            i += per_batch
            t0 = time.perf_counter()
            res = self.pool.map(_oracle_task, [(self.dir, r, sr, kind) for r, sr in batch], chunksize=1)
            wall += time.perf_counter() - t0
            edges += sum(e for e, _ in res)
            cpu += sum(t for _, t in res)
            runs += len(res)
        return edges, wall, cpu, runs

    def close(self):
        import shutil
        self.pool.terminate()
        shutil.rmtree(self.dir, ignore_errors=True)


def oracle_workers() -> int:
    """Every host core (one serial oracle run per core)."""
    return max(1, os.cpu_count() or 1)


def cpu_oracle_sample(g, roots, cpu_seconds: float):
    """Time the oracle on the host cores over bounded samples of the workload's
    runs: the serial queue BFS plus max-id parent pass (every core, batches of
    one run per core until `cpu_seconds` of CPU time), and the plain CSR
    semiring BFS (one root, its four semirings run side by side)."""
    pool = OraclePool(g, oracle_workers())
    try:
        tasks = [(int(r), sr) for r in roots for sr in SEMIRINGS]
        queue = pool.run_for(tasks, cpu_seconds, "queue")
        semiring = pool.run_for(tasks[:4], 0.0, "semiring", per_batch=4)
    finally:
        pool.close()
    return queue, semiring, pool.workers


def run_reference(args, world, rank, pg):
    if rank != 0:
        return
    g = gg.kronecker(args.scale, seed=1)
    roots = gg.roots(g, args.roots, seed=2)
    per_step = args.ref_seconds if args.ref_seconds is not None else \
        max(10.0, min(30.0, 150.0 / max(1, args.steps + args.warmup)))
    pool = OraclePool(g, oracle_workers())
    tasks = [(int(r), sr) for r in roots for sr in SEMIRINGS]
    times, edges_l, cpu_l = [], [], []
    try:
        for s in range(args.warmup + args.steps):
            k = (s * pool.workers) % len(tasks)
            edges, wall, cpu, runs = pool.run_for(tasks[k:] + tasks[:k], per_step, "queue")
            if s >= args.warmup:
                times.append(wall)
                edges_l.append(edges)
                cpu_l.append(cpu)
    finally:
        pool.close()
    value = sum(edges_l) / sum(times) / 1e9
    ms = 1000.0 * sum(times) / len(times)
    sample = (f"oracle serial queue BFS + max-id parent pass (C, one run per (root, semiring) of "
              f"the workload; the four semirings give the same dist/parent), one run per worker "
              f"process on {pool.workers} host cores, ~{per_step:.0f} CPU-seconds per step on "
              f"kronecker scale {args.scale}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": workload_config(args, g),
            "cpu_baseline": {"kind": "oracle", "cores": pool.workers, "sample": sample, "value": value,
                             "unit": "GTEPS"},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args, g):
    return {"workload": f"kronecker scale {args.scale} edgefactor 16, {args.roots} roots one at a "
                        f"time x 4 semirings, C=32, sigma=n, SlimWork + SlimChunk w={args.split_w}",
            "graph": {"n": g.n, "nnz": g.nnz, "undirected_edges": g.m},
            "semirings": SEMIRINGS, "C": 32, "sigma": "n", "split_w": args.split_w,
            "l2": f"inputs larger than L2: SlimSell col is ~{(g.nnz * 4) >> 20} MiB+ (L2 129 MB)",
            "outputs": "int32 dist + parent per run (DP for tropical/real/boolean)"}


def time_policy(ss, torch, h, roots, policy, stream, runs_edges):
    """Device-side loops, CUDA events around every run of every semiring."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for sr in SEMIRINGS:
        for r in roots:
            ss.slimsell_bfs(h, int(r), SR_ID[sr], policy, None, None, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return runs_edges / (ms / 1000.0) / 1e9, ms


SELECTOR_MARGIN = 100  # thousandths of a log-time unit the network must gain over the rule


def train_selector(ss, torch, g, h, args):
    """Collect per-iteration variant timings and fit the selector on the GPU."""
    from paper_2010_09913_gb300 import selector
    t0 = time.perf_counter()
    Xs, Ts, Ms = [], [], []
    G = ss.SlimSellGraph.wrap(h, g.n)
    X, T, M = selector.collect(G, gg.roots(g, 64, seed=99), "tropical", repeats=2, max_per_root=24)
    Xs.append(X); Ts.append(T); Ms.append(M)
    for tg, nr in ((gg.kronecker(14, seed=7), 8), (gg.kronecker(18, seed=7), 16),
                   (gg.kronecker(23, seed=7), 8), (gg.kronecker(24, seed=7), 8),
                   (gg.lattice(4096, 0.05, seed=7), 1),
                   (gg.erdos_renyi(1 << 22, 16.0, seed=7), 8)):
        G = ss.SlimSellGraph.from_host(tg.row_ptr, tg.col, C=32, sigma=tg.n, split_w=args.split_w)
        X, T, M = selector.collect(G, gg.roots(tg, nr, seed=8), "tropical", repeats=2, max_per_root=24)
        Xs.append(X); Ts.append(T); Ms.append(M)
        G.close()
    w, loss = selector.train(np.concatenate(Xs), np.concatenate(Ts), np.concatenate(Ms), steps=12000,
                             lr=1e-3)
    return w, {"samples": int(sum(x.shape[0] for x in Xs)), "final_loss": loss,
               "seconds": time.perf_counter() - t0, "margin_log_units": SELECTOR_MARGIN / 1000.0,
               "graphs": f"kronecker {args.scale} (64 roots other than the timed ones), kronecker 14, 18, "
                         "23 and 24, lattice 4096^2 (5% deleted, seed 7), ER 2^22 (mean deg 16, seed 7)"}


def batched_learned(ss, torch, g, h, roots, args, stream, dev, runs_edges):
    """On the same graph: heuristic and learned per-iteration schedules of
    single-source BFS, and bit-packed multi-source batches."""
    from paper_2010_09913_gb300 import selector
    out = {"unit": "GTEPS", "graph": f"kronecker scale {args.scale}"}
    gte, _ = time_policy(ss, torch, h, roots, ss.V_SLIMWORK, stream, runs_edges)
    out["plain_slimwork_single"] = gte
    gte, _ = time_policy(ss, torch, h, roots, ss.V_HEURISTIC, stream, runs_edges)
    out["heuristic_single"] = gte
    # train the selector on timings the method generates on the configurations'
    # graph families: Kronecker scale 14 and 18, this scale-22 graph with other
    # roots than the timed ones, a lattice and an Erdos-Renyi graph (24 evenly
    # spaced iterations per run at most, so long runs do not dominate)
    w, tr = train_selector(ss, torch, g, h, args)
    out["selector_training"] = tr
    ss.slimsell_selector_load(h, w)
    ss.slimsell_set_option(h, ss.OPT_SELECTOR_MARGIN, SELECTOR_MARGIN)
    for sr in SEMIRINGS:  # build the learned loop graphs outside the timed region
        ss.slimsell_bfs(h, int(roots[0]), SR_ID[sr], ss.V_LEARNED, None, None, stream)
    gte, _ = time_policy(ss, torch, h, roots, ss.V_LEARNED, stream, runs_edges)
    out["learned_single"] = gte
    ev = selector.evaluate(ss.SlimSellGraph.wrap(h, g.n), roots[:4], "tropical", weights=w, repeats=2)
    out["schedule_kernel_ms_tropical_4roots"] = {k: round(v, 4) for k, v in ev.items()}
    # multi-source batches on the same graph
    for k in (64, 256, 1024):
        mroots = gg.roots(g, k, seed=20 + k)
        r_d = torch.from_numpy(mroots).to(dev)
        dist = torch.empty((g.n, k), dtype=torch.int32, device=dev)
        ss.slimsell_bfs_multi(h, r_d, ss.V_SLIMWORK, dist, stream)  # warm
        st, _ = ss.slimsell_get_run_stats(h)
        edges = st.reached_degree // 2
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 2
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            ss.slimsell_bfs_multi(h, r_d, ss.V_SLIMWORK, dist, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[f"multi_{k}"] = edges / (ms / 1000.0) / 1e9
        out[f"multi_{k}_ms"] = ms
        if k == 64:  # the same sources with largest-id parents as well
            par = torch.empty((g.n, k), dtype=torch.int32, device=dev)
            ss.slimsell_bfs_multi_parents(h, r_d, ss.V_SLIMWORK, dist, par, stream)  # warm
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                ss.slimsell_bfs_multi_parents(h, r_d, ss.V_SLIMWORK, dist, par, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            out[f"multi_{k}_parents"] = edges / (ms / 1000.0) / 1e9
            out[f"multi_{k}_parents_ms"] = ms
            del par
        del dist
    ss.slimsell_selector_load(h, None)
    out["selector_weights"] = w
    best_single = max(out["heuristic_single"], out["learned_single"])
    out["best_batched_or_learned_over_plain"] = max(best_single, out["multi_1024"]) / out["plain_slimwork_single"]
    return out


def batch_workload(ss, torch, ngraphs, stream, dev):
    """The many-graph configuration: `ngraphs` Kronecker graphs with scales drawn
    uniformly from 10..18 (seeded), layout parameters autotuned once per scale
    (C x sigma x split width grid, tropical SlimWork timings), one handle per
    graph and one seeded root each.  Returns (graphs, scales, handles, roots,
    tuned, autotune seconds)."""
    from paper_2010_09913_gb300 import autotune
    rng = np.random.default_rng(17)
    scales = rng.integers(10, 19, ngraphs)
    graphs = [gg.kronecker(int(s), seed=1000 + i) for i, s in enumerate(scales)]
    t0 = time.perf_counter()
    tuned = {}
    for s in sorted(set(int(x) for x in scales)):
        g = graphs[int(np.flatnonzero(scales == s)[0])]
        best, _ = autotune.tune(g.row_ptr, g.col, gg.roots(g, 2, seed=3), "tropical", "slimwork",
                                repeats=2)
        tuned[s] = best
    tune_s = time.perf_counter() - t0
    handles = []
    for g, s in zip(graphs, scales):
        p = tuned[int(s)]
        rp = torch.from_numpy(g.row_ptr).to(dev)
        cl = torch.from_numpy(g.col).to(dev)
        sigma = g.n if p["sigma"] == "n" else int(p["sigma"])
        handles.append(ss.slimsell_build(rp, cl, g.n, g.nnz, p["C"], sigma, p["split_w"], stream))
    roots = [int(gg.roots(g, 1, seed=2)[0]) for g in graphs]
    return graphs, scales, handles, roots, tuned, tune_s


def batched_graphs(ss, torch, ngraphs, stream, dev):
    """Many Kronecker graphs of uneven size (scales drawn from 10..18), one root
    each: layout parameters autotuned once per scale, then every BFS one after
    another vs all of them in one CUDA-graph launch."""
    graphs, scales, handles, roots, tuned, tune_s = batch_workload(ss, torch, ngraphs, stream, dev)
    r_d = torch.tensor(roots, dtype=torch.int32, device=dev)
    out = {"graphs": ngraphs, "scales": {int(s): int((scales == s).sum()) for s in sorted(set(scales))},
           "tuned": {str(k): v for k, v in tuned.items()}, "autotune_seconds": tune_s,
           "unit": "GTEPS"}
    # every BFS one after another (device-side loops)
    for h, r in zip(handles, roots):
        ss.slimsell_bfs(h, r, SR_ID["tropical"], ss.V_SLIMWORK, None, None, stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for h, r in zip(handles, roots):
        ss.slimsell_bfs(h, r, SR_ID["tropical"], ss.V_SLIMWORK, None, None, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    edges = 0
    for policy in ("slimwork", "heuristic"):
        b = ss.slimsell_batch_create(handles, SR_ID["tropical"], ss.POLICIES[policy])
        ss.slimsell_batch_run(b, r_d, None, None, stream)
        stats = ss.slimsell_batch_get_stats(b, ngraphs)
        edges = sum(st.reached_degree // 2 for st in stats)
        reps = 5
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            ss.slimsell_batch_run(b, r_d, None, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[f"batch_{policy}_ms"] = ms
        out[f"batch_{policy}"] = edges / (ms / 1000.0) / 1e9
        ss.slimsell_batch_destroy(b)
    out["sequential_slimwork_ms"] = seq_ms
    out["sequential_slimwork"] = edges / (seq_ms / 1000.0) / 1e9
    out["edges"] = edges
    for h in handles:
        ss.slimsell_destroy(h)
    return out


def roofline_at_scale(ss, torch, scale, nroots, split_w, stream, dev):
    """Plain single-source SlimSell BFS (SlimWork + SlimChunk) at a larger scale:
    iteration-kernel GB/s from per-launch CUDA events, and whole-run GTEPS; then
    bit-packed multi-source BFS with 64, 256 and 1024 roots on the same graph."""
    g = gg.kronecker(scale, seed=1)
    roots = gg.roots(g, nroots, seed=2)
    rp_d = torch.from_numpy(g.row_ptr).to(dev)
    col_d = torch.from_numpy(g.col).to(dev)
    h = ss.slimsell_build(rp_d, col_d, g.n, g.nnz, 32, g.n, split_w, stream)
    del rp_d, col_d
    hbm, kind = load_peaks()
    out = {"graph": f"kronecker scale {scale}", "n": g.n, "nnz": g.nnz, "roots": nroots}
    for sr in SEMIRINGS:
        ss.slimsell_set_profiling(h, True)
        bytes_, ms_, edges = 0.0, 0.0, 0
        for r in roots:
            ss.slimsell_bfs(h, int(r), SR_ID[sr], ss.V_SLIMWORK, None, None, stream)
            st, its = ss.slimsell_get_run_stats(h, cap=4096)
            for i in range(1, st.iterations + 1):
                bytes_ += iteration_bytes(its[i], sr, g.n, 32)
            ms_ += st.iter_kernel_ms
            edges += st.reached_degree // 2
        ss.slimsell_set_profiling(h, False)
        ach = bytes_ / (ms_ / 1000.0) / 1e9
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for r in roots:
            ss.slimsell_bfs(h, int(r), SR_ID[sr], ss.V_SLIMWORK, None, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[sr] = {"iteration_kernel_gbs": ach, "hbm_frac": ach / hbm, "peak": hbm, "peak_kind": kind,
                   "gteps_slimwork": edges / (ms / 1000.0) / 1e9}
        gte, _ = time_policy(ss, torch, h, roots, ss.V_HEURISTIC, stream, 4 * edges)
        out[sr]["gteps_heuristic_all4"] = gte
    # bit-packed multi-source BFS on the same graph (k seeded roots at once, k x n
    # int32 distances written), against the single-source runs above
    for k in (64, 256, 1024):
        mroots = gg.roots(g, k, seed=20 + k)
        r_d = torch.from_numpy(mroots).to(dev)
        dist = torch.empty((g.n, k), dtype=torch.int32, device=dev)
        ss.slimsell_bfs_multi(h, r_d, ss.V_SLIMWORK, dist, stream)  # warm-up
        st, _ = ss.slimsell_get_run_stats(h)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        ss.slimsell_bfs_multi(h, r_d, ss.V_SLIMWORK, dist, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[f"multi_{k}"] = {"gteps": (st.reached_degree // 2) / (ms / 1000.0) / 1e9, "ms": ms}
        del dist
    ss.slimsell_destroy(h)
    return out


def format_ab(ss, torch, g, sigmas, stream, dev, nroots=4):
    """Speedup of SlimSell over Sell-C-sigma (Section IV) on the same layout (C =
    32, SlimChunk w = 256), for each sigma and semiring: the plain value-vector
    BFS-SpMV in both formats (summed device time of the iteration kernels), and
    the production SlimWork pull streaming either format (device-side loops,
    CUDA events around the runs); `nroots` roots, each format warmed up once
    (which builds the Sell arrays)."""
    roots = gg.roots(g, nroots, seed=5)
    rp_d = torch.from_numpy(g.row_ptr).to(dev)
    col_d = torch.from_numpy(g.col).to(dev)
    dist = torch.empty(g.n, dtype=torch.int32, device=dev)
    out = {"n": g.n, "nnz": g.nnz, "roots": nroots}
    for sigma in sigmas:
        h = ss.slimsell_build(rp_d, col_d, g.n, g.nnz, 32, sigma, 256, stream)
        inf = ss.slimsell_get_info(h)
        edges = 0
        for r in roots:
            ss.slimsell_bfs(h, int(r), SR_ID["tropical"], ss.V_SLIMWORK, None, None, stream)
            st, _ = ss.slimsell_get_run_stats(h)
            edges += st.reached_degree // 2
        row = {"sigma": inf.sigma, "slots": inf.slots, "slots_per_nnz": inf.slots / max(1, g.nnz)}
        for sr in SEMIRINGS:
            ms = {}
            for name, f in (("slimsell", ss.FORMAT_SLIMSELL), ("sell", ss.FORMAT_SELL)):
                ss.slimsell_bfs_spmv(h, int(roots[0]), SR_ID[sr], f, dist, stream, timed=True)
                ms[name] = sum(ss.slimsell_bfs_spmv(h, int(r), SR_ID[sr], f, dist, stream, timed=True)
                               for r in roots)
            # the production pull (SlimWork, bitmaps, device-side loop) streaming
            # either format: CUDA events around all roots' runs
            pull = {}
            for name, f in (("slimsell", ss.FORMAT_SLIMSELL), ("sell", ss.FORMAT_SELL)):
                ss.slimsell_set_option(h, ss.OPT_FORMAT, f)
                ss.slimsell_bfs(h, int(roots[0]), SR_ID[sr], ss.V_SLIMWORK, None, None, stream)  # warm
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                for r in roots:
                    ss.slimsell_bfs(h, int(r), SR_ID[sr], ss.V_SLIMWORK, None, None, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                pull[name] = e0.elapsed_time(e1)
            ss.slimsell_set_option(h, ss.OPT_FORMAT, ss.FORMAT_SLIMSELL)
            row[sr] = {"slimsell_ms": ms["slimsell"], "sell_ms": ms["sell"],
                       "speedup_slimsell_over_sell": ms["sell"] / ms["slimsell"],
                       "gteps_slimsell": edges / (ms["slimsell"] / 1000.0) / 1e9,
                       "gteps_sell": edges / (ms["sell"] / 1000.0) / 1e9,
                       "pull_slimwork_slimsell_ms": pull["slimsell"], "pull_slimwork_sell_ms": pull["sell"],
                       "pull_speedup_slimsell_over_sell": pull["sell"] / pull["slimsell"]}
        out[f"sigma_{inf.sigma}"] = row
        ss.slimsell_destroy(h)
        torch.cuda.empty_cache()
    del rp_d, col_d, dist
    return out


def bc_measure(ss, torch, g, h, stream, dev, nsources=64):
    """Betweenness centrality (Brandes, fp64) over `nsources` seeded sources (one
    batch of the bit-packed multi-source passes) on the benchmark graph's
    handle: summed device time of the level kernels and TEPS = sources *
    undirected edges / time."""
    src = torch.from_numpy(gg.roots(g, nsources, seed=11)).to(dev)
    out = torch.empty(g.n, dtype=torch.float64, device=dev)
    ss.slimsell_bc(h, src[:1], out, stream)  # warm-up (allocates the scratch)
    ms = ss.slimsell_bc(h, src, out, stream, timed=True)
    m = g.nnz // 2
    return {"sources": nsources, "kernel_ms": ms, "ms_per_source": ms / nsources,
            "gteps": nsources * m / (ms / 1000.0) / 1e9,
            "definition": "sources x undirected edges / summed device time of the level kernels"}


def format_ab_sections(ss, torch, stream, dev, g22=None):
    """The format comparison on Kronecker 22 with sigma = C = 32 (the paper's
    sigma = 2^4 rounded up to a multiple of C) and on Kronecker 24 (the paper's
    n = 2^24) with sigma = 2^12 and 2^18; at scale 24 sigma = 32 would need about
    20 slots per edge (over 150 GB with the Sell arrays)."""
    g22 = g22 if g22 is not None else gg.kronecker(22, seed=1)
    out = {"kronecker22": format_ab(ss, torch, g22, (32,), stream, dev)}
    out["kronecker24"] = format_ab(ss, torch, gg.kronecker(24, seed=1), (1 << 12, 1 << 18), stream, dev)
    return out


def selector_heldout(ss, torch, stream, dev, weights):
    """The selector trained above, on graphs it never saw: Kronecker scale 25
    (edgefactor 16) and a 8192 x 8192 lattice with 5% of its edges deleted, 64
    seeded roots each; tropical; learned against the frontier-size rule and
    plain SlimWork (plain SlimWork on the lattice on a 2-root sample: one run
    takes seconds there)."""
    out = {}
    for name, g, nr, nplain in (("kronecker scale 25", gg.kronecker(25, seed=3), 64, 64),
                                ("lattice 8192^2 (5% deleted)", gg.lattice(8192, 0.05, seed=3), 64, 2)):
        roots = gg.roots(g, nr, seed=4)
        rp_d = torch.from_numpy(g.row_ptr).to(dev)
        col_d = torch.from_numpy(g.col).to(dev)
        h = ss.slimsell_build(rp_d, col_d, g.n, g.nnz, 32, g.n, 256, stream)
        res = {"roots": nr, "n": int(g.n), "nnz": int(g.nnz)}
        del rp_d, col_d, g
        ss.slimsell_selector_load(h, weights)
        ss.slimsell_set_option(h, ss.OPT_SELECTOR_MARGIN, SELECTOR_MARGIN)
        for pol_name, pol, rs in (("learned", ss.V_LEARNED, roots), ("heuristic", ss.V_HEURISTIC, roots),
                                  ("slimwork", ss.V_SLIMWORK, roots[:nplain])):
            ss.slimsell_bfs(h, int(rs[0]), SR_ID["tropical"], pol, None, None, stream)  # warm-up
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            ms, edges = 0.0, 0
            for r in rs:
                torch.cuda.synchronize()
                e0.record(stream)
                ss.slimsell_bfs(h, int(r), SR_ID["tropical"], pol, None, None, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
                edges += ss.slimsell_get_run_stats(h)[0].reached_degree // 2
            res[pol_name] = {"gteps": edges / (ms / 1000.0) / 1e9, "ms_per_run": ms / len(rs), "runs": len(rs)}
        res["learned_over_heuristic"] = res["learned"]["gteps"] / res["heuristic"]["gteps"]
        res["learned_over_slimwork"] = res["learned"]["gteps"] / res["slimwork"]["gteps"]
        ss.slimsell_destroy(h)
        out[name] = res
    return out


def summary(line):
    """Compact digest of the sections, printed as the line's last key (a reader
    that keeps only the end of the output still sees it)."""
    def r3(x):
        return None if x is None else float(f"{x:.4g}")
    out = {}
    if "per_semiring" in line:
        out["kron22_gteps"] = {sr: r3(v["gteps"]) for sr, v in line["per_semiring"].items()}
        out["kron22_whole_run_hbm_frac"] = {sr: r3(v["whole_run_hbm_frac"])
                                            for sr, v in line["per_semiring"].items()}
    if "scale24" in line:
        out["kron24_k_pull_hbm_frac"] = {sr: r3(line["scale24"][sr]["hbm_frac"]) for sr in SEMIRINGS}
    bl = line.get("batched_learned")
    if bl:
        out["kron22_single"] = {k: r3(bl[k]) for k in ("plain_slimwork_single", "heuristic_single",
                                                       "learned_single")}
        out["kron22_multi"] = {k: r3(bl[f"multi_{k}"]) for k in (64, 256, 1024)}
        out["best_batched_or_learned_over_plain"] = r3(bl["best_batched_or_learned_over_plain"])
    ho = line.get("selector_heldout")
    if ho:
        out["heldout"] = {name.split(" (")[0]: {p: r3(v[p]["gteps"]) for p in ("learned", "heuristic",
                                                                              "slimwork")}
                          for name, v in ho.items()}
    hd = line.get("high_diameter")
    if hd:
        out["high_diameter_tropical"] = {name.split(" (")[0]: {p: r3(v[f"tropical_{p}"]["gteps"])
                                                              for p in ("heuristic", "learned", "slimwork")
                                                              if f"tropical_{p}" in v}
                                         for name, v in hd.items()}
    bg = line.get("batched_graphs")
    if bg:
        out["batch200"] = {k: r3(bg[k]) for k in ("batch_slimwork", "batch_heuristic", "sequential_slimwork")}
    return out


def high_diameter(ss, torch, stream, dev, weights=None, nroots=16, host_loop=False):
    """High-diameter and low-skew graphs: a 4096 x 4096 lattice with 5% of its
    edges deleted and an Erdos-Renyi graph (n = 2^22, mean degree 16); sel-max
    and tropical; C = 32, sigma = N; 16 seeded roots.  The adaptive schedule
    (frontier-size rule, small levels in the cluster push) next to the plain
    SlimWork pass, which on the lattice is timed on a 2-root sample (one run
    takes most of a second there)."""
    out = {}
    for name, g in (("lattice 4096^2 (5% deleted)", gg.lattice(4096, 0.05, seed=1)),
                    ("erdos-renyi 2^22 (mean degree 16)", gg.erdos_renyi(1 << 22, 16.0, seed=1))):
        roots = gg.roots(g, nroots, seed=2)
        rp_d = torch.from_numpy(g.row_ptr).to(dev)
        col_d = torch.from_numpy(g.col).to(dev)
        h = ss.slimsell_build(rp_d, col_d, g.n, g.nnz, 32, g.n, 256, stream)
        del rp_d, col_d
        if host_loop:
            ss.slimsell_set_option(h, ss.OPT_DEVICE_LOOP, 0)
        res = {"n": g.n, "nnz": g.nnz, "roots": nroots}
        lattice = name.startswith("lattice")
        pols = [("heuristic", ss.V_HEURISTIC, roots), ("slimwork", ss.V_SLIMWORK, roots[:2] if lattice else roots)]
        if weights is not None:
            ss.slimsell_selector_load(h, weights)
            ss.slimsell_set_option(h, ss.OPT_SELECTOR_MARGIN, SELECTOR_MARGIN)
            pols.append(("learned", ss.V_LEARNED, roots))
        for sr in ("selmax", "tropical"):
            for pol_name, pol, rs in pols:
                ss.slimsell_bfs(h, int(rs[0]), SR_ID[sr], pol, None, None, stream)  # warm-up
                edges, iters, local = 0, 0, 0
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                ms = 0.0
                for r in rs:
                    torch.cuda.synchronize()
                    e0.record(stream)
                    ss.slimsell_bfs(h, int(r), SR_ID[sr], pol, None, None, stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms += e0.elapsed_time(e1)
                    st, its = ss.slimsell_get_run_stats(h, cap=16384)
                    edges += st.reached_degree // 2
                    iters += st.iterations
                    local += sum(1 for i in range(1, min(st.iterations, 16383) + 1)
                                 if its[i].variant == ss.VARIANT_PUSH_LOCAL)
                res[f"{sr}_{pol_name}"] = {"gteps": edges / (ms / 1000.0) / 1e9,
                                           "ms_per_run": ms / len(rs), "runs": len(rs),
                                           "levels_per_run": iters / len(rs),
                                           "cluster_push_levels_per_run": local / len(rs)}
        ss.slimsell_destroy(h)
        out[name] = res
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=22)
    ap.add_argument("--roots", type=int, default=64)
    ap.add_argument("--split-w", type=int, default=256)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ablations", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-scale24", action="store_true")
    ap.add_argument("--no-high-diameter", action="store_true")
    ap.add_argument("--no-format-ab", action="store_true")
    ap.add_argument("--no-bc", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=None,
                    help="reference arm: seconds of oracle work per step (default 10-30)")
    ap.add_argument("--only", choices=["high-diameter", "format-ab", "bc"], default=None,
                    help="run one section alone and print it (profiling runs)")
    ap.add_argument("--host-loop", action="store_true",
                    help="host-driven iteration loop (kernels visible to a profiler)")
    ap.add_argument("--no-heldout", action="store_true",
                    help="skip the selector's held-out evaluation (Kronecker 25, lattice 8192^2)")
    ap.add_argument("--batch-graphs", type=int, default=200)
    args = ap.parse_args()
    world, rank, local, pg = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank, pg)
        return

    import torch
    import paper_2010_09913_gb300 as ss
    ss.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    if args.only == "high-diameter":
        if rank == 0:
            print(json.dumps({"high_diameter": high_diameter(ss, torch, stream, dev, None, nroots=args.roots,
                                                             host_loop=args.host_loop)}), flush=True)
        return
    if args.only == "bc":
        if rank == 0:
            g = gg.kronecker(args.scale, seed=1)
            rp_d = torch.from_numpy(g.row_ptr).to(dev)
            col_d = torch.from_numpy(g.col).to(dev)
            h = ss.slimsell_build(rp_d, col_d, g.n, g.nnz, 32, g.n, args.split_w, stream)
            print(json.dumps({"bc": bc_measure(ss, torch, g, h, stream, dev)}), flush=True)
            ss.slimsell_destroy(h)
        return
    if args.only == "format-ab":
        if rank == 0:
            print(json.dumps({"format_ab": format_ab_sections(ss, torch, stream, dev)}), flush=True)
        return

    g = gg.kronecker(args.scale, seed=1)
    roots = gg.roots(g, args.roots, seed=2 + 1000 * rank)
    n = g.n
    rp_d = torch.from_numpy(g.row_ptr).to(dev)
    col_d = torch.from_numpy(g.col).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = ss.slimsell_build(rp_d, col_d, n, g.nnz, 32, n, args.split_w, stream)
    torch.cuda.synchronize()
    build_ms = 1000.0 * (time.perf_counter() - t0)
    info = ss.slimsell_get_info(h)
    dist = torch.empty(n, dtype=torch.int32, device=dev)
    parent = torch.empty(n, dtype=torch.int32, device=dev)

    # one untimed pass collects the deterministic per-run statistics
    ss.slimsell_set_profiling(h, True)
    runs = []
    for sr in SEMIRINGS:
        for r in roots:
            ss.slimsell_bfs(h, int(r), SR_ID[sr], ss.V_SLIMWORK, dist, parent, stream)
            st, iters = ss.slimsell_get_run_stats(h, cap=4096)
            its = [iters[i] for i in range(1, min(st.iterations, 4095) + 1)]
            pull_bytes = sum(iteration_bytes(it, sr, n, 32) for it in its)
            launches = 2 + st.iterations + 1  # init, root, one kernel per iteration, output
            runs.append({"sr": sr, "root": int(r), "edges": st.reached_degree // 2,
                         "iterations": st.iterations, "pull_bytes": pull_bytes,
                         "slots": st.slots, "dp_slots": st.dp_slots, "launches": launches})
    edges_per_step = sum(x["edges"] for x in runs)
    launches_per_step = sum(x["launches"] for x in runs)
    pull_bytes_per_step = sum(x["pull_bytes"] for x in runs)
    pull_launches_per_step = sum(x["iterations"] for x in runs)

    def step(record=None):
        for sr in SEMIRINGS:
            if record is not None:
                record[sr][0].record(stream)
            for r in roots:
                ss.slimsell_bfs(h, int(r), SR_ID[sr], ss.V_SLIMWORK, dist, parent, stream)
            if record is not None:
                record[sr][1].record(stream)

    # timed region: device-side iteration loops, no host round trips
    ss.slimsell_set_profiling(h, False)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(pg)
    clocks = Clocks(local)
    rec = {sr: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for sr in SEMIRINGS}
    per_sr_ms = {sr: 0.0 for sr in SEMIRINGS}
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step(rec)
        torch.cuda.synchronize()
        for sr in SEMIRINGS:
            per_sr_ms[sr] += rec[sr][0].elapsed_time(rec[sr][1])
    ev1.record(stream)
    torch.cuda.synchronize()
    total_ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    barrier(pg)
    total_ms_max = max_over_ranks(pg, total_ms, dev)
    edges_all = sum_over_ranks(pg, float(edges_per_step * args.steps), dev)
    value = edges_all / (total_ms_max / 1000.0) / 1e9

    # roofline of the iteration kernel: one step with CUDA events around every
    # iteration-kernel launch (host-driven loop, same kernels)
    ss.slimsell_set_profiling(h, True)
    pull_ms = 0.0
    for sr in SEMIRINGS:
        for r in roots:
            ss.slimsell_bfs(h, int(r), SR_ID[sr], ss.V_SLIMWORK, dist, parent, stream)
            pull_ms += ss.slimsell_get_run_stats(h)[0].iter_kernel_ms
    ss.slimsell_set_profiling(h, False)
    hbm, peak_kind = load_peaks()
    achieved = pull_bytes_per_step / (pull_ms / 1000.0) / 1e9 if pull_ms > 0 else 0.0
    per_sr = {}
    for sr in SEMIRINGS:
        e = sum(x["edges"] for x in runs if x["sr"] == sr) * args.steps
        b = sum(x["pull_bytes"] for x in runs if x["sr"] == sr) * args.steps
        ms = per_sr_ms[sr]
        per_sr[sr] = {"gteps": e / (ms / 1000.0) / 1e9,
                      "ms_per_run": ms / (args.steps * len(roots)),
                      "pull_bytes_per_run": b / (args.steps * len(roots)),
                      "whole_run_gbs": b / (ms / 1000.0) / 1e9,
                      "whole_run_hbm_frac": b / (ms / 1000.0) / 1e9 / hbm}
    # Graph500 convention alongside the aggregate: the harmonic mean over roots of
    # per-root GTEPS (each run timed alone with CUDA events, device-side loop)
    ev_a = torch.cuda.Event(enable_timing=True)
    ev_b = torch.cuda.Event(enable_timing=True)
    for sr in SEMIRINGS:
        inv = 0.0
        for x in (x for x in runs if x["sr"] == sr):
            ev_a.record(stream)
            ss.slimsell_bfs(h, x["root"], SR_ID[sr], ss.V_SLIMWORK, dist, parent, stream)
            ev_b.record(stream)
            torch.cuda.synchronize()
            inv += (ev_a.elapsed_time(ev_b) / 1000.0) / max(1, x["edges"])
        per_sr[sr]["gteps_harmonic_mean_over_roots"] = len(roots) / inv / 1e9
    traffic = NCU_TRAFFIC.get(kernel_source_hash())

    line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": workload_config(args, g),
            "gpu_launches": launches_per_step * args.steps,
            "roofline": {"bound": "hbm", "kernel": "k_pull (SlimSell pull iteration)",
                         "achieved": achieved, "peak": hbm, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": traffic,
                         "algorithmic_bytes_per_launch": pull_bytes_per_step / max(1, pull_launches_per_step),
                         "avg_launch_ms": pull_ms / max(1, pull_launches_per_step),
                         "launch_timing": "one step through the host-driven iteration loop (same "
                                          "kernels as the timed device-side loop), CUDA events on "
                                          "the launching stream around every k_pull launch",
                         "frac_of_nominal_8tbs": achieved / 8000.0},
            "per_semiring": per_sr, "clocks": clk,
            "build_ms": build_ms,
            "layout": {"slots": info.slots, "padding": info.padding, "n_items": info.n_items,
                       "n_split_chunks": info.n_split_chunks, "max_degree": info.max_degree}}

    sel_w = None
    if not args.no_batched and rank == 0:
        line["batched_learned"] = batched_learned(ss, torch, g, h, roots, args, stream, dev,
                                                  edges_per_step)
        sel_w = line["batched_learned"].pop("selector_weights")
        line["batched_graphs"] = batched_graphs(ss, torch, args.batch_graphs, stream, dev)
    if not args.no_e2e:
        line["e2e"] = e2e_measure(ss, torch, g, roots, args, stream, dev, pg)
    if not args.no_ablations and rank == 0:
        line["ablations"] = ablations(ss, torch, g, roots[:8], h, rp_d, col_d, args, stream, dev)
    if not args.no_bc and rank == 0:
        line["bc"] = bc_measure(ss, torch, g, h, stream, dev)
    ss.slimsell_destroy(h)
    del rp_d, col_d
    if not args.no_scale24 and rank == 0:
        torch.cuda.empty_cache()
        line["scale24"] = roofline_at_scale(ss, torch, 24, 8, args.split_w, stream, dev)
        # the single-source roofline target is set on this graph: carry its
        # per-semiring fractions in the roofline object itself
        line["roofline"]["scale24_frac"] = {sr: line["scale24"][sr]["hbm_frac"] for sr in SEMIRINGS}
        line["roofline"]["scale24_frac_min"] = min(line["roofline"]["scale24_frac"].values())
    if not args.no_format_ab and rank == 0:
        torch.cuda.empty_cache()
        line["format_ab"] = format_ab_sections(ss, torch, stream, dev, g)
    if not args.no_high_diameter and rank == 0:
        torch.cuda.empty_cache()
        line["high_diameter"] = high_diameter(ss, torch, stream, dev, sel_w)
    if not args.no_heldout and rank == 0 and sel_w is not None:
        torch.cuda.empty_cache()
        line["selector_heldout"] = selector_heldout(ss, torch, stream, dev, sel_w)
    if rank == 0 and world == 1 and not args.no_cpu:
        (edges, wall, cpu, nruns), (s_edges, s_wall, s_cpu, s_runs), workers = \
            cpu_oracle_sample(g, roots, 20.0)
        line["cpu_baseline"] = {"value": edges / wall / 1e9, "unit": "GTEPS", "cores": workers,
                                "kind": "oracle",
                                "sample": f"{nruns} runs (roots x 4 semirings) of the oracle's serial "
                                          f"queue BFS + max-id parent pass on kronecker scale "
                                          f"{args.scale}, one run per worker process on every host "
                                          f"core, {cpu:.0f} CPU-seconds in {wall:.1f} s",
                                "semiring_bfs": {"value": s_edges / s_wall / 1e9, "unit": "GTEPS",
                                                 "cores": min(4, workers),
                                                 "sample": f"{s_runs} runs (one root x 4 semirings) of "
                                                           f"the oracle's plain CSR semiring BFS (fp64), "
                                                           f"side by side, {s_cpu:.0f} CPU-seconds in "
                                                           f"{s_wall:.1f} s"}}
    if rank == 0:
        line["summary"] = summary(line)
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def e2e_measure(ss, torch, g, roots, args, stream, dev, pg):
    """Same metric through the public C ABI from host memory: per step, pinned
    host CSR -> device, build, every run, device -> pinned host dist + parent.
    The read-back of run i (a copy stream) overlaps run i + 1 (double-buffered
    device outputs), as a serving loop would do it."""
    n = g.n
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    out_h = [torch.empty((2, n), dtype=torch.int32).pin_memory() for _ in range(2)]
    outs = [torch.empty((2, n), dtype=torch.int32, device=dev) for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=dev)
    ran = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    h2d = rp_h.numel() * 8 + col_h.numel() * 4
    # edges per run are deterministic: count them once, outside the timed region
    rp_d = rp_h.to(dev)
    col_d = col_h.to(dev)
    h = ss.slimsell_build(rp_d, col_d, n, g.nnz, 32, n, args.split_w, stream)
    edges_per_step = 0
    for sr in SEMIRINGS:
        for r in roots:
            ss.slimsell_bfs(h, int(r), SR_ID[sr], ss.V_SLIMWORK, None, None, stream)
            edges_per_step += ss.slimsell_get_run_stats(h)[0].reached_degree // 2
    ss.slimsell_destroy(h)
    del rp_d, col_d
    d2h = 8 * n * len(SEMIRINGS) * len(roots)

    def one_step():
        rp_d = rp_h.to(dev, non_blocking=True)
        col_d = col_h.to(dev, non_blocking=True)
        h = ss.slimsell_build(rp_d, col_d, n, g.nnz, 32, n, args.split_w, stream)
        i = 0
        for sr in SEMIRINGS:
            for r in roots:
                j = i & 1
                stream.wait_event(copied[j])  # the read-back of run i - 2 is done with this buffer
                ss.slimsell_bfs(h, int(r), SR_ID[sr], ss.V_SLIMWORK, outs[j][0], outs[j][1], stream)
                ran[j].record(stream)
                with torch.cuda.stream(copy_stream):
                    copy_stream.wait_event(ran[j])
                    out_h[j].copy_(outs[j], non_blocking=True)
                    copied[j].record(copy_stream)
                i += 1
        stream.synchronize()
        copy_stream.synchronize()
        ss.slimsell_destroy(h)
        del rp_d, col_d

    steps = max(1, min(args.steps, 3))
    for j in range(2):
        copied[j].record(copy_stream)
    one_step()
    torch.cuda.synchronize()
    barrier(pg)
    t0 = time.perf_counter()
    for _ in range(steps):
        one_step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dt = max_over_ranks(pg, dt, dev)
    edges = sum_over_ranks(pg, float(edges_per_step * steps), dev)
    return {"value": edges / dt / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": steps,
            "timed": "host wall clock around, per step, pinned H2D of the CSR, slimsell_build, all "
                     "runs, and the D2H of every run's dist+parent (a copy stream overlapping the "
                     "next run), synchronised"}


def ablations(ss, torch, g, roots, h_main, rp_d, col_d, args, stream, dev):
    """Paper experiments on the same graph: sigma sweep, SlimWork off, SlimChunk off."""
    n = g.n
    out = {}
    dist = torch.empty(n, dtype=torch.int32, device=dev)
    parent = torch.empty(n, dtype=torch.int32, device=dev)

    def measure(h, policy):
        res = {}
        for sr in SEMIRINGS:
            ss.slimsell_bfs(h, int(roots[0]), SR_ID[sr], policy, dist, parent, stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            edges = 0
            e0.record(stream)
            for r in roots:
                ss.slimsell_bfs(h, int(r), SR_ID[sr], policy, dist, parent, stream)
                edges += ss.slimsell_get_run_stats(h)[0].reached_degree // 2
            e1.record(stream)
            torch.cuda.synchronize()
            res[sr] = round(edges / (e0.elapsed_time(e1) / 1000.0) / 1e9, 3)
        return res

    out["sigma_n_slimwork"] = measure(h_main, ss.V_SLIMWORK)
    out["sigma_n_no_slimwork"] = measure(h_main, ss.V_FULL)
    for label, sigma, w in [("sigma_1024", 1024, args.split_w), ("sigma_1", 1, args.split_w),
                            ("sigma_n_no_slimchunk", n, 0)]:
        h = ss.slimsell_build(rp_d, col_d, n, g.nnz, 32, sigma, w, stream)
        inf = ss.slimsell_get_info(h)
        out[label] = measure(h, ss.V_SLIMWORK)
        out[label + "_padding"] = int(inf.padding)
        ss.slimsell_destroy(h)
    out["roots"] = len(roots)
    out["unit"] = "GTEPS"
    return out


if __name__ == "__main__":
    main()
