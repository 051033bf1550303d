#!/usr/bin/env python
"""Benchmark: GTEPS (harmonic mean over roots) of direction-optimizing BFS on one GB300.

Workload (default): R-MAT scale 26, edge factor 16, initiator .57/.19/.19/.05,
symmetrised, self-loops and duplicates removed, ids relabelled from seed
1026; 64 distinct seeded roots with degree > 0; CSR layout; alpha 14, beta 24;
bottom-up steps scan the hub-first copy of the rows (neighbours by degree, highest
first; --bu-rows id scans the id-sorted rows the paper stores).
A step is one full search (the whole level loop: init, top-down / bottom-up
levels, conversions, direction switches) from the next root, cycling through
the 64 roots; inputs (the 9 GB graph) are resident and larger than L2.

value   = undirected edges x steps / total device time of the steps, summed
          over ranks (= harmonic mean of per-root GTEPS when every step is one
          root); CUDA events on the launching stream, after W warm-up steps.
e2e     = the same through the public API with host buffers: each step also
          copies level[] and parent[] (8n bytes) back to pinned host memory
          (double-buffered: a step's copy-out overlaps the next step's search).
roofline: algorithmic bytes per search from the search's own per-level
          counters (paper_1705_04590_gb300.roofline) / measured duration,
          against the measured HBM copy bandwidth (MEASURED_PEAKS.json).
cpu_baseline: the serial CPU oracle (Algorithm 1) on 4 roots of the headline graph
          itself (the device CSR copied to host: the parity tests prove it equal
          to the oracle's), one search per host core; cpu_multithreaded: the
          multithreaded direction-optimizing CPU BFS (the paper's in-node
          algorithm, OpenMP) on the same roots with every host thread.
tuned:   the autotuner's options (alpha, beta, hub cut-off, top-down chunk,
          CTAs per SM, cluster size) on 4 sample roots, timed over the same steps.
batched: 64-lane multi-source search (R-MAT 22, 64 roots, one launch) and an
          uneven batch of 256 graphs (one multi-root launch over their union),
          each against looping the plain single-source search.
served:  continuous-batching server over 8 resident graphs; the sustained
          capacity is the highest Poisson rate it keeps up with (>= 97 % served,
          p99 under half the 100 ms target over 1000 queries); Poisson arrivals at
          0.25/0.5/0.9 of it, p50/p99 latency (also per graph) and GTEPS, against a
          one-at-a-time plain FIFO on the same trace.
configs: R-MAT 24 over CSR (hub-first and id-ordered rows) and DCSC tiles, each
          direction-optimizing / top-down only / bottom-up only, and as a directed
          graph (out-rows top-down, their transpose bottom-up); Erdos-Renyi
          n = 2^26; the 4096^2 torus; a Twitter-sized power-law graph (61.5 M
          vertices, 1.47 B edges): a few roots each, GTEPS and roofline.

--impl reference times the oracle alone on the headline graph (built by the oracle),
one whole search per step, one search per host core at a time.
Multi-GPU (torchrun): replicas only -- each rank searches its own copy of the
graph from its own roots; no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "bfs_single_kernel_traffic.json")
KERNEL_SOURCES = ["paper_1705_04590_gb300/csrc/bfs_single.cu", "paper_1705_04590_gb300/csrc/bfs_common.cuh"]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={CLOCK_QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "of measured"}
    return {"hbm_gbs": 6800.0, "source": "of fallback"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ replicas (multi-GPU, no data-path collective)

def replica_roots(roots_all: list, rank: int) -> list:
    """Rank r cycles through the same roots starting at root r, so replicas search
    different roots at any moment while every rank's steps cover the same set."""
    k = rank % len(roots_all)
    return roots_all[k:] + roots_all[:k]


def max_over_ranks(ms: float, ws: int, device: str = "cuda") -> float:
    """Timed-region length of the job: the slowest rank's (all_reduce MAX)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gteps(ws: int, steps: int, m: int, total_ms: float) -> float:
    """Whole-job throughput: every rank ran `steps` searches of m edges in total_ms."""
    return ws * steps * m / (total_ms / 1e3) / 1e9


def e2e_pipelined(g, roots, opts, n: int, steps: int, stream, copy_streams: int = 4) -> float:
    """Milliseconds for `steps` searches whose outputs (level, parent: 8n bytes) reach
    pinned host memory; double-buffered device outputs, copies on `copy_streams` streams."""
    import torch
    dev = [(torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"))
           for _ in range(2)]
    host = [(torch.empty(n, dtype=torch.int32, pin_memory=True), torch.empty(n, dtype=torch.int32, pin_memory=True))
            for _ in range(2)]
    cs = [torch.cuda.Stream() for _ in range(copy_streams)]
    copied = [None, None]          # per output set: events of its last copy-out, one per copy stream
    torch.cuda.synchronize()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    for i in range(steps):
        j = i % 2
        if copied[j] is not None:
            for e in copied[j]:
                stream.wait_event(e)      # this set's previous results have left the device
        lv, pa = dev[j]
        g.run(roots[i % len(roots)], parent=pa, level=lv, opts=opts, stream=stream)
        done = torch.cuda.Event()
        done.record(stream)
        evs = []
        for k, c in enumerate(cs):
            c.wait_event(done)
            lo, hi = n * k // len(cs), n * (k + 1) // len(cs)
            with torch.cuda.stream(c):
                host[j][0][lo:hi].copy_(lv[lo:hi], non_blocking=True)
                host[j][1][lo:hi].copy_(pa[lo:hi], non_blocking=True)
            e = torch.cuda.Event()
            e.record(c)
            evs.append(e)
        copied[j] = evs
    for evs in copied:
        for e in evs or []:
            stream.wait_event(e)
    eb.record(stream)
    torch.cuda.synchronize()
    return ea.elapsed_time(eb)


# ------------------------------------------------------------------ CPU oracle (baseline / reference arm)

def host_cpu() -> dict:
    """nproc and the CPU model of this host (for the CPU lines)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu part", "hardware"):
                    model = model or line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "model": model}


def oracle_parallel(offsets, cols, roots, threads: int):
    """Serial Algorithm 1 (the oracle, as it stands), one search per host thread, all
    `roots` through a pool of `threads` (the C oracle releases the interpreter lock).
    Returns (wall seconds, per-search seconds)."""
    import concurrent.futures as cf
    import oracle
    ref = oracle.CSR(len(offsets) - 1, offsets, cols)

    def one(r):
        t0 = time.perf_counter()
        oracle.bfs_topdown(ref, r)
        return time.perf_counter() - t0

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(threads) as ex:
        per = list(ex.map(one, roots))
    return time.perf_counter() - t0, per


def cpu_baselines(g, roots, m: int, alpha: int, beta: int) -> tuple[dict, dict]:
    """CPU comparators on the headline graph itself.  Its CSR is copied from the device
    (the parity tests prove it equal, bit for bit, to the oracle's own CSR of the same
    edges), then (1) the serial oracle runs 4 roots, one per host core, and (2) the
    multithreaded direction-optimizing CPU BFS runs 4 roots on every core."""
    import cpubfs
    off, cols = g.csr_host()
    cpu = host_cpu()
    k = min(4, len(roots))
    wall, per = oracle_parallel(off, cols, roots[:k], k)
    oracle_line = {"value": k * m / wall / 1e9, "unit": "GTEPS", "cores": k, "kind": "oracle",
                   "per_core_gteps": float(k / sum(p for p in per) * m / 1e9),
                   "sample": f"serial Algorithm 1 (the oracle) on {k} roots of this graph, one search per host core "
                             f"at a time ({sum(per):.1f} s of CPU work); graph = the device CSR copied to host",
                   "nproc": cpu["nproc"], "cpu_model": cpu["model"]}
    cpubfs.build()
    times, dups = [], 0
    for r in roots[:k]:
        t0 = time.perf_counter()
        _, _, st = cpubfs.dobfs(off, cols, r, alpha=alpha, beta=beta)
        times.append(time.perf_counter() - t0)
        dups += st["duplicates"]
    mt_line = {"value": k * m / sum(times) / 1e9, "unit": "GTEPS", "cores": cpu["nproc"],
               "kind": "multithreaded direction-optimizing BFS (OpenMP, the paper's in-node algorithm)",
               "sample": f"{k} roots of this graph, one search at a time on all {cpu['nproc']} host threads",
               "ms_per_search": [round(t * 1e3, 1) for t in times], "duplicate_insertions": dups,
               "cpu_model": cpu["model"]}
    del off, cols
    return oracle_line, mt_line


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload != "rmat" or args.layout != "csr" or args.mode != "do":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the default workload "
                          "(R-MAT, CSR, direction-optimizing) only"}), flush=True)
        return 0
    import oracle
    from graphgen import workloads
    oracle.build()
    w = workloads.RMAT[args.scale]
    e = w.edges()
    roots = w.roots(e, args.roots).tolist()
    t0 = time.perf_counter()
    ref = oracle.build_csr(e.n, e.src, e.dst)
    build_s = time.perf_counter() - t0
    del e
    m = ref.nnz // 2
    cpu = host_cpu()
    threads = max(1, min(args.steps, cpu["nproc"] or 1))
    oracle_parallel(ref.offsets, ref.cols, [roots[i % len(roots)] for i in range(args.warmup)], threads)
    wall, per = oracle_parallel(ref.offsets, ref.cols, [roots[i % len(roots)] for i in range(args.steps)], threads)
    value = args.steps * m / wall / 1e9
    sample = (f"serial Algorithm 1 (the oracle, as it stands) on the R-MAT scale-{args.scale} graph itself "
              f"(oracle-built CSR, {build_s:.0f} s untimed), one whole search per step, {args.steps} steps through "
              f"{threads} host threads (one search per core at a time), roots cycled over {len(roots)}")
    line = {"impl": "reference", "metric": metric_name(args, w), "value": value,
            "unit": "GTEPS", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"{w.name} single-source BFS, {len(roots)} roots cycled",
                       "n": ref.n, "nnz": ref.nnz, "undirected_edges": m},
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": threads, "kind": "oracle", "sample": sample,
                             "per_search_s_mean": float(sum(per) / len(per)), "nproc": cpu["nproc"],
                             "cpu_model": cpu["model"]},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ batched / served sections

def _events(stream):
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def batched_section(seed: int = 4242, hub: bool = True) -> dict:
    """Batched multi-source BFS against looping the plain search.

    (i)  R-MAT scale 22, 64 roots: one bfs_run_multi (64 lanes, one persistent
         launch) vs 64 bfs_run, levels only, CUDA events, best of 3; again with
         both arms tuned (the autotuner for the plain arm, a grid over the
         direction thresholds for the multi-source launch).
    (ii) 256 R-MAT graphs with scales drawn uniformly from 10..20 (seeded), one
         root each: one bfs_run_multiroot over their disjoint union (one
         launch) vs a loop of 256 plain searches on the separate graphs.
    """
    import numpy as np
    import torch

    import graphgen
    import paper_1705_04590_gb300 as bfs
    from graphgen import workloads

    out = {}
    w = workloads.RMAT[22]
    e = w.edges()
    roots = w.roots(e, 64).tolist()
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, hub_first=hub)
    n, m = e.n, g.nnz // 2
    del e
    lv1 = torch.empty(n, dtype=torch.int32, device="cuda")
    lvk = torch.empty(64 * n, dtype=torch.int32, device="cuda")
    # both arms scan the same rows bottom-up
    o = bfs.options(bu_rows=bfs.BU_ROWS_HUB_FIRST if hub else bfs.BU_ROWS_BY_ID)

    def best_ms(fn, reps=3):
        best = None
        for _ in range(reps + 1):
            a, b = _events(None)
            torch.cuda.synchronize()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b)
            best = t if best is None else min(best, t)
        return best

    t_multi = best_ms(lambda: g.run_multi(roots, lvk, opts=o))
    t_plain = best_ms(lambda: [g.run(r, level=lv1, opts=o) for r in roots])
    g.sync()
    out["rmat22_64roots"] = {"multi_ms": t_multi, "plain_ms": t_plain, "multi_gteps": 64 * m / t_multi / 1e6,
                             "plain_gteps": 64 * m / t_plain / 1e6, "speedup": t_plain / t_multi,
                             "launches_multi": 1, "launches_plain": 64}
    # both arms tuned: the plain arm with the autotuner's choice on 4 of the roots (every
    # plain-search knob), the multi-source launch with the direction thresholds that time
    # best for it over the same grid (its levels count 64 lanes, so its best thresholds differ)
    from paper_1705_04590_gb300 import autotune
    ot, _ = autotune.autotune(g, roots[:4], base=o)
    t_plain_t = best_ms(lambda: [g.run(r, level=lv1, opts=ot) for r in roots])
    grid_ab = [(a_, b_) for a_ in (6, 14, 24, 32, 96) for b_ in (12, 24, 64, 128)]
    tm = {ab: best_ms(lambda ab=ab: g.run_multi(roots, lvk, opts=bfs.options(bu_rows=o.bu_rows, alpha=ab[0],
                                                                              beta=ab[1])), reps=1)
          for ab in grid_ab}
    am, bm = min(tm, key=tm.get)
    t_multi_t = best_ms(lambda: g.run_multi(roots, lvk, opts=bfs.options(bu_rows=o.bu_rows, alpha=am, beta=bm)))
    g.sync()
    out["rmat22_64roots_tuned"] = {"plain": {"alpha": ot.alpha, "beta": ot.beta, "td_big_degree": ot.td_big_degree,
                                             "td_chunk": ot.td_chunk, "ctas_per_sm": ot.ctas_per_sm,
                                             "cluster_size": ot.cluster_size},
                                   "multi": {"alpha": am, "beta": bm}, "multi_ms": t_multi_t, "plain_ms": t_plain_t,
                                   "speedup": t_plain_t / t_multi_t}
    g.close()
    del lvk
    rng = np.random.default_rng(seed)
    scales = rng.integers(10, 21, 256)
    parts = [graphgen.rmat(int(sc), seed=50_000 + i) for i, sc in enumerate(scales)]
    u, offs = graphgen.disjoint_union(parts)
    uroots = [int(offs[i]) + int(graphgen.pick_roots(pp, 1, 7 + i)[0]) for i, pp in enumerate(parts)]
    gu = bfs.Graph.from_edges(u.src, u.dst, u.n)
    gs = [bfs.Graph.from_edges(pp.src, pp.dst, pp.n) for pp in parts]
    mu = gu.nnz // 2
    lu = torch.empty(u.n, dtype=torch.int32, device="cuda")
    bufs = [torch.empty(pp.n, dtype=torch.int32, device="cuda") for pp in parts]
    t_union = best_ms(lambda: gu.run_multiroot(uroots, level=lu))
    t_loop = best_ms(lambda: [gg.run(uroots[i] - int(offs[i]), level=bufs[i]) for i, gg in enumerate(gs)])
    out["uneven_256_graphs"] = {"scales": "U{10..20} seed %d" % seed, "vertices": int(u.n), "undirected_edges": mu,
                                "union_ms": t_union, "loop_ms": t_loop, "union_gteps": mu / t_union / 1e6,
                                "loop_gteps": mu / t_loop / 1e6, "speedup": t_loop / t_union}
    for gg in gs:
        gg.close()
    gu.close()
    return out


def time_searches(g, roots, opts, n: int, reps: int = 1):
    """Device time of one search per root (CUDA events around each), levels and parents
    written; returns (per-search ms list, records of each root from an untimed pass)."""
    import torch
    from paper_1705_04590_gb300 import roofline
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    bytes_of = []
    for r in roots:
        info = g.run(r, parent=parent, level=level, opts=opts, stats=True, record_levels=8192)
        bytes_of.append(roofline.search_bytes(n, info["records"]))
    g.run(roots[0], parent=parent, level=level, opts=opts)
    ms = []
    for _ in range(reps):
        for r in roots:
            a, b = _events(None)
            torch.cuda.synchronize()
            a.record()
            g.run(r, parent=parent, level=level, opts=opts)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
    return ms, bytes_of * reps


def configs_section(peak_gbs: float) -> dict:
    """Configurations 2 and 3 besides the headline, a few seeded roots each: R-MAT scale
    24 over CSR and over DCSC column-block tiles, each direction-optimizing, top-down
    only and bottom-up only; Erdos-Renyi n = 2^26 (E[deg] 16); the 4096 x 4096 torus.
    GTEPS = edges x searches / summed device time (the harmonic mean over roots);
    roofline = the byte model over each search's own level records."""
    import numpy as np

    import paper_1705_04590_gb300 as bfs
    from graphgen import workloads

    out = {}

    def line(name, g, roots, opts, n, m, reps=1):
        ms, by = time_searches(g, roots, opts, n, reps)
        t = sum(ms)
        out[name] = {"gteps": len(ms) * m / t / 1e6, "ms_per_search": t / len(ms), "roots": len(roots),
                     "roofline_frac": sum(by) / (t / 1e3) / 1e9 / peak_gbs, "p99_ms": float(np.percentile(ms, 99))}

    w = workloads.RMAT[24]
    e = w.edges()
    roots = w.roots(e, 4).tolist()
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, dcsc=True, hub_first=True)
    n, m = e.n, g.nnz // 2
    del e
    for mode, mname in ((bfs.MODE_DO, "do"), (bfs.MODE_TD_ONLY, "td"), (bfs.MODE_BU_ONLY, "bu")):
        line(f"rmat24_csr_{mname}", g, roots, bfs.options(mode=mode, bu_rows=bfs.BU_ROWS_HUB_FIRST), n, m)
        line(f"rmat24_csr_idrows_{mname}", g, roots, bfs.options(mode=mode), n, m)
        line(f"rmat24_dcsc_{mname}", g, roots[:2], bfs.options(mode=mode, layout=bfs.LAYOUT_DCSC_TILED), n, m)
    # the two layouts' sizes: CSR offsets + ids against the p x p tiles' pointers, JC, CP and IR
    d = g.dcsc_layout()
    p2 = d.num_blocks * d.num_blocks
    out["rmat24_dcsc_do"]["layout_bytes"] = {"csr": 8 * (n + 1) + 4 * g.nnz,
                                             "dcsc": 8 * (p2 + 1) + 4 * d.nzc + 8 * (d.nzc + 1) + 4 * g.nnz,
                                             "tiles": p2, "nzc": d.nzc, "nnz": g.nnz}
    g.close()
    # the same R-MAT edges as a directed graph (edge i: src -> dst; top-down over out-rows,
    # bottom-up over their transpose); GTEPS over its directed edge count
    e = w.edges()
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, directed=True)
    n, md = e.n, g.nnz
    del e
    line("rmat24_directed_do", g, roots, bfs.options(), n, md)
    out["rmat24_directed_do"]["directed_edges"] = md
    g.close()
    e = workloads.ER26.edges()
    roots = workloads.ER26.roots(e, 8).tolist()
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, hub_first=True)
    n, m = e.n, g.nnz // 2
    del e
    line("er26_do", g, roots, bfs.options(bu_rows=bfs.BU_ROWS_HUB_FIRST), n, m)
    g.close()
    e = workloads.TORUS4096.edges()
    roots = workloads.TORUS4096.roots(e, 4).tolist()
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, hub_first=True)
    n, m = e.n, g.nnz // 2
    del e
    line("torus4096_do", g, roots, bfs.options(bu_rows=bfs.BU_ROWS_HUB_FIRST), n, m)
    g.close()
    # the paper's real-world graph has Twitter's size: a seeded power-law stand-in of that size
    w = workloads.TWITTERLIKE
    e = w.edges()
    roots = w.roots(e, 8).tolist()
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, hub_first=True)
    n, m = e.n, g.nnz // 2
    del e
    line("twitterlike_do", g, roots, bfs.options(bu_rows=bfs.BU_ROWS_HUB_FIRST), n, m)
    out["twitterlike_do"]["graph"] = {"n": n, "undirected_edges": m, "generated_edges": 1_470_000_000}
    g.close()
    return out


def keeps_pace(arrivals, served_qps: float, p99_ms: float, p99_target_ms: float) -> bool:
    """Whether a server run kept up with a Poisson trace: it served at least 97 % of the
    trace's own arrival rate (k queries over the span of their arrival times; a Poisson trace
    spans k / rate only on average) with a p99 under half the target."""
    k = len(arrivals)
    realized = (k - 1) / max(float(arrivals[-1]) - float(arrivals[0]), 1e-9)
    return served_qps >= 0.97 * realized and p99_ms <= 0.5 * p99_target_ms


def served_section(g26, roots26, n_queries: int = 2000, seed: int = 5151) -> dict:
    """Served BFS: 8 resident graphs (R-MAT 16, 18, 20, 22, 24, 25, 26 and the
    4096x4096 torus), queries = (graph uniform over the 8, seeded root), each
    returning level[] into pinned host memory.  The saturated throughput is
    measured with a burst; then Poisson arrivals at 0.25, 0.5 and 0.9 of it,
    n_queries each, through the continuous-batching server and through a
    one-at-a-time plain FIFO (bfs_run + copy-out) on the same trace.
    Latency = submit -> result in host memory."""
    import numpy as np
    import torch

    import paper_1705_04590_gb300 as bfs
    from graphgen import workloads

    specs = [("rmat16", workloads.RMAT[16]), ("rmat18", workloads.RMAT[18]), ("rmat20", workloads.RMAT[20]),
             ("rmat22", workloads.RMAT[22]), ("rmat24", workloads.RMAT[24]), ("rmat25", workloads.RMAT[25]),
             ("rmat26", None), ("torus4096", workloads.TORUS4096)]
    graphs, rootsets, ms = [], [], []
    for name, wl in specs:
        if wl is None:
            g, rs = g26, roots26
        else:
            e = wl.edges()
            rs = wl.roots(e, 64).tolist()
            g = bfs.Graph.from_edges(e.src, e.dst, e.n)
            del e
        graphs.append(g)
        rootsets.append(rs)
        ms.append(g.nnz // 2)
    # client-side result buffers per graph: enough that a graph's 64 lanes can all be busy
    pool_size = [128 if g.n < (1 << 24) else 64 for g in graphs]
    pinned = [[torch.empty(g.n, dtype=torch.int32, pin_memory=True) for _ in range(k)]
              for g, k in zip(graphs, pool_size)]
    pools = [[t.numpy() for t in pl] for pl in pinned]
    srv = bfs.Server(hbm_budget_bytes=96 << 30, max_lanes=64)
    slots = [srv.add_graph(g) for g in graphs]
    rng = np.random.default_rng(seed)

    def trace(k):
        gi = rng.integers(0, len(graphs), k)
        ri = rng.integers(0, 64, k)
        return [(int(a), rootsets[int(a)][int(b)]) for a, b in zip(gi, ri)]

    def run_server(tr, arrivals):
        free = [list(range(len(pl))) for pl in pools]
        inflight = []    # (ticket, graph, buffer index)
        lat, lat_g, done_m = [], [], 0
        submitted = 0
        t0 = time.perf_counter()
        for (gi, root), at in zip(tr, arrivals):
            while time.perf_counter() - t0 < at:
                pass
            while not free[gi]:
                # buffer pool of this graph exhausted: retire the oldest in-flight query of that graph
                for idx, (tk, gj, bi) in enumerate(inflight):
                    if gj == gi:
                        if not srv.wait(tk, 300_000):
                            raise RuntimeError("served query did not complete within 300 s")
                        lat.append(srv.latency_us(tk))
                        lat_g.append(gj)
                        done_m += ms[gj]
                        free[gj].append(bi)
                        inflight.pop(idx)
                        break
            bi = free[gi].pop()
            inflight.append((srv.submit(slots[gi], root, pools[gi][bi]), gi, bi))
            submitted += 1
            # retire finished queries now and then (polling every ticket on every
            # submission would make this client loop, not the server, the bottleneck)
            if submitted % 32 == 0 or not free[gi]:
                keep = []
                for tk, gj, bj in inflight:
                    if srv.poll(tk):
                        lat.append(srv.latency_us(tk))
                        lat_g.append(gj)
                        done_m += ms[gj]
                        free[gj].append(bj)
                    else:
                        keep.append((tk, gj, bj))
                inflight = keep
        for tk, gj, bj in inflight:
            if not srv.wait(tk, 300_000):
                raise RuntimeError("served query did not complete within 300 s")
            lat.append(srv.latency_us(tk))
            lat_g.append(gj)
            done_m += ms[gj]
        wall = time.perf_counter() - t0
        lat = np.array(lat) / 1e3
        lat_g = np.array(lat_g)
        by_graph = {specs[i][0]: round(float(np.percentile(lat[lat_g == i], 99)), 2)
                    for i in range(len(graphs)) if (lat_g == i).any()}
        return {"wall_s": wall, "qps": len(tr) / wall, "gteps": done_m / wall / 1e9,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "p99_ms_by_graph": by_graph}

    def run_fifo(tr, arrivals):
        lvs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in graphs]
        lat, done_m = [], 0
        t0 = time.perf_counter()
        for (gi, root), at in zip(tr, arrivals):
            while time.perf_counter() - t0 < at:
                pass
            graphs[gi].run(root, level=lvs[gi])
            pinned[gi][0].copy_(lvs[gi], non_blocking=True)
            torch.cuda.synchronize()
            lat.append((time.perf_counter() - t0 - at) * 1e3)
            done_m += ms[gi]
        wall = time.perf_counter() - t0
        lat = np.array(lat)
        return {"wall_s": wall, "qps": len(tr) / wall, "gteps": done_m / wall / 1e9,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}

    # warm-up and saturated throughput: a burst of queries all at time 0 (its p99 is a queue
    # of 1024 queries draining, reported on its own)
    run_server(trace(256), np.zeros(256))
    sat = run_server(trace(1024), np.zeros(1024))
    # the sustained capacity: the highest Poisson rate (searched from below the burst's) at
    # which the server keeps up, i.e. serves >= 97 % of the offered rate with a p99 under
    # half the target over 1000 queries (the margin keeps the longer runs at the offered
    # loads under the target); the offered loads are fractions of it
    p99_target_ms = 100.0
    probes = []

    def keeps_up(rate, k=1000):
        tr = trace(k)
        arr = np.cumsum(rng.exponential(1.0 / rate, k))
        arr -= arr[0]
        r = run_server(tr, arr)
        ok = keeps_pace(arr, r["qps"], r["p99_ms"], p99_target_ms)
        probes.append({"offered_qps": rate, "served_qps": r["qps"], "p99_ms": r["p99_ms"], "keeps_up": ok})
        return ok

    lo, hi = 0.0, None
    rate = 0.5 * sat["qps"]
    for _ in range(6):
        if keeps_up(rate):
            lo = rate
            rate = rate * 1.3 if hi is None else 0.5 * (rate + hi)
        else:
            hi = rate
            rate = 0.5 * (lo + rate) if lo > 0 else 0.5 * rate
    capacity = lo if lo > 0 else 0.25 * sat["qps"]
    out = {"graphs": [nme for nme, _ in specs], "saturated": sat, "sustained_capacity_qps": capacity,
           "p99_target_ms": p99_target_ms, "capacity_probes": probes, "loads": []}
    for frac in (0.25, 0.5, 0.9):
        rate = frac * capacity
        tr = trace(n_queries)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n_queries))
        arrivals -= arrivals[0]
        sv = run_server(tr, arrivals)
        fi = run_fifo(tr, arrivals)
        out["loads"].append({"offered_frac": frac, "offered_qps": rate, "served": sv, "plain_fifo": fi,
                             "gteps_ratio": sv["gteps"] / fi["gteps"]})
    st = srv.stats()
    out["server_counters"] = st
    srv.close()
    for g in graphs:
        if g is not g26:
            g.close()
    return out


# ------------------------------------------------------------------ our arm

def metric_name(args, w) -> str:
    what = {"do": "direction-optimizing", "td": "top-down only", "bu": "bottom-up only"}[args.mode]
    graph = {"rmat": f"R-MAT scale {args.scale}", "er": f"Erdos-Renyi n=2^{args.scale} deg 16",
             "torus": "4096x4096 torus",
             "twitterlike": "Twitter-sized power-law graph (61.5M vertices, 1.47B edges)"}[args.workload]
    lay = ", DCSC tiles" if args.layout == "dcsc" else ""
    return f"GTEPS harmonic mean, {graph}, 1 GB300 (single-source, {what}{lay})"


def our_arm(args):
    import numpy as np
    import torch

    import paper_1705_04590_gb300 as bfs
    from graphgen import workloads
    from paper_1705_04590_gb300 import roofline

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    bfs.build()
    bfs.load()

    if args.workload == "er":
        w = workloads.Workload("er", args.scale)
    elif args.workload == "torus":
        w = workloads.TORUS4096
    elif args.workload == "twitterlike":
        w = workloads.TWITTERLIKE
    else:
        w = workloads.RMAT[args.scale]
    t0 = time.time()
    e = w.edges()
    roots_all = w.roots(e, args.roots).tolist()
    hub = args.bu_rows == "hub" and args.layout == "csr"
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, dcsc=(args.layout == "dcsc"), hub_first=hub)
    n = e.n
    del e
    setup_s = time.time() - t0
    m = g.nnz // 2
    roots = replica_roots(roots_all, rank)
    mode = {"do": bfs.MODE_DO, "td": bfs.MODE_TD_ONLY, "bu": bfs.MODE_BU_ONLY}[args.mode]
    layout = bfs.LAYOUT_DCSC_TILED if args.layout == "dcsc" else bfs.LAYOUT_CSR
    opts = bfs.options(mode=mode, layout=layout, alpha=14, beta=24,
                       bu_rows=bfs.BU_ROWS_HUB_FIRST if hub else bfs.BU_ROWS_BY_ID)
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    # per-root algorithmic bytes from the search's own counters (untimed pass)
    bytes_of = {}
    levels_of = {}
    for r in roots:
        info = g.run(r, parent=parent, level=level, opts=opts, stats=True, record_levels=4096)
        bytes_of[r] = roofline.search_bytes(n, info["records"])
        levels_of[r] = info["num_levels"]

    for i in range(args.warmup):
        g.run(roots[i % len(roots)], parent=parent, level=level, opts=opts)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    evs[0].record(stream)
    for i in range(args.steps):
        g.run(roots[i % len(roots)], parent=parent, level=level, opts=opts)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    g.sync()
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    total_ms = max_over_ranks(total_ms, ws)
    value = aggregate_gteps(ws, args.steps, m, total_ms)
    alg_bytes = sum(bytes_of[roots[i % len(roots)]] for i in range(args.steps))
    achieved = alg_bytes / (sum(step_ms) / 1e3) / 1e9
    peaks = measured_peaks()

    # end to end: the same searches through the public API with level[] and parent[] copied
    # to pinned host memory every step.  Two output sets alternate, so that step i's copy-out
    # (split over several copy streams) overlaps step i+1's search; the timed region ends when
    # the last copy has landed.
    e2e_steps = min(args.steps, 64)
    e2e_ms = e2e_pipelined(g, roots, opts, n, e2e_steps, stream)
    e2e_value = aggregate_gteps(ws, e2e_steps, m, max_over_ranks(e2e_ms, ws))

    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        with open(TRAFFIC_FILE) as f:
            tr = json.load(f)
        if tr.get("kernel_source_hash") == kernel_source_hash() and tr.get("workload") == w.name \
                and args.layout == "csr" and args.mode == "do" and tr.get("bu_rows", "id") == args.bu_rows:
            traffic = tr.get("dram_bytes_per_launch")

    # the autotuner's choice (direction thresholds, hub cut-off, top-down chunk, CTAs per
    # SM, cluster size) on 4 sample roots, timed over the same steps as the headline
    tuned = None
    if rank == 0 and not args.no_tuned and args.layout == "csr":
        from paper_1705_04590_gb300 import autotune
        best, _ = autotune.autotune(g, roots[:4], base=opts)
        t_ms, t_bytes = time_searches(g, [roots[i % len(roots)] for i in range(args.steps)], best, n)
        tuned = {"alpha": best.alpha, "beta": best.beta, "td_big_degree": best.td_big_degree,
                 "td_chunk": best.td_chunk, "ctas_per_sm": best.ctas_per_sm, "cluster_size": best.cluster_size,
                 "value": args.steps * m / sum(t_ms) / 1e6, "unit": "GTEPS", "ms_per_step": sum(t_ms) / args.steps,
                 "roofline_frac": sum(t_bytes) / (sum(t_ms) / 1e3) / 1e9 / peaks["hbm_gbs"],
                 "note": "same roots and outputs as the headline, CUDA events per search; the headline keeps "
                         "the configured alpha 14 / beta 24"}

    batched = served = configs = None
    if rank == 0 and not args.no_batched:
        batched = batched_section(hub=(args.bu_rows == "hub"))
    if rank == 0 and not args.no_served:
        served = served_section(g, roots, n_queries=args.served_queries)

    cpu = cpu_mt = None
    if rank == 0 and not args.no_cpu_baseline and args.layout == "csr":
        cpu, cpu_mt = cpu_baselines(g, roots, m, 14, 24)

    if rank == 0:
        line = {
            "metric": metric_name(args, w),
            "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"{w.name} single-source BFS, {len(roots)} roots cycled",
                       "n": n, "nnz": g.nnz, "undirected_edges": m, "alpha": 14, "beta": 24,
                       "mode": args.mode, "layout": args.layout,
                       "bu_rows": ("hub-first (bottom-up scans rows ordered by neighbour degree; "
                                   "top-down uses the id-ordered rows)") if hub else "by id",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "l2": "inputs larger than L2 (graph resident in HBM, %.1f GB)" % (g.device_bytes() / 1e9),
                       "levels_per_search": float(np.mean([levels_of[r] for r in roots])),
                       "setup_s": round(setup_s, 1)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                         "peak_source": peaks["source"],
                         "kernel": "bfs_dcsc_kernel" if args.layout == "dcsc" else "bfs_single_kernel",
                         "algorithmic_bytes_per_search": alg_bytes / args.steps},
            "e2e": {"value": e2e_value, "unit": "GTEPS", "h2d_bytes_per_step": 4, "d2h_bytes_per_step": 8 * n,
                    "steps": e2e_steps},
            "gpu_launches": args.steps,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "cpu_multithreaded": cpu_mt,
            "tuned": tuned,
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "batched": batched,
            "served": served,
        }
        if not args.no_configs and args.workload == "rmat" and args.scale == 26:
            g.close()
            g = None
            line["configs"] = configs_section(peaks["hbm_gbs"])
        print(json.dumps(line), flush=True)
    if g is not None:
        g.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=26, help="R-MAT scale, or log2 n for --workload er")
    ap.add_argument("--workload", default="rmat", choices=["rmat", "er", "torus", "twitterlike"])
    ap.add_argument("--layout", default="csr", choices=["csr", "dcsc"])
    ap.add_argument("--mode", default="do", choices=["do", "td", "bu"])
    ap.add_argument("--bu-rows", default="hub", choices=["hub", "id"],
                    help="row order of the bottom-up scans: hub-first copy (default) or the id-sorted rows")
    ap.add_argument("--roots", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched multi-source section")
    ap.add_argument("--no-served", action="store_true", help="skip the served section")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the configurations besides the headline (R-MAT 24 CSR/DCSC x DO/TD/BU, ER 2^26, torus)")
    ap.add_argument("--no-tuned", action="store_true", help="skip the autotuned line")
    ap.add_argument("--served-queries", type=int, default=2000, help="queries per offered load")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    return our_arm(args)


if __name__ == "__main__":
    sys.exit(main())
