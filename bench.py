#!/usr/bin/env python3
"""Polar stroking hot path on GB300: stroked segments/s and covered samples/s.

Workload (the configuration the metric is quoted on): 10,000 open paths of mixed
line / quadratic / cubic / conic segments (mean 30 segments, max 200), 20% of the
cubics exact cusps or loops, widths 0.5-64 px, miter/round/bevel joins and
butt/square/round caps, dtheta = 1 degree, rasterized at 2048x2048 with 16
samples per pixel; synthetic, seeded.

One step = the whole hot path over the batch: link setup and rib offsets,
rib emission (t(psi) solve, vertices, joins, caps), cumulative arc length,
tile binning and 16-sample per-path coverage.  The batched variant captures the
step's launches in one CUDA graph; the plain variant runs one path per launch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank strokes its own share of
the job, a batch of the workload seeded per rank (weak scaling, no collective on
the data path); the timed region is bracketed by barriers and the maximum over
ranks is reported.  (One batch split over ranks by links, with its one exchange of
rib counts and lengths, is paper_2007_00308_gb300/shard.py with
ps_tessellate_links.)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "stroked segments/s and covered samples/s at 1 GB300: batched+mixed vs plain"
WORKLOAD = ("c2 batching: 10,000 paths, segments/path geometric (mean 30, max 200), "
            "20% line / 20% quadratic / 45% cubic / 15% conic (w_B log-uniform 0.1-10), "
            "20% of cubics exact cusps or loops, widths log-uniform 0.5-64 px, "
            "miter(4)/round/bevel joins, butt/square/round caps, dtheta 1 deg, "
            "2048x2048 at 16 samples/pixel")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-paths", type=int, default=10000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--exact", action="store_true",
                    help="rasterize quads as polygons (bow-ties as such) instead of two triangles")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch parameters (profiling runs)")
    ap.add_argument("--pixel-tol", type=float, default=0.0,
                    help="pixel-scale boost of the angle step per link, tolerance in px "
                         "(0, the default, keeps the configured dtheta everywhere)")
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "facet"],
                    help="c2 (default) is the configuration the metric is quoted on; the "
                         "others print their own line for the per-configuration table")
    return ap.parse_args()


# ---------------------------------------------------------------------------
def max_over_ranks(value: float, device) -> float:
    """Maximum of a per-rank scalar over the process group (the slowest rank's
    timed region bounds the whole job's throughput)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


PG_TIMEOUT_S = 300


def job_throughput(units_per_rank: int, world: int, max_ms: float) -> float:
    """Whole-job units/s: every rank processes its own batch (weak scaling)."""
    return world * units_per_rank / (max_ms * 1e-3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
def oracle_sample(batch, paths):
    """FP64 oracle on a subset of paths: tessellation + arc length + coverage."""
    import numpy as np
    import oracle
    sub = batch.subset(paths)
    t0 = time.perf_counter()
    o = oracle.tessellate(sub)
    oracle.raster(o["rib"], o["tag"], batch.canvas[0], batch.canvas[1], sub.n_path)
    return time.perf_counter() - t0, int(sub.n_seg)


def _oracle_chunk(job):
    """Worker of the all-core baseline (a spawned process): one chunk of paths."""
    batch, paths = job
    return oracle_sample(batch, paths)


def host_cpu():
    """The host's logical CPU count and CPU model (from /proc/cpuinfo or lscpu)."""
    model = ""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.strip().lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown"}


def cpu_baseline(batch, budget_s=12.0):
    """The FP64 oracle as it stands on random paths of the workload: single
    thread, then one spawned process per available core taking chunks of 25
    paths (processes, not threads: the oracle keeps static buffers)."""
    import multiprocessing as mp
    import numpy as np
    rng = np.random.default_rng(0)
    order = rng.permutation(batch.n_path)
    spent, segs, k = 0.0, 0, 0
    while spent < budget_s and k < len(order):
        chunk = order[k:k + 25]
        dt, n = oracle_sample(batch, chunk)
        spent += dt
        segs += n
        k += len(chunk)
    single = segs / spent
    host = host_cpu()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    jobs = [(batch.subset(order[i:i + 25]), None) for i in range(0, len(order), 25)]
    jobs = [(b, np.arange(b.n_path)) for b, _ in jobs]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_chunk, jobs[:cores])  # start-up (imports, oracle load) untimed
        t0 = time.perf_counter()
        asegs, done = 0, 0
        for dt, n in pool.imap_unordered(_oracle_chunk, jobs[cores:]):
            asegs += n
            done += 1
            if time.perf_counter() - t0 > budget_s:
                break
        wall = time.perf_counter() - t0
        pool.terminate()
    return {"value": asegs / wall, "unit": "segments/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} chunks of 25 random paths of the workload ({asegs} segments), FP64 "
                      f"tessellation + arc length + 16-sample raster, {cores} processes, "
                      f"{wall:.1f} s wall",
            "single_thread": {"value": single, "unit": "segments/s", "cores": 1,
                              "sample": f"{k} random paths ({segs} segments), {spent:.1f} s"},
            "host": host}


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle as it stands, on all host cores (one
    spawned process per core; each step is 4 chunks of 6 random paths per
    process, handed out one chunk at a time)."""
    if rank != 0:
        return 0
    import multiprocessing as mp
    from paper_2007_00308_gb300 import workloads as W
    import numpy as np
    batch = W.c2_batching(n_paths=args.n_paths)
    rng = np.random.default_rng(1)
    per_chunk, chunks_per_proc = 6, 4  # paths per step: keeps steps * warmup within minutes
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()

    def step_jobs():
        return [(batch.subset(rng.choice(batch.n_path, per_chunk, replace=False)), None)
                for _ in range(cores * chunks_per_proc)]

    def run(pool):
        jobs = [(b, np.arange(b.n_path)) for b, _ in step_jobs()]
        t0 = time.perf_counter()
        res = pool.map(_oracle_chunk, jobs, chunksize=1)
        return time.perf_counter() - t0, sum(n for _, n in res)

    with mp.get_context("spawn").Pool(cores) as pool:
        for _ in range(args.warmup):
            run(pool)
        total, segs = 0.0, 0
        for _ in range(args.steps):
            dt, n = run(pool)
            total += dt
            segs += n
    value = segs / total
    sample = (f"{cores * chunks_per_proc} chunks of {per_chunk} random paths per step, "
              f"{cores} processes, {args.steps} steps")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "segments/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "variant": "FP64 CPU oracle (reference arm), all cores",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": "segments/s", "cores": cores, "kind": "oracle",
                         "sample": sample, "host": host_cpu()},
        "e2e": {"value": value, "unit": "segments/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# Algorithmic work per launch of each kernel: the bytes the method itself must
# move for the HBM-class kernels, sample tests for the coverage kernel.  The
# tessellation stage reads 40 B per segment and 24 B per path and writes 16 B
# per rib (N, P), 4 B per rib (s) and 4 B per link (offset): 40S + 24P + 20R +
# 4L, split as link set-up 40S + 24P + 4L, emitter 16R, arc length 4R (the
# emitter hands each rib's chord to the scan through s).  Binning
# reads 16 B per rib once, writes 4 B per (quad, tile) entry and 4 B per tile
# offset: 16R + 4 pairs + 4 tiles, split as count 16R, tile scan 4 tiles,
# scatter 4 pairs.  The library's own workspace (per-link records, per-rib tags
# and chords, the binning passes' per-rib hit words) is not the method's work:
# it is listed per kernel as workspace_bytes (design figures, not measured
# traffic).
def algorithmic(kernel, c):
    R, L, S, P, pairs, tiles = c["R"], c["L"], c["S"], c["P"], c["pairs"], c["tiles"]
    table = {
        "k_link_setup": ("hbm", 40 * S + 24 * P + 4 * L),
        "k_emit": ("hbm", 16 * R),
        "k_arclen_scan": ("hbm", 4 * R),
        "k_bin_count": ("hbm", 16 * R),
        "k_tile_scan": ("hbm", 4 * tiles),
        "k_bin_scatter": ("hbm", 4 * pairs),
        "k_coverage": ("alu", 16 * c["span_px"]),
    }
    return table.get(kernel)


def workspace_bytes(kernel, c):
    """Bytes of the library's own workspace a kernel writes and reads (design
    figures): 240 B link records, 4 B tags and 4 B chords per rib, and the two
    4 B words per rib ({hits, box}) that the count pass leaves for the scatter
    pass (which re-reads ribs only for quads with more than 31 candidate
    tiles)."""
    R, L = c["R"], c["L"]
    return {"k_link_setup": 240 * L, "k_emit": 240 * L + 8 * R, "k_arclen_scan": 8 * R,
            "k_bin_count": 4 * R + 8 * R, "k_bin_scatter": 8 * R}.get(kernel, 0)


STAGES = {
    "tessellation": (("k_link_setup", "k_emit", "k_arclen_scan"),
                     lambda c: 40 * c["S"] + 24 * c["P"] + 20 * c["R"] + 4 * c["L"]),
    "binning": (("k_bin_count", "k_tile_scan", "k_bin_scatter"),
                lambda c: 16 * c["R"] + 4 * c["pairs"] + 4 * c["tiles"]),
}


def stage_report(kmean, c, hbm_peak):
    out = {}
    for name, (ks, fn) in STAGES.items():
        ms = sum(kmean.get(k, 0.0) for k in ks)
        if ms <= 0:
            continue
        b = fn(c)
        out[name] = {"kernels": list(ks), "ms": ms, "algorithmic_bytes": b,
                     "achieved_gbs": b / (ms * 1e-3) / 1e9,
                     "frac": b / (ms * 1e-3) / 1e9 / hbm_peak}
    return out


# ALU peak for the coverage kernel.  One sample test is one sample against one
# quad.  The branch-free masks step every edge value from sample to sample with
# one add, combine sign bits with three-input logic ops and shift the result's
# sign bit into the mask with one funnel shift: a convex quad (or single
# triangle) takes 4 adds + 2 logic ops + 1 shift, 7 lane ops; a non-convex quad
# (two triangles sharing the diagonal) 5 adds + 3 logic ops + 1 shift, 9 lane
# ops; the general path (edges over 1024 px) ~12.  The SM issues at most 128
# lane ops per clock (4 schedulers x 32 lanes).
OPS_PER_TEST = {"convex_pixels": 7.0, "two_triangle_pixels": 9.0, "general_pixels": 12.0}
# the crossing-rule mask (--exact): per sample and edge one add and one funnel
# shift of its sign bit, 4 edges (the y-range terms are per pixel); its int32
# form counts as "convex" pixels
OPS_PER_TEST_EXACT = {"convex_pixels": 8.0, "two_triangle_pixels": 8.0, "general_pixels": 24.0}


# Measured issue rates of the coverage mask's per-sample operation mixes on this
# GB300 (a microbenchmark of independent IADD/LOP3/SHF chains, 16 warps per
# scheduler, best of 2,000 launches, every sampled SM clock 2070 MHz): the
# convex step (4 adds, 2 logic ops, 1 funnel shift) ran 4.802 T sample tests/s,
# i.e. 106.8 lane ops per SM per clock; the two-triangle step (5 + 3 + 1)
# 3.668 T tests/s, 104.9 lane ops per SM per clock.  Each INT op class alone
# issues 63 lane ops per SM per clock; the mixes co-issue on two pipes.  Per
# SM and clock:
MEASURED_TESTS_PER_SM_CLK = {"convex_pixels": 4.802e12 / (152 * 2.07e9),
                             "two_triangle_pixels": 3.668e12 / (152 * 2.07e9)}


def measured_peak_tests(rstat, sm_mhz, exact=False):
    """Peak sample tests/s of the coverage kernel's pixel-class mix from the
    measured issue rates (None for the crossing-rule mask, not measured): the
    harmonic mean of the class rates weighted by the classes' pixels, at the
    sampled SM clock.  The general (int64) class has no measurement and takes
    the derived rate."""
    if exact:
        return None
    n = sum(rstat.get(k, 0) for k in OPS_PER_TEST)
    if n <= 0:
        return None
    per_test = 0.0
    for k in OPS_PER_TEST:
        f = rstat.get(k, 0) / n
        rate = MEASURED_TESTS_PER_SM_CLK.get(k, 128.0 / OPS_PER_TEST[k])
        per_test += f / rate
    return 152 * sm_mhz * 1e6 / per_test


def ops_per_test(rstat, exact=False):
    table = OPS_PER_TEST_EXACT if exact else OPS_PER_TEST
    n = sum(rstat.get(k, 0) for k in table)
    if n <= 0:
        return table["general_pixels"]
    return sum(table[k] * rstat.get(k, 0) for k in table) / n


def alu_peak_tests(sm_mhz, ops):
    return 152 * 128 * sm_mhz * 1e6 / ops


# DRAM traffic of one k_coverage launch per bin entry, from an ncu capture of
# the first 1,000 paths of the workload (dram__bytes_read.sum + write.sum =
# 124.4 MB over 8,357,160 bin entries); scaled to the launch by its bin
# entries.
COVERAGE_TRAFFIC_PER_PAIR = (117.854208e6 + 6.578688e6) / 8357160


AUTOTUNE = True


TESS_KERNELS = ("k_link_path", "k_link_setup", "k_emit", "k_arclen_scan")


def tessellation_only(kmean: dict, n_seg: int, world: int) -> dict:
    """The tessellation stages of the timed step alone (what the plain variant
    times), from the per-kernel CUDA events."""
    ms = sum(kmean.get(k, 0.0) for k in TESS_KERNELS)
    return {"ms": ms, "segments_per_s": world * n_seg / (ms * 1e-3) if ms > 0 else None,
            "kernels": list(TESS_KERNELS)}


def tune_step(ps, ctx, step, n_tile, R, key, flush, raster=True):
    """Size the bins from the step's own count, then autotune the launch
    parameters (cached per device and workload signature; skipped, keeping the
    defaults, under --no-autotune)."""
    import torch
    from paper_2007_00308_gb300 import autotune as AT
    pairs_reserved = None
    step()
    torch.cuda.synchronize()
    st = ctx.status()
    if raster and st == ps.PS_ERR_CAPACITY:
        pairs = ps.ps_raster_stats(ctx)["pairs"]
        pairs_reserved = AT.reserve_bins(ctx, n_tile, pairs)
        step()
        torch.cuda.synchronize()
        st = ctx.status()
    if st != 0:
        raise RuntimeError(f"device status {st}: {ps.error_string(st)}")
    if not AUTOTUNE:
        return {"params": AT.current(ctx), "skipped": True, "bin_entries_reserved": pairs_reserved}
    res = AT.tuned(ctx, step, key, flush=flush.zero_ if flush is not None else None)
    torch.cuda.synchronize()
    st = ctx.status()
    if st != 0:
        raise RuntimeError(f"device status {st}: {ps.error_string(st)}")
    res = {k: v for k, v in res.items() if k != "trials"}
    res["bin_entries_reserved"] = pairs_reserved
    return res


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2007_00308_gb300 as ps
    from paper_2007_00308_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    # the job's share of rank r: its own batch of the workload (seeded per rank;
    # rank 0 strokes the standard batch), so per-GPU work is fixed as ranks are
    # added and no collective touches the data path
    batch = W.c2_batching(n_paths=args.n_paths, seed=W.SEED_BASE + 2 + 1000 * rank)
    Wd, Ht = batch.canvas
    ctx = ps.Context()
    if args.pixel_tol > 0:
        ctx.set_pixel_tolerance(args.pixel_tol)
    db = ps.DeviceBatch(batch, device=dev)
    prec = ps.PS_PREC_MIXED
    # exact rib count once at set-up; the step itself never synchronizes
    probe = ps.TessOutput(db.n_link, db.n_path, 0, arclength=False, device=dev)
    R = ps.ps_count_ribs_sync(ctx, db, probe, prec)
    out = ps.TessOutput(db.n_link, db.n_path, R, arclength=True, device=dev)
    canvas = torch.zeros((Ht, Wd), dtype=torch.int16, device=dev)
    covered = torch.zeros(db.n_path, dtype=torch.int64, device=dev)
    n_tile = ((Wd + 15) // 16) * ((Ht + 15) // 16)
    # bins start at one entry per rib; the first step's count sizes them
    ctx.reserve(n_link=db.n_link, n_rib=R, n_tile=n_tile, n_pair=R)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(stream=None):
        ps.ps_tessellate_strokes(ctx, db, out, prec, ps.PS_TESS_ARCLENGTH, stream=stream)
        ps.ps_rasterize_coverage(ctx, out.rib, out.tag, out.n_rib, out.capacity, db.n_path, Wd, Ht,
                                 canvas, covered, stream=stream, exact=args.exact)

    # eager steps: bin sizing and autotuning (allocates workspace), then one
    # step captured in a graph
    from paper_2007_00308_gb300 import autotune as AT
    tuning = tune_step(ps, ctx, step, n_tile, R,
                       AT.signature(torch.cuda.get_device_name(dev), batch.n_seg, db.n_path, R,
                                    (Wd, Ht)), flush)
    ctx.profile(True)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step(stream=s)  # warm the side stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        step()
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        g.replay()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kern = {}
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()  # L2 (129 MB) flushed before every step
        ev[i][0].record()
        g.replay()
        ev[i][1].record()
        for k, v in ctx.profile_read().items():  # waits for this step's events
            kern.setdefault(k, []).append(v)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dev)
    if world > 1:
        dist.barrier()
    st = ctx.status()
    if st != 0:
        raise RuntimeError(f"device status {st}: {ps.error_string(st)}")
    ms_per_step = total_ms / args.steps
    segs = batch.n_seg
    value = job_throughput(segs, world, ms_per_step)
    cov_samples = int(covered.sum().item())
    R_now = int(out.n_rib.item())

    # kernel table and the dominant kernel's roofline
    import math
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    kmean = {k: statistics.mean(v) for k, v in kern.items()}
    dom = max(kmean, key=kmean.get)
    rstat = ps.ps_raster_stats(ctx)
    pairs, span_px = rstat["pairs"], rstat["span_pixels"]
    counts = {"R": R_now, "L": db.n_link, "S": segs, "P": db.n_path, "px": Wd * Ht,
              "pairs": pairs, "span_px": span_px,
              "tiles": ((Wd + 15) // 16) * ((Ht + 15) // 16)}
    sm_mhz = clk.get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    kernels = {}
    for k, ms in kmean.items():
        alg = algorithmic(k, counts)
        if not alg:
            kernels[k] = {"ms": ms}
            continue
        bound, work = alg
        if bound == "hbm":
            ach = work / (ms * 1e-3) / 1e9
            kernels[k] = {"ms": ms, "bound": "hbm", "algorithmic_bytes": work,
                          "achieved_gbs": ach, "frac": ach / hbm_peak,
                          "workspace_bytes": workspace_bytes(k, counts)}
        else:
            ach = work / (ms * 1e-3) / 1e9
            opt = ops_per_test(rstat, args.exact)
            pk_derived = alu_peak_tests(sm_mhz, opt) / 1e9
            pk_meas = measured_peak_tests(rstat, sm_mhz, args.exact)
            pk = pk_meas / 1e9 if pk_meas else pk_derived
            kernels[k] = {"ms": ms, "bound": "alu", "sample_tests": work,
                          "achieved_gtests": ach, "peak_gtests": pk, "frac": ach / pk,
                          "peak_derived_gtests": pk_derived, "peak_measured": bool(pk_meas)}
    kd = kernels[dom]
    if kd.get("bound") == "alu":
        opt = ops_per_test(rstat, args.exact)
        roof = {"kernel": dom, "bound": "alu", "achieved": kd["achieved_gtests"],
                "peak": kd["peak_gtests"], "unit": "Gsample-tests/s", "frac": kd["frac"],
                # measured on the two-triangle kernel; none for the crossing-rule mode
                "traffic": (int(COVERAGE_TRAFFIC_PER_PAIR * pairs)
                            if dom == "k_coverage" and not args.exact else None),
                "peak_source": (("measured: issue rate of the mask's op mix per pixel class "
                                 f"(microbenchmark), pixel-class mix, {sm_mhz:.0f} MHz; derived "
                                 f"(128 lane ops/clock / {opt:.2f} ops per test) "
                                 f"{kd['peak_derived_gtests']:.0f} G tests/s")
                                if kd.get("peak_measured") else
                                (f"derived: 152 SMs x 128 lane ops/clock x {sm_mhz:.0f} MHz / "
                                 f"{opt:.2f} lane ops per sample test (pixel-class mix)")),
                "algorithmic_work": kd["sample_tests"],
                "traffic_source": "ncu capture of 1,000 paths scaled by bin entries"}
    elif kd.get("bound") == "hbm":
        roof = {"kernel": dom, "bound": "hbm", "achieved": kd["achieved_gbs"], "peak": hbm_peak,
                "unit": "GB/s", "frac": kd["frac"], "traffic": None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback",
                "algorithmic_bytes": kd["algorithmic_bytes"]}
    else:
        roof = None

    # end to end through the C ABI with host buffers
    e2e = run_e2e(args, ps, batch, ctx, db, out, canvas, covered, prec, dev)

    plain = None if args.no_plain else run_plain(ps, batch, dev)

    line = {
        "metric": METRIC, "value": value, "unit": "segments/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "variant": "batched+mixed: one CUDA graph per step, "
                   "FP32 pipe with double-float angles, normals, t and vertices; FP64 only "
                   "in the curvature discriminant and near-double-root islands" +
                   (", quads rasterized as polygons" if args.exact else "") +
                   (f", per-link step boosted to pixel scale (tolerance {args.pixel_tol:g} px)"
                    if args.pixel_tol > 0 else ""), "n_segments": segs,
                   "n_paths": db.n_path, "n_ribs": R_now, "canvas": [Wd, Ht], "spp": 16,
                   "l2": "flushed before every timed step (256 MiB write)",
                   "wall_s_timed_region": t_wall, "autotune": tuning},
        "covered_samples_per_s": world * cov_samples / (ms_per_step * 1e-3),
        "covered_samples": cov_samples,
        "kernel_ms": kmean,
        "tessellation_only": tessellation_only(kmean, segs, world),
        "kernels": kernels,
        "stages": stage_report(kmean, counts, hbm_peak),
        "raster_work": rstat,
        "roofline": roof,
        "e2e": e2e,
        # our kernels per step, from the profile slots that recorded a launch
        "gpu_launches": len(kmean) * args.steps,
        "clocks": clk,
        "plain": plain,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(batch)
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_e2e(args, ps, batch, ctx, db, out, canvas, covered, prec, dev):
    import numpy as np
    import torch
    Wd, Ht = batch.canvas
    host = {k: getattr(db, k).cpu().pin_memory() for k in
            ("seg_type", "seg_pts", "seg_w", "path_seg_off", "path_width", "path_join", "path_cap",
             "path_miter", "path_closed")}
    h_canvas = torch.empty(canvas.shape, dtype=canvas.dtype).pin_memory()
    h_cov = torch.empty(covered.shape, dtype=covered.dtype).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = h_canvas.numel() * 2 + h_cov.numel() * 8
    n = max(5, min(args.steps, 30))
    times = []
    for i in range(n + 2):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for k, t in host.items():
            getattr(db, k).copy_(t, non_blocking=True)
        ps.ps_tessellate_strokes(ctx, db, out, prec, ps.PS_TESS_ARCLENGTH)
        ps.ps_rasterize_coverage(ctx, out.rib, out.tag, out.n_rib, out.capacity, db.n_path, Wd, Ht,
                                 canvas, covered, exact=args.exact)
        h_canvas.copy_(canvas, non_blocking=True)
        h_cov.copy_(covered, non_blocking=True)
        b.record()
        b.synchronize()
        if i >= 2:
            times.append(a.elapsed_time(b))
    ms = statistics.mean(times)
    return {"value": batch.n_seg / (ms * 1e-3), "unit": "segments/s", "ms_per_step": ms,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}


def run_plain(ps, batch, dev, max_paths=2000):
    """One path per launch, all FP32, host-driven (count synchronously, then emit)."""
    import torch
    n = min(max_paths, batch.n_path)
    sub = batch.subset(range(n))
    ctx = ps.Context()
    dbs = []
    for p in range(n):
        dbs.append(ps.DeviceBatch(sub.subset([p]), device=dev))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    segs = 0
    for d in dbs:
        probe = ps.TessOutput(d.n_link, d.n_path, 0, arclength=False, device=dev)
        R = ps.ps_count_ribs_sync(ctx, d, probe, ps.PS_PREC_FP32)
        o = ps.TessOutput(d.n_link, d.n_path, max(R, 1), arclength=True, device=dev)
        ps.ps_tessellate_strokes(ctx, d, o, ps.PS_PREC_FP32, ps.PS_TESS_ARCLENGTH)
        segs += d.n_seg
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"segments_per_s": segs / dt, "sample": f"first {n} paths, tessellation only, "
            "one path per launch, FP32, host-synchronous count", "s": dt}


CONFIG_DESC = {
    "c1": "c1 plain small: one path of 64 chained cubics in [0,512]^2, width 8 px, round joins "
          "and caps, dtheta 2 deg, 512x512 at 16 samples/pixel; step = tessellation + coverage",
    "c3": "c3 large single path: 5,031 chained cubics on a random walk, width 2 px, round joins "
          "and caps, dtheta 0.5 deg, dash [12 on, 6 off], 4096x4096 at 16 samples/pixel; step = "
          "tessellation + arc length + dash + coverage of the dashed quads",
    "c4": "c4 precision stress: 1,000,000 single-cubic paths near cusps and near collinearity, "
          "coordinates up to 1e6 px, width 1 px, butt caps, dtheta 1 deg; step = tessellation "
          "(no raster)",
    "c5": "c5 differentiation: 4,096 paths x 32 chained cubics in [0,1024]^2, widths 1-16 px, "
          "round joins and caps, dtheta 2 deg; step = forward tessellation + adjoint",
    "facet": "uniform-parametric comparison: 20,000 single cubics (half serpentines, a quarter "
             "exact cusps, a quarter loops), chords 20-400 px, widths 1-100 px, dtheta 4 deg; "
             "step = polar tessellation + uniform tessellation at the same counts + facet "
             "statistics of both",
}


def run_config(args, rank, world, local_rank):
    """One line for a configuration other than the headline one (same timing rules:
    graph-captured step, L2 flushed before every step, CUDA events on the stream)."""
    import torch
    import paper_2007_00308_gb300 as ps
    from paper_2007_00308_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = args.workload
    batch = {"c1": W.c1_plain_small, "c3": W.c3_large_path, "c4": W.c4_precision,
             "c5": W.c5_differentiation, "facet": W.facet_comparison}[wl]()
    ctx = ps.Context()
    db = ps.DeviceBatch(batch, device=dev)
    prec = ps.PS_PREC_MIXED
    probe = ps.TessOutput(db.n_link, db.n_path, 0, arclength=False, device=dev)
    R = ps.ps_count_ribs_sync(ctx, db, probe, prec)
    out = ps.TessOutput(db.n_link, db.n_path, R, arclength=True, want_t=(wl == "c5"), device=dev)
    raster = wl in ("c1", "c3")
    Wd, Ht = batch.canvas if raster else (0, 0)
    extra = {}
    if raster:
        canvas = torch.zeros((Ht, Wd), dtype=torch.int16, device=dev)
        covered = torch.zeros(db.n_path, dtype=torch.int64, device=dev)
    if wl == "c3":
        pattern, offset = batch.dash
        cap = 3 * R + 4096
        d_rib = torch.empty((cap, 4), dtype=torch.float32, device=dev)
        d_s = torch.empty(cap, dtype=torch.float32, device=dev)
        d_tag = torch.empty(cap, dtype=torch.int32, device=dev)
        d_src = torch.empty(cap, dtype=torch.int32, device=dev)
        d_n = torch.zeros(1, dtype=torch.int64, device=dev)
    if wl == "facet":
        uni = torch.empty_like(out.rib)
        st_p = torch.empty((db.n_link, 4), dtype=torch.float32, device=dev)
        st_u = torch.empty_like(st_p)
    if wl == "c5":
        gen = torch.Generator(device="cpu").manual_seed(20200705)
        g_rib = torch.randn((R, 4), generator=gen).to(dev)
        g_s = torch.randn(R, generator=gen).to(dev)
        g_pts = torch.zeros((db.n_seg, 4, 2), dtype=torch.float32, device=dev)
        g_w = torch.zeros(db.n_path, dtype=torch.float32, device=dev)
    n_tile = ((Wd + 15) // 16) * ((Ht + 15) // 16)
    if raster:
        ctx.reserve(n_link=db.n_link, n_rib=R, n_tile=n_tile, n_pair=R)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(stream=None):
        ps.ps_tessellate_strokes(ctx, db, out, prec, ps.PS_TESS_ARCLENGTH, stream=stream)
        if wl == "c1":
            ps.ps_rasterize_coverage(ctx, out.rib, out.tag, out.n_rib, out.capacity, db.n_path,
                                     Wd, Ht, canvas, covered, stream=stream)
        elif wl == "c3":
            ps.ps_dash(ctx, out.rib, out.s, out.tag, out.n_rib, out.capacity, pattern, offset,
                       d_rib, d_s, d_tag, d_src, d_n, cap, stream=stream)
            ps.ps_rasterize_coverage(ctx, d_rib, d_tag, d_n, cap, db.n_path, Wd, Ht, canvas,
                                     covered, stream=stream)
        elif wl == "facet":
            ps.ps_uniform_tessellate(ctx, db, out, uni, stream=stream)
            ps.ps_facet_stats(ctx, out.rib, out.tag, out.link_rib_off, out.n_rib, out.capacity,
                              st_p, stream=stream)
            ps.ps_facet_stats(ctx, uni, out.tag, out.link_rib_off, out.n_rib, out.capacity,
                              st_u, stream=stream)
        elif wl == "c5":
            g_pts.zero_()
            g_w.zero_()
            ps.ps_tessellate_backward(ctx, db, out, g_rib, g_s, g_pts, g_w, prec, stream=stream)

    from paper_2007_00308_gb300 import autotune as AT
    tuning = tune_step(ps, ctx, step, n_tile, R,
                       AT.signature(torch.cuda.get_device_name(dev), batch.n_seg, db.n_path, R,
                                    (Wd, Ht)) + f"|{wl}", flush, raster=raster)
    ctx.profile(True)
    g = torch.cuda.CUDAGraph()
    sside = torch.cuda.Stream(device=dev)
    sside.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(sside):
        step(stream=sside)
    torch.cuda.current_stream().wait_stream(sside)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        step()
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        g.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kern = {}
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record()
        g.replay()
        ev[i][1].record()
        for k, v in ctx.profile_read().items():
            kern.setdefault(k, []).append(v)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_per_step = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dev) / args.steps
    st = ctx.status()
    if st != 0:
        raise RuntimeError(f"device status {st}: {ps.error_string(st)}")
    line = {
        "metric": METRIC, "value": job_throughput(batch.n_seg, world, ms_per_step),
        "unit": "segments/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": CONFIG_DESC[wl], "variant": "batched+mixed, one CUDA graph per step",
                   "n_segments": int(batch.n_seg), "n_paths": int(batch.n_path),
                   "n_ribs": int(out.n_rib.item()),
                   "l2": "flushed before every timed step (256 MiB write)", "autotune": tuning},
        "kernel_ms": {k: statistics.mean(v) for k, v in kern.items()},
        "tessellation_only": tessellation_only({k: statistics.mean(v) for k, v in kern.items()},
                                               int(batch.n_seg), world),
        "clocks": clk,
    }
    if raster:
        cs = int(covered.sum().item())
        line["covered_samples"] = cs
        line["covered_samples_per_s"] = world * cs / (ms_per_step * 1e-3)
        line["raster_work"] = ps.ps_raster_stats(ctx)
    if wl == "c3":
        line["config"]["n_dashed_ribs"] = int(d_n.item())
    if wl == "facet":
        import math
        sp = st_p.cpu().double().numpy()
        su = st_u.cpu().double().numpy()

        def summary(a):
            n = a[:, 3].sum()
            m = a[:, 1].sum() / n
            return {"max_deg": math.degrees(a[:, 0].max()), "mean_deg": math.degrees(m),
                    "sd_deg": math.degrees(math.sqrt(max(a[:, 2].sum() / n - m * m, 0.0))),
                    "ordinary_facets": int(n)}
        segs = (sp[:, 3] > 0) & (su[:, 3] > 0)
        line["facets"] = {"polar": summary(sp), "uniform": summary(su),
                          "segments_polar_max_smaller": float((sp[segs, 0] < su[segs, 0]).mean()),
                          "bound_2q_deg": math.degrees(2 * batch.dtheta)}
    if not args.no_plain and wl not in ("c5", "facet"):
        line["plain"] = run_plain(ps, batch, dev, max_paths=2000 if wl == "c4" else batch.n_path)
    if rank == 0:
        print(json.dumps(line))
    return 0


def main():
    global AUTOTUNE
    args = parse()
    AUTOTUNE = not args.no_autotune
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import datetime
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        # a rank that dies ends the others' next collective with an error within
        # this time instead of holding the job (the timed work is about a minute)
        dist.init_process_group("nccl", timeout=datetime.timedelta(seconds=PG_TIMEOUT_S))
    try:
        if args.workload != "c2":
            return run_config(args, rank, world, local_rank)
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
