"""Benchmark: time-to-tolerance and stencil GLUP/s of the multisplitting solver.

One step = one complete solve of the 256^3 Laplace workload (4x4x4 blocks of
64^3, Dirichlet data iid U(-1,1) seed 2009, x0 = 0) to relative residual
1e-8, FP32 inner CG / FP64 outer, synchronous block Jacobi -- every row of
the hot path (residual with halo, inner CG, update, global norm and stop).
Inputs are resident on the GPU before the timed region; the e2e figure goes
through the host-buffer entry point (ms_solve_host) with the copies inside
the timed region.

value = stencil lattice updates (inner CG iterations x block points plus one
residual pass per sweep) per second over the K timed solves, summed over
ranks (N > 1: independent replicas, weak scaling).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-rel-residual-1e-8 and stencil GLUP/s vs plain FP64 sync; HBM GB/s vs peak"
UNIT = "GLUP/s"
WORKLOAD = "laplace256_u11"
# algorithmic bytes per lattice update (the roofline's numerator): the inner CG must
# read and write r, p and d once per iteration (24 B at FP32, 48 B at FP64);
# an outer sweep reads x (8 B) and writes r (4 B), then reads x and d and
# writes x (20 B): 32 B per point at FP32 (the FP64 r/d add 8 B).
INNER_BYTES = {"mixed": 24.0, "fp64": 48.0}
OUTER_BYTES = {"mixed": 32.0, "fp64": 40.0}
# DRAM traffic per launch of the dominant kernel, from one ncu capture, with
# the hash of the kernel sources it was taken on (null once they change)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "res_sweep_laplace256_traffic.json")
KERNEL_SOURCES = ["ms_resident_kernels.cuh", "ms_resident_variants.h", "ms_resident.cuh", "ms_async.cuh", "ms_device.cuh",
                  "ms_cg.cuh", "ms_internal.h"]


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2009_12638_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_record(kernel_name):
    """The ncu record of the dominant kernel (DRAM bytes per launch and on-chip
    utilisation), or None when it was taken on other kernel sources."""
    try:
        rec = json.load(open(TRAFFIC_FILE))
    except Exception:
        return None
    if rec.get("source_hash") != kernel_source_hash() or rec.get("kernel") != kernel_name:
        return None
    return rec


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ms", choices=["ms", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--mode", default="sync", choices=["sync", "async"])
    ap.add_argument("--engine", default="auto", choices=["auto", "streaming", "resident"],
                    help="inner-CG engine (default: the autotuner's choice)")
    ap.add_argument("--overlap", type=int, default=0, help="overlapping blocks: points per face (sync mode)")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64-sync and async comparison solves")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched workloads (uneven blocks x 16 rhs, 512^3 x 4 rhs)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--clock-log", default=None, help="directory for the raw nvidia-smi clock samples (CSV)")
    ap.add_argument("--scale", type=int, default=1,
                    help="profiling aid with --sweeps: shrink every block edge by this factor (block counts kept)")
    ap.add_argument("--sweeps", type=int, default=0,
                    help="profiling aid: run exactly this many outer sweeps once (no warm-up, no timing) and exit")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, log_dir=None):
        """Samples nvidia-smi every 200 ms into a CSV (in log_dir if given, else a temporary file)."""
        self.index = index
        self.proc = None
        if log_dir:
            self.path = os.path.join(log_dir, f"clocks_rank{index}.csv")
        else:
            import tempfile
            self.path = os.path.join(tempfile.gettempdir(), f"ms_bench_clocks_{os.getpid()}_{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
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
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [v.strip() for v in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = max(mx, float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        loaded = [v for v in sm if v >= 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle timing (CPU)
def oracle_sample(cfg, sweeps, threads):
    """Times `sweeps` outer sweeps of the FP64 CPU oracle on the full workload."""
    import oracle
    oracle.build()
    oracle.set_threads(threads)
    opts = dict(cfg["opts"])
    t0 = time.perf_counter()
    lups = 0
    for s in range(cfg["nrhs"]):
        r = oracle.solve(cfg["nx"], cfg["ny"], cfg["nz"], cfg["cx"], cfg["cy"], cfg["cz"], bnd=cfg["bnd"][s],
                         inner_rtol=opts["inner_rtol"], inner_maxit=opts["inner_maxit"], outer_tol=0.0,
                         outer_maxit=sweeps)
        npts = cfg["nx"] * cfg["ny"] * cfg["nz"]
        nblocks = (len(cfg["cx"]) - 1) * (len(cfg["cy"]) - 1) * (len(cfg["cz"]) - 1)
        lups += (sweeps + 1) * npts + r["inner_its"] * (npts // nblocks)
    el = time.perf_counter() - t0
    return lups, el


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2009_12638_gb300 import inputs
    import oracle
    cfg = inputs.make_config(args.workload)
    threads = oracle.max_threads()
    sweeps = 1
    for _ in range(args.warmup):
        oracle_sample(cfg, sweeps, threads)  # untimed
    total_lups, total_s = 0, 0.0
    for _ in range(args.steps):
        lups, el = oracle_sample(cfg, sweeps, threads)
        total_lups += lups
        total_s += el
    value = total_lups / total_s / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": f"{args.workload}: 256^3, 4x4x4 blocks of 64^3, U(-1,1) "
                                                        "boundary seed 2009, inner CG 50 its / rtol 1e-6"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": f"{sweeps} outer sweep(s) of the full workload per step (FP64 CPU oracle, "
                                      f"OpenMP over blocks)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# overlap of the batched measurement's blocks (points per face): the fastest of 5, 6, 8
# and 10 to 1e-8 on the uneven 16-rhs workload, with 10 within 2% of it
BATCH_OVERLAP = 8


def run_batched(dev):
    """The batched workloads, one measurement each (not part of the headline):

    * uneven: 384x320x256 cut into 5x6x4 blocks with edges of 40-96 points,
      16 rhs (N(0,1) boundary data) -- the mixed synchronous solve with
      overlapping blocks (8 points per face) from x0 = 0 to 1e-8, timed once;
      the FP64 synchronous path timed per sweep (3 sweeps, CUDA events) with
      and without overlap; its time to tolerance is extrapolated as per-sweep
      time x the mixed solve's sweep count (FP64 and mixed sweeps to 1e-8 agree
      within one on every workload solved both ways);
    * laplace512: 512^3, 8x8x8 blocks of 64^3, 4 rhs -- per-sweep rates of the
      mixed sync and async and FP64 sync paths, and one global FP64 CG to 1e-8.
    """
    import torch
    from paper_2009_12638_gb300 import Grid, inputs
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1)

    def per_sweep(g, b, x, n, **kw):
        # the sweep kernels of a capped solve end with one residual-only launch:
        # the difference of a 1-sweep and a (1 + n)-sweep solve is n full sweeps
        runs = []
        for k in (1, 1 + n):
            x.zero_()
            _, st = g.solve(bnd=b, out=x, outer_tol=0.0, outer_maxit=k, profile=True, use_graph=False, **kw)
            runs.append(st)
        ms = (runs[1].sweep_ms - runs[0].sweep_ms) / n
        lup = (runs[1].lups - runs[0].lups) / n
        return {"per_sweep_ms": ms, "sweeps_timed": n, "glups": lup / (ms * 1e-3) / 1e9 if ms > 0 else None}

    res = {}
    cfg = inputs.make_config("batched_uneven")
    g = Grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["nrhs"], device=dev)
    g.partition(len(cfg["cx"]) - 1, len(cfg["cy"]) - 1, len(cfg["cz"]) - 1, cfg["cx"], cfg["cy"], cfg["cz"])
    b = torch.from_numpy(cfg["bnd"]).to(dev)
    x = torch.zeros(g.shape, dtype=torch.float64, device=dev)
    (_, st), ms = timed(lambda: g.solve(bnd=b, out=x, precision="mixed", overlap=BATCH_OVERLAP, time_limit_ms=180000))
    true_rel = g.residual(x, bnd=b)
    mixed = {"status": st.status_name, "time_to_tol_s": ms / 1e3, "sweeps": st.outer_its,
             "per_rhs_sweeps": list(st.per_rhs_outer_its), "glups": st.lups / (ms * 1e-3) / 1e9,
             "max_true_rel_residual": float(true_rel.max()), "overlap": BATCH_OVERLAP, "engine": st.engine,
             "variant": st.variant}
    f64o = per_sweep(g, b, x, 2, precision="fp64", overlap=BATCH_OVERLAP)
    f64o["sweeps"] = st.outer_its
    f64o["time_to_tol_s"] = f64o["per_sweep_ms"] * st.outer_its / 1e3
    f64o["extrapolated"] = "per-sweep time (CUDA events) x the mixed solve's sweep count"
    res["uneven_16rhs"] = {
        "workload": "384x320x256 Laplace 7-point, 5x6x4 uneven blocks (edges 40-96, seed 12638), 16 rhs, boundary "
                    "iid N(0,1) seed 12639, x0=0, inner CG <=50 its rtol 1e-6, outer rel tol 1e-8",
        "mixed_sync_overlap": mixed,
        "fp64_sync_overlap": f64o,
        "fp64_sync_per_sweep": per_sweep(g, b, x, 2, precision="fp64"),
        "mixed_sync_per_sweep": per_sweep(g, b, x, 3, precision="mixed"),
        "speedup_vs_fp64_sync_overlap": f64o["time_to_tol_s"] / mixed["time_to_tol_s"] if ms > 0 else None,
    }
    del g, b, x
    torch.cuda.empty_cache()
    cfg = inputs.make_config("laplace512_async")
    g = Grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["nrhs"], device=dev)
    g.partition(8, 8, 8, cfg["cx"], cfg["cy"], cfg["cz"])
    b = torch.from_numpy(cfg["bnd"]).to(dev)
    x = torch.zeros(g.shape, dtype=torch.float64, device=dev)
    x.zero_()
    (_, sa), ms_a = timed(lambda: g.solve(bnd=b, out=x, precision="mixed", mode="async", outer_tol=0.0, outer_maxit=6))
    x.zero_()
    (_, sc), ms_c = timed(lambda: g.gcg_solve(bnd=b, out=x, outer_tol=1e-8, time_limit_ms=120000))
    res["laplace512_4rhs"] = {
        "workload": "512^3 Laplace 7-point, 8x8x8 blocks of 64^3, 4 rhs, boundary iid U(-1,1) seed 512, x0=0",
        "mixed_sync_per_sweep": per_sweep(g, b, x, 3, precision="mixed"),
        "mixed_async": {"sweeps_per_block": sa.outer_its, "ms_per_sweep": ms_a / max(1, sa.outer_its),
                        "glups": sa.lups / (ms_a * 1e-3) / 1e9},
        "fp64_sync_per_sweep": per_sweep(g, b, x, 1, precision="fp64"),
        "global_fp64_cg": {"status": sc.status_name, "time_to_tol_s": ms_c / 1e3, "iterations": sc.outer_its,
                           "rel_residual": sc.rel_residual},
    }
    del g, b, x
    torch.cuda.empty_cache()
    return res


def reduce_over_ranks(total_ms, lups, device):
    """Job-level timing over ranks: the slowest rank's time (max) and the sum of
    every rank's lattice updates (N > 1 runs independent replicas)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1):
        return float(total_ms), float(lups)
    tm = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    tl = torch.tensor([float(lups)], dtype=torch.float64, device=device)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    dist.all_reduce(tl, op=dist.ReduceOp.SUM)
    return float(tm.item()), float(tl.item())


# ------------------------------------------------------------------ GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    from paper_2009_12638_gb300 import Grid, inputs
    if args.scale != 1 and not args.sweeps:
        raise SystemExit("--scale is a profiling aid for --sweeps runs; the measured workload is the stated one")
    cfg = inputs.make_config(args.workload, scale=args.scale)
    # each rank solves its own replica (different boundary seed for rank > 0)
    bnd_np = cfg["bnd"] if rank == 0 else inputs.boundary_uniform(cfg["nx"], cfg["ny"], cfg["nz"], cfg["nrhs"],
                                                                   2009 + rank)
    grid = Grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["nrhs"], device=dev)
    grid.partition(len(cfg["cx"]) - 1, len(cfg["cy"]) - 1, len(cfg["cz"]) - 1, cfg["cx"], cfg["cy"], cfg["cz"])
    bnd = torch.from_numpy(bnd_np).to(dev)
    x = torch.zeros(grid.shape, dtype=torch.float64, device=dev)
    opts = dict(cfg["opts"], precision=args.precision, mode=args.mode, engine=args.engine, overlap=args.overlap)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)

    def solve_once(**extra):
        x.zero_()
        return grid.solve(bnd=bnd, out=x, **dict(opts, **extra))

    if args.sweeps:
        # a short, fixed run for ncu captures: the shape the autotuner would pick, one plain
        # launch of the sweep kernel per sweep (the launch mode of the timed solves)
        _, st = solve_once(outer_tol=0.0, outer_maxit=args.sweeps, use_graph=False, persistent=False)
        torch.cuda.synchronize(dev)
        print(json.dumps({"sweeps": args.sweeps, "status": st.status_name, "engine": st.engine,
                          "variant": st.variant, "shape": [st.cluster, st.threads, st.slots],
                          "time_ms": st.time_ms}))
        return

    for _ in range(max(args.warmup, 3)):
        _, st = solve_once()
        assert st.status == 0, st
    sampler = ClockSampler(local, args.clock_log)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    times, lups, launches, stats = [], 0, 0, []
    for _ in range(args.steps):
        flush.fill_(1.0)  # evict L2 between timed solves (not timed)
        x.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = grid.solve(bnd=bnd, out=x, **opts)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        lups += st.lups
        launches += st.launches
        stats.append(st)
        assert st.status == 0 and st.rel_residual < opts["outer_tol"], st
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms, lups_all = reduce_over_ranks(sum(times), lups, dev)
    value = lups_all / (total_ms * 1e-3) / 1e9
    st0 = stats[0]

    # ---- end to end through the host-buffer entry point (pinned host memory)
    xh = torch.zeros(grid.shape, dtype=torch.float64).pin_memory().numpy()
    bh = torch.from_numpy(bnd_np.copy()).pin_memory().numpy()
    grid.solve_host(bnd=bh, x=xh, **opts)  # warm the host-side workspace
    e2e_ms, e2e_lups = 0.0, 0
    e2e_steps = min(args.steps, 5)  # each is a full solve; five give a stable mean
    for _ in range(e2e_steps):
        xh[...] = 0.0
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, sh = grid.solve_host(bnd=bh, x=xh, **opts)
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_lups += sh.lups
        assert sh.status == 0
    e2e_value = e2e_lups / (e2e_ms * 1e-3) / 1e9 * world

    # ---- roofline of the dominant kernel (the sweep kernel), per-launch CUDA events
    _, sp = solve_once(profile=True)
    sweeps = sp.outer_its + 1
    inner_lups = sp.lups - sweeps * grid.npts * grid.nrhs
    alg_bytes = INNER_BYTES[args.precision] * inner_lups + OUTER_BYTES[args.precision] * sweeps * grid.npts
    per_launch_ms = sp.sweep_ms / max(1, sp.sweep_launches)
    achieved = alg_bytes / sweeps / (per_launch_ms * 1e-3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    kname = {True: "res_sweep_kernel", False: "strip_sweep_kernel" if sp.variant == -2 else "sweep_kernel"}[sp.variant >= 0]
    rec = measured_record(kname)
    traffic = float(rec["dram_bytes_per_launch"]) if rec else None
    dram_gbs = traffic / (per_launch_ms * 1e-3) / 1e9 if traffic is not None else None
    roofline = {"bound": "on-chip" if sp.variant >= 0 else "l2",
                "achieved": dram_gbs, "peak": peak, "unit": "GB/s",
                "frac": dram_gbs / peak if dram_gbs is not None else None,
                "traffic": traffic, "kernel": kname, "per_launch_ms": per_launch_ms,
                "launches_timed": sp.sweep_launches,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                "equivalent": {"achieved": achieved, "frac": achieved / peak, "unit": "GB/s",
                               "alg_bytes_per_launch": alg_bytes / sweeps,
                               "meaning": "algorithmic bytes of an HBM-streaming CG (24 B per inner LUP, 32 B per "
                                          "point and sweep) / launch time: the HBM bandwidth a streaming kernel "
                                          "would need to match this one"},
                "on_chip": ({k: rec[k] for k in ("smem_wavefront_frac", "issue_active_frac", "sms_used",
                                                 "duration_ms_ncu") if k in rec} if rec else None),
                "note": "achieved/frac = DRAM bytes measured by ncu per launch (same kernel sources) / live "
                        "launch time; the resident kernel keeps the CG state in registers and shared memory, so "
                        "HBM is nearly idle and the bound is on chip (barriers, shared-memory and FP64 latency); "
                        "on_chip gives its shared-memory and issue utilisation from the same capture"}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
           "data": "synthetic",
           "config": {"workload": f"{args.workload}: 256^3 Laplace 7-point, 4x4x4 blocks of 64^3, boundary iid "
                                  "U(-1,1) seed 2009, x0=0, inner CG <=50 its rtol 1e-6, outer rel tol 1e-8",
                      "precision": args.precision, "mode": args.mode, "engine": args.engine,
                      "overlap": args.overlap,
                      "launch_shape": {"cluster": st0.cluster, "threads": st0.threads, "slots": st0.slots},
                      "kernel_source_hash": kernel_source_hash(),
                      "l2": "flushed (256 MB write) between timed solves"},
           "time_to_tol_s": total_ms / args.steps / 1e3, "outer_its": st0.outer_its, "inner_its": st0.inner_its,
           "rel_residual": max(s.rel_residual for s in stats), "gpu_launches": launches,
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(bh.nbytes + xh.nbytes),
                   "d2h_bytes_per_step": int(xh.nbytes), "ms_per_step": e2e_ms / e2e_steps, "steps": e2e_steps},
           "roofline": roofline, "clocks": clocks}

    if rank == 0 and not args.no_compare:
        comp = {}
        for name, extra in [("fp64_sync", dict(precision="fp64", mode="sync")),
                            ("mixed_async", dict(precision="mixed", mode="async")),
                            ("mixed_sync_adaptive_inner", dict(precision="mixed", mode="sync", inner_adapt=True)),
                            ("mixed_sync_overlap5", dict(precision="mixed", mode="sync", overlap=5))]:
            if extra["precision"] == args.precision and extra["mode"] == args.mode and len(extra) == 2:
                continue
            x.zero_()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, sc = grid.solve(bnd=bnd, out=x, **dict(opts, **extra, time_limit_ms=120000))
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            comp[name] = {"status": sc.status_name, "time_to_tol_s": ms / 1e3, "outer_its": sc.outer_its,
                          "rel_residual": sc.rel_residual, "glups": sc.lups / (ms * 1e-3) / 1e9}
            if "inner_adapt" in extra:
                comp[name]["inner_rtol_final"] = sc.inner_rtol_final
        # one global FP64 CG on the whole grid (no blocks), same stop rule and tolerance
        x.zero_()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, sc = grid.gcg_solve(bnd=bnd, out=x, outer_tol=opts["outer_tol"], time_limit_ms=120000)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        comp["global_fp64_cg"] = {"status": sc.status_name, "time_to_tol_s": ms / 1e3, "iterations": sc.outer_its,
                                  "rel_residual": sc.rel_residual, "glups": sc.lups / (ms * 1e-3) / 1e9}
        out["compare"] = comp
        if "fp64_sync" in comp and comp["fp64_sync"]["status"] == "OK":
            out["speedup_vs_fp64_sync"] = comp["fp64_sync"]["time_to_tol_s"] / out["time_to_tol_s"]
    if rank == 0 and not args.no_batched:
        out["batched"] = run_batched(dev)
    if rank == 0 and world == 1 and not args.no_cpu:
        threads = int(os.environ.get("MS_ORACLE_THREADS", "0")) or None
        import oracle
        threads = threads or oracle.max_threads()
        olups, osec = oracle_sample(cfg, 1, threads)
        out["cpu_baseline"] = {"value": olups / osec / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": "1 outer sweep (residual of x^0 and x^1, 64 inner CG solves) of the full "
                                         "workload, FP64 CPU oracle with OpenMP over blocks",
                               "seconds": osec}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
