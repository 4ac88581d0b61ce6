#!/usr/bin/env python3
"""Benchmark of the batched FP32 Peaceman-Rachford ADI step (libadi) on GB300.

Workload (one "step" = one full PR step -- stage 1 over every x-line, stage 2 over every
y-line -- of every member of the batch):
    batched FP32 at 4096 x 4096 cells: one CFD and one MFD simulation of the layered
    seismic medium (c 1500-4500 m/s in four layers times a seeded 10 % Gaussian, a 15 Hz
    Ricker point source at the centre, h = 5 m, dt = cfl_max h / c_max).
Metric: grid-point updates per second (cells x steps / s), whole job over all ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica of the batch ("replicas
only": the scheme has no data-path collective); value = all ranks' updates / max time.
--impl reference times the FP64 CPU oracle on the same workload (bounded per-step sample)
on rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

N_SIDE = 4096
METRIC = "ADI grid-point updates/s (batched FP32 vs plain FP64, 4096^2); p50/p99 latency"
UNIT = "updates/s"
REF_BUDGET_S = 90.0  # host seconds of the reference arm (warm-up + timed steps)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=N_SIDE)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-peak", action="store_true", help="skip the 8192^2 roofline leg")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper's fixed-point iteration leg")
    ap.add_argument("--ref-budget", type=float, default=REF_BUDGET_S,
                    help="seconds of oracle work the reference arm aims at")
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="requests of the config-4 serving stream (sides 64-4096, 100-5000 steps)")
    ap.add_argument("--no-serve-fp64", action="store_true",
                    help="skip the FP64 one-at-a-time comparator of the serving leg")
    ap.add_argument("--no-batch256", action="store_true", help="skip the 256-simulation batch leg")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner leg")
    ap.add_argument("--batch-only", type=int, default=0, metavar="NSIMS",
                    help="run only the config-3 batch leg with NSIMS simulations (half CFD, half MFD) "
                         "and print its JSON (the profiling case of the many-short-lines launches)")
    ap.add_argument("--batch-steps", type=int, default=100, help="graph-captured steps of the batch leg")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="arithmetic of the main batched leg (fp64: the profiling case of the FP64 kernels)")
    ap.add_argument("--solver", default="default", choices=["default", "line", "chunked", "factored"],
                    help="line solver of the FP32 batch (default: the library's choice)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "adi_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def start(self):
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the timed region starts only once sampling is under way
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        res = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return res
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if sm:
            res["sm_mhz"] = float(np.median(sm))
            res["sm_max_mhz"] = float(max(smax))
            res["samples"] = len(sm)
        res["reasons"] = sorted(reasons)
        return res


# The factored line kernel's translation unit and the headers it includes: the committed DRAM
# traffic figure stays valid while these are unchanged.
KERNEL_SOURCES = ("adi_factored.cu", "adi_internal.h", "adi_line.cuh", "adi_ops.cuh")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2006_07583_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic_per_point():
    """DRAM bytes per grid point per stage from the committed ncu summary
    (profiles/line_solve_traffic.txt), valid only while the kernel sources are unchanged since
    the capture."""
    p = os.path.join(ROOT, "profiles", "line_solve_traffic.txt")
    if not os.path.exists(p):
        return None
    d = {}
    for line in open(p):
        if ":" in line and not line.lstrip().startswith("#"):
            k, v = line.split(":", 1)
            d[k.strip()] = v.strip()
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return float(d["dram_bytes_per_point"])


def replica_throughput(local_ms, pts_per_rank, steps, device=None):
    """Whole-job updates/s of N independent replicas: every rank advanced pts_per_rank points by
    `steps` steps; the job's time is the slowest rank's (max over ranks).  Returns
    (updates/s, max ms).  Single process when torch.distributed is not initialised."""
    import torch

    ws = 1
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        ws = torch.distributed.get_world_size()
        t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        local_ms = float(t.item())
    return ws * pts_per_rank * steps / (local_ms / 1e3), local_ms


def make_specs(side, steps):
    from paper_2006_07583_gb300 import workloads as wl

    return [wl.seismic_spec(wl.CFD, side, side, steps, h=5.0, seed=1),
            wl.seismic_spec(wl.MFD, side, side, steps, h=5.0, seed=2)]


def emit(obj):
    print(json.dumps(obj), flush=True)


def run_reference(args):
    """The oracle as it stands, timed on the host cores on the same workload.  Each step is a
    bounded sample of it: one PR step of a horizontal strip of each simulation (full line
    length along x, the expensive direction of the line solves), the strip height chosen from
    a calibration step so that warm-up plus timed steps take about REF_BUDGET_S seconds."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2006_07583_gb300 import workloads as wl

    threads = os.cpu_count() or 1
    specs = make_specs(args.side, args.steps)

    def cases_for(strip):
        out = []
        for sp in specs:
            su, sv, sw = wl.shapes(sp.method, sp.nx, strip)
            c = sp.c[:su[0], :su[1]].copy()
            out.append((sp.method, sp.nx, strip, sp.h, sp.dt, c ** 2, np.zeros(su), np.zeros(sv), np.zeros(sw)))
        return out

    def one(cases):
        for (m, nx, ny, h, dt, kap, U, V, W) in cases:
            oracle.run(m, nx, ny, h, dt, kap, U, V, W, 1, threads=threads)

    # calibration: seconds per strip row of one step
    t0 = time.perf_counter()
    one(cases_for(16))
    per_row = (time.perf_counter() - t0) / 16
    strip = int(args.ref_budget / max(1, args.steps + args.warmup) / max(per_row, 1e-9))
    strip = max(16, min(512, args.side, strip))
    cases = cases_for(strip)
    pts = sum(nx * ny for _, nx, ny, *_ in cases)
    for _ in range(args.warmup):
        one(cases)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one(cases)
    el = time.perf_counter() - t0
    val = pts * args.steps / el
    emit({"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
          "data": "synthetic",
          "config": {"workload": "oracle sample: %d-row strips of the %d^2 CFD+MFD seismic batch"
                                 % (strip, args.side), "global_batch": 2, "side": args.side,
                     "parallelism": "host cores"},
          "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                           "sample": "one PR step of a %dx%d strip of each simulation per step"
                                     % (args.side, strip)},
          "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    return 0


def cpu_baseline_sample(side):
    """Oracle on the host cores on a bounded sample of the bench workload (a 256-row strip
    of each 4096-wide simulation, one PR step), scaled to updates/s."""
    import oracle
    from paper_2006_07583_gb300 import workloads as wl

    def sample(strip, threads):
        pts = 0
        t0 = time.perf_counter()
        for sp in make_specs(side, 1):
            su, sv, sw = wl.shapes(sp.method, sp.nx, strip)
            c = sp.c[:su[0], :su[1]].copy()
            oracle.run(sp.method, sp.nx, strip, sp.h, sp.dt, c ** 2, np.zeros(su), np.zeros(sv),
                       np.zeros(sw), 1, threads=threads)
            pts += sp.nx * strip
        return pts, time.perf_counter() - t0

    threads = os.cpu_count() or 1
    pts, el = sample(256, threads)
    pts1, el1 = sample(32, 1)
    return {"value": pts / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "one PR step of a %dx256 strip of each of the two simulations "
                      "(%.1f s of CPU wall time)" % (side, el),
            "single_thread": {"value": pts1 / el1, "unit": UNIT, "cores": 1,
                              "sample": "one PR step of a %dx32 strip of each simulation "
                                        "(%.1f s)" % (side, el1)}}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    ws, rank, local = dist_env()
    import torch

    torch.cuda.set_device(local)
    if args.batch_only:
        from paper_2006_07583_gb300 import adi

        adi.lib()
        peak, _ = measured_peaks()
        emit(batch256_leg(adi, torch, peak, steps=args.batch_steps, n_sims=args.batch_only))
        return 0
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2006_07583_gb300 import adi

    adi.lib()
    specs = make_specs(args.side, args.steps)
    sims = []
    for sp in specs:
        kw = {} if args.solver == "default" else {"solver": getattr(adi, "ADI_SOLVER_" + args.solver.upper())}
        prec = adi.ADI_FP64 if args.precision == "fp64" else adi.ADI_FP32
        s = adi.Sim(sp.method, sp.nx, sp.ny, sp.h, sp.dt, sp.c, precision=prec, **kw)
        s.set_source(*sp.source.as_tuple())
        sims.append(s)
    batch = adi.Batch(sims)
    stream = torch.cuda.Stream()
    batch.set_stream(stream.cuda_stream)
    pts = sum(sp.nx * sp.ny for sp in specs)

    for _ in range(args.warmup):
        batch.half_step(1)
        batch.half_step(2)
    stream.synchronize()

    clocks = ClockSampler(local)
    K = args.steps
    batch.set_timing(True)  # CUDA events around the line-solve launches of every half step
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K + 1)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(K):
            batch.half_step(1)
            ev[2 * k + 1].record(stream)
            batch.half_step(2, write_natural=(k == K - 1))
            ev[2 * k + 2].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    ck = clocks.stop()
    if ws > 1:
        torch.distributed.barrier()
    st1 = [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(K)]
    st2 = [ev[2 * k + 1].elapsed_time(ev[2 * k + 2]) for k in range(K)]
    solve_ms = {}
    for stage in (1, 2):
        tot, n = batch.solve_time(stage)
        solve_ms[stage] = tot / max(n, 1)
    step_ms = [a + b for a, b in zip(st1, st2)]
    value, total_ms = replica_throughput(ev[0].elapsed_time(ev[2 * K]), pts, K, device="cuda")

    # roofline of the dominant kernel, the line solve (one launch per kernel variant, CFD and
    # MFD, per stage; timed by events recorded around those launches only), algorithmic bytes:
    # each stage reads the carried pressure, the velocity and alpha and writes the first two
    # -> 5 words per grid point (20 B in FP32) over both simulations.
    peak, peak_kind = measured_peaks()
    esz = 8 if args.precision == "fp64" else 4
    alg_bytes = 5 * esz * pts
    avg1, avg2 = float(np.mean(st1)), float(np.mean(st2))
    dom_stage = 1 if solve_ms[1] >= solve_ms[2] else 2
    dom_ms = solve_ms[dom_stage]
    achieved = alg_bytes / (dom_ms / 1e3) / 1e9
    tpp = ncu_traffic_per_point() if esz == 4 else None  # the committed figure is the FP32 kernels'
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": (tpp * pts if tpp is not None else None),
            "kernel": "line_solve_factored_kernel (stage %d, CFD + MFD launches)" % dom_stage,
            "alg_bytes_per_launch": alg_bytes, "peak_kind": peak_kind,
            "solve_ms": {"x_lines": solve_ms[1], "y_lines": solve_ms[2]},
            "stage_ms_with_transpose": {"x_lines": avg1, "y_lines": avg2},
            # the natural (u, v, w) formulation would move 7 words per point and stage
            "frac_natural_state": achieved * 7 / 5 / peak}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
           "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64" if esz == 8 else "f32",
           "data": "synthetic",
           "config": {"workload": "batched %s PR-ADI, 1 CFD + 1 MFD seismic sim at "
                                  "%dx%d cells" % (args.precision.upper(), args.side, args.side),
                      "global_batch": 2 * ws, "side": args.side,
                      "parallelism": "replicas x%d" % ws, "l2": "inputs larger than L2",
                      "h_m": 5.0, "source": "15 Hz Ricker",
                      "solver": {0: "line", 1: "chunked", 2: "factored"}[sims[0].solver]},
           "latency_ms": {"p50_step": float(np.percentile(step_ms, 50)),
                          "p99_step": float(np.percentile(step_ms, 99))},
           "clocks": ck, "roofline": roof,
           "gpu_launches": 2 * K * (len({sp.method for sp in specs}) + 1)}

    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_leg(adi, torch, sims, batch, specs, min(K, 8), f32=esz == 4, overlap=True)
        out["e2e_sequential"] = e2e_leg(adi, torch, sims, batch, specs, min(K, 8), f32=esz == 4)
        if esz == 4:
            out["e2e_fp64_host"] = e2e_leg(adi, torch, sims, batch, specs, min(K, 8), f32=False)
    if rank == 0 and not args.no_fp64:
        out["fp64_plain"] = fp64_plain(adi, args.side)
    batch.close()
    for s in sims:
        s.close()
    if rank == 0 and not args.no_fp64:
        out["fp64_factored"] = fp64_factored_leg(adi, torch, args.side, peak)
    if rank == 0 and not args.no_batch256:
        out["batch256"] = batch256_leg(adi, torch, peak, steps=args.batch_steps)
    if rank == 0 and not args.no_serve:
        out["serving"] = serving_leg(adi, args.serve_requests, not args.no_serve_fp64)
    if rank == 0 and not args.no_tune:
        out["autotune"] = tune_leg(adi)
    if rank == 0 and not args.no_peak:
        out["peak_8192"] = peak_leg(adi, torch, 8192, 20, peak)
    if rank == 0 and not args.no_paper:
        out["paper_iteration"] = paper_leg(adi, args.side)
    if rank == 0 and ws == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline_sample(args.side)
    if rank == 0:
        emit(out)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def peak_leg(adi, torch, side, steps, peak):
    """The 8192^2 FP32 heterogeneous roofline run: one CFD and one MFD seismic simulation of
    side^2 cells batched (split-line factored solver), `steps` graph-free half-step pairs after
    three warm-up steps, CUDA events on the batch's stream."""
    specs = make_specs(side, steps)
    sims = []
    for sp in specs:
        s = adi.Sim(sp.method, sp.nx, sp.ny, sp.h, sp.dt, sp.c, precision=adi.ADI_FP32)
        s.set_source(*sp.source.as_tuple())
        sims.append(s)
    b = adi.Batch(sims)
    stream = torch.cuda.Stream()
    b.set_stream(stream.cuda_stream)
    for _ in range(3):
        b.half_step(1)
        b.half_step(2)
    stream.synchronize()
    b.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(steps):
            b.half_step(1)
            b.half_step(2)
        e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / steps
    solve = [b.solve_time(st) for st in (1, 2)]
    solve_ms = max(t / max(n, 1) for t, n in solve)
    pts = sum(sp.nx * sp.ny for sp in specs)
    achieved = 5 * 4 * pts / (solve_ms / 1e3) / 1e9
    solver = {0: "line", 1: "chunked", 2: "factored"}[sims[0].solver]
    b.close()
    for s in sims:
        s.close()
    return {"workload": "batched FP32 PR-ADI, 1 CFD + 1 MFD seismic sim at %dx%d cells" % (side, side),
            "value": pts / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "solver": solver + (" (split lines)" if solver == "factored" else ""),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "solve_ms": solve_ms}}


def paper_leg(adi, side, steps=2, kmax=6):
    """The paper's own stage solver on this GPU for comparison: the fixed-point iteration of
    Eq. 9 with kmax sweeps per stage (no early stop), one thread per line, on the same two
    simulations, FP32; device time of the steps."""
    pts, ms = 0, 0.0
    for sp in make_specs(side, steps):
        from paper_2006_07583_gb300 import workloads as wl

        su, sv, sw = wl.shapes(sp.method, sp.nx, sp.ny)
        _, _, _, sweeps, t = adi.fixed_point(sp.method, sp.nx, sp.ny, sp.h, sp.dt, sp.c, np.zeros(su),
                                             np.zeros(sv), np.zeros(sw), steps, source=sp.source.as_tuple(),
                                             kmax=kmax, eps=0.0, precision=adi.ADI_FP32)
        pts += sp.nx * sp.ny
        ms += t / steps
    return {"workload": "the paper's fixed-point stage solver (Eq. 9, %d sweeps per stage, one thread "
                        "per line), same two %dx%d simulations, FP32, one after the other" % (kmax, side, side),
            "value": pts / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps}


def e2e_leg(adi, torch, sims, batch, specs, n, f32=True, overlap=False):
    """Same metric through the public API with host buffers: every step uploads each
    member's fields from pinned host memory (adi_set_fields_f32, or adi_set_fields with FP64
    arrays), advances the batch one step and reads the fields back (adi_read_fields_f32 /
    adi_read_fields); wall-clock timed.  overlap: one host thread per member, as a user
    driving several simulations would run them: the members read their results in turn, so
    one member's upload (and its carried-state rebuild) overlaps the next member's readback
    on the other direction of the host link; each member still uploads exactly the fields it
    read back the step before."""
    from paper_2006_07583_gb300 import workloads as wl

    dt = torch.float32 if f32 else torch.float64
    bufs = []
    for sp in specs:
        shp = wl.shapes(sp.method, sp.nx, sp.ny)
        bufs.append([torch.zeros(s, dtype=dt, pin_memory=True).numpy() for s in shp])
    h2d = sum(sum(b.nbytes for b in bb) for bb in bufs)
    read = (lambda s, bb: s.read_into_f32(*bb)) if f32 else (lambda s, bb: s.read_into(*bb))
    write = (lambda s, bb: s.set_fields_f32(*bb)) if f32 else (lambda s, bb: s.set_fields(*bb))
    batch.sync()
    for s, bb in zip(sims, bufs):
        read(s, bb)
    for s, bb in zip(sims, bufs):  # one untimed round trip: first-use buffers are set up here
        write(s, bb)
    batch.step(1)
    batch.sync()
    for s, bb in zip(sims, bufs):
        read(s, bb)
    if not overlap:
        t0 = time.perf_counter()
        for _ in range(n):
            for s, bb in zip(sims, bufs):
                write(s, bb)
            batch.step(1)
            batch.sync()
            for s, bb in zip(sims, bufs):
                read(s, bb)
        el = time.perf_counter() - t0
    else:
        import threading

        m = len(sims)
        bar = threading.Barrier(m + 1)
        turn = [threading.Semaphore(1 if i == 0 else 0) for i in range(m)]
        errors = []

        def member(i):
            try:
                for _ in range(n):
                    write(sims[i], bufs[i])
                    bar.wait()  # every member uploaded: the batch steps
                    bar.wait()  # the step is done
                    turn[i].acquire()  # members read in turn
                    read(sims[i], bufs[i])
                    turn[(i + 1) % m].release()
            except Exception as e:  # noqa: BLE001 - reported below
                errors.append(e)
                bar.abort()

        threads = [threading.Thread(target=member, args=(i,)) for i in range(m)]
        t0 = time.perf_counter()
        for t in threads:
            t.start()
        try:
            for _ in range(n):
                bar.wait()
                batch.step(1)
                batch.sync()
                bar.wait()
        except threading.BrokenBarrierError:
            pass
        for t in threads:
            t.join()
        el = time.perf_counter() - t0
        if errors:
            raise errors[0]
    pts = sum(sp.nx * sp.ny for sp in specs)
    api = "adi_set_fields_f32 / adi_read_fields_f32" if f32 else "adi_set_fields / adi_read_fields (FP64)"
    if overlap:
        api += ", one host thread per simulation (readbacks in turn)"
    return {"value": pts * n / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": h2d, "steps": n, "api": api}


def _run_server(adi, reqs, arrivals, budget=150 << 30):
    """One pass of the serving loop over `reqs` arriving at `arrivals` (seconds from the start):
    returns (wall seconds, latencies in ms from submission to completion)."""
    srv = adi.Server(budget, precision=adi.ADI_FP32, quantum=100, max_active=64)
    order = sorted(range(len(reqs)), key=lambda k: arrivals[k])
    tickets = []
    t0 = time.perf_counter()
    nxt, running, pending = 0, 0, 0
    while True:
        now = time.perf_counter() - t0
        submitted = False
        while nxt < len(order) and arrivals[order[nxt]] <= now:
            sp = reqs[order[nxt]].spec
            tickets.append(srv.submit(sp.method, sp.nx, sp.ny, sp.h, sp.dt, sp.c, sp.steps,
                                      source=sp.source.as_tuple()))
            nxt += 1
            submitted = True
        if running or pending or submitted:
            running, pending = srv.tick()
        elif nxt < len(order):
            time.sleep(max(0.0, min(0.01, arrivals[order[nxt]] - now)))
        else:
            break
    wall = time.perf_counter() - t0
    lat = []
    for t in tickets:
        _st, ts, _ta, td = srv.status(t)
        lat.append(1e3 * (td - ts))
    srv.close()
    return wall, lat


def _one_at_a_time(adi, reqs, precision):
    """Every request alone, one after the other, with the library's default solver: create,
    source, steps, read the fields back, destroy -- the same per-request work the serving loop
    does (creation at admission, results read at retirement).  Wall-clock seconds."""
    t0 = time.perf_counter()
    for r in reqs:
        sp = r.spec
        s = adi.Sim(sp.method, sp.nx, sp.ny, sp.h, sp.dt, sp.c, precision=precision)
        s.set_source(*sp.source.as_tuple())
        s.step(sp.steps)
        s.read()
        s.close()
    return time.perf_counter() - t0


def serving_leg(adi, n_req, with_fp64=True):
    """The serving loop (adi_server_*) on the config-4 request stream: square grids with sides
    log-uniform in [64, 4096], 100-5000 steps, CFD/MFD 50/50, FP32, 150 GB HBM budget, seeded
    Poisson arrivals.  Capacity is the throughput with every request submitted at once; the
    offered load is then swept over 0.5, 0.8, 1.0 and 1.2 x capacity (same requests, arrival
    times of one seeded Poisson stream scaled to the rate).  Comparators on the same full
    request set: the default (factored) solver one simulation at a time in FP32 -- isolating
    what continuous batching gains -- and in FP64, the plain one-at-a-time FP64 path."""
    from paper_2006_07583_gb300 import workloads as wl

    reqs = wl.serving_stream(n_req, 1.0, seed=3)  # arrivals at rate 1/s, rescaled below
    work = float(sum(r.spec.points * r.spec.steps for r in reqs))
    mean_work = work / len(reqs)
    wall_sat, lat_sat = _run_server(adi, reqs, [0.0] * len(reqs))
    capacity = work / wall_sat
    loads = {}
    for f in (0.5, 0.8, 1.0, 1.2):
        rate = f * capacity / mean_work
        wall, lat = _run_server(adi, reqs, [r.arrival / rate for r in reqs])
        loads["%.1f" % f] = {"offered_rate_per_s": rate, "wall_s": wall, "value": work / wall,
                             "p50_ms": float(np.percentile(lat, 50)),
                             "p99_ms": float(np.percentile(lat, 99))}
    out = {"requests": len(reqs), "updates": work, "unit": UNIT,
           "capacity": {"value": capacity, "wall_s": wall_sat, "p50_ms": float(np.percentile(lat_sat, 50)),
                        "p99_ms": float(np.percentile(lat_sat, 99))},
           "loads": loads,
           # headline: throughput at saturation (comparable with the one-at-a-time arms, which
           # also run back to back), latency at an offered load of 0.8 x capacity
           "value": capacity, "p50_ms": loads["0.8"]["p50_ms"], "p99_ms": loads["0.8"]["p99_ms"],
           "workload": "config 4: Poisson stream of %d requests, sides log-uniform 64-4096, 100-5000 "
                       "steps, CFD/MFD, FP32, 150 GB budget, quantum 100 steps" % len(reqs)}
    t32 = _one_at_a_time(adi, reqs, adi.ADI_FP32)
    out["fp32_one_at_a_time"] = {"value": work / t32, "unit": UNIT, "wall_s": t32, "requests": len(reqs)}
    if with_fp64:
        t64 = _one_at_a_time(adi, reqs, adi.ADI_FP64)
        out["fp64_one_at_a_time"] = {"value": work / t64, "unit": UNIT, "wall_s": t64, "requests": len(reqs)}
    return out


def tune_leg(adi, sides=(256, 1024, 4096, 8192)):
    """adi_autotune on single FP32 seismic simulations per size class: ms per step of every
    solver with the automatic launch, and of the factored solver with the launch parameters the
    tuner keeps (lines per CTA cap, ring depth cap; 0 = automatic)."""
    from paper_2006_07583_gb300 import workloads as wl

    names = {0: "line", 1: "chunked", 2: "factored"}
    out = {}
    for side in sides:
        for method in (wl.CFD, wl.MFD):
            sp = wl.seismic_spec(method, side, side, 4, h=5.0, seed=5)
            s = adi.Sim(sp.method, sp.nx, sp.ny, sp.h, sp.dt, sp.c, precision=adi.ADI_FP32)
            s.set_source(*sp.source.as_tuple())
            chosen, ms = s.autotune(trials=4, force=True)
            cap, ring = s.launch()
            s.step(8)  # graph capture of the 8-step loop
            s.sync()
            t0 = time.perf_counter()
            s.step(8)
            s.sync()
            tuned = 1e3 * (time.perf_counter() - t0) / 8
            s.close()
            out["%s_%d" % (wl.METHOD_NAMES[method], side)] = {
                "ms_per_step": {names[k]: v for k, v in ms.items()}, "chosen": names[chosen],
                "lines_per_cta_cap": cap, "ring_cap": ring, "tuned_wall_ms_per_step": tuned}
    return out


def batch256_leg(adi, torch, peak, steps=100, n_sims=256):
    """Config 3: 256 independent simulations (128 CFD + 128 MFD), sides uniform in [128, 1024],
    seeded layered media, Ricker sources, FP32, batched.  `steps` graph-captured steps after
    warm-up, CUDA events on the batch's stream; then a few half-step pairs with events around
    the solve launches for the kernels' roofline (20 B per point and stage).  A smaller n_sims
    draws a smaller batch the same way, half CFD and half MFD (the profiling case)."""
    from paper_2006_07583_gb300 import workloads as wl

    specs = wl.batch_specs(n_sims, 128, 1024, steps, seed=2)
    sims = []
    for sp in specs:
        s = adi.Sim(sp.method, sp.nx, sp.ny, sp.h, sp.dt, sp.c, precision=adi.ADI_FP32)
        s.set_source(*sp.source.as_tuple())
        sims.append(s)
    b = adi.Batch(sims)
    stream = torch.cuda.Stream()
    b.set_stream(stream.cuda_stream)
    b.step(steps)  # graph capture and warm-up
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / steps
    b.set_timing(True)
    for _ in range(10):
        b.half_step(1)
        b.half_step(2)
    solve = [b.solve_time(st) for st in (1, 2)]
    solve_ms = max(t / max(n, 1) for t, n in solve)
    pts = sum(sp.nx * sp.ny for sp in specs)
    achieved = 5 * 4 * pts / (solve_ms / 1e3) / 1e9
    b.close()
    for s in sims:
        s.close()
    return {"workload": "config 3: %d sims (%d CFD + %d MFD), sides uniform 128-1024, FP32, "
                        "one batch, graph-captured steps" % (n_sims, n_sims // 2, n_sims - n_sims // 2),
            "value": pts / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms, "steps": steps, "points": pts,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "solve_ms": solve_ms}}


def fp64_factored_leg(adi, torch, side, peak, steps=4):
    """The default (factored) solver in FP64 on the bench's two 4096^2 simulations, batched:
    updates/s, the solve kernels' fraction of HBM (40 B per point and stage in FP64), and the
    device's measured FP64 and FP32 FMA throughput (adi_fma_peak) for the ALU roofline."""
    specs = make_specs(side, steps)
    sims = []
    for sp in specs:
        s = adi.Sim(sp.method, sp.nx, sp.ny, sp.h, sp.dt, sp.c, precision=adi.ADI_FP64)
        s.set_source(*sp.source.as_tuple())
        sims.append(s)
    b = adi.Batch(sims)
    stream = torch.cuda.Stream()
    b.set_stream(stream.cuda_stream)
    b.half_step(1)
    b.half_step(2)
    stream.synchronize()
    b.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(steps):
            b.half_step(1)
            b.half_step(2)
        e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / steps
    solve = [b.solve_time(st) for st in (1, 2)]
    solve_ms = max(t / max(n, 1) for t, n in solve)
    pts = sum(sp.nx * sp.ny for sp in specs)
    solver = {0: "line", 1: "chunked", 2: "factored"}[sims[0].solver]
    b.close()
    for s in sims:
        s.close()
    hbm = 5 * 8 * pts / (solve_ms / 1e3) / 1e9
    return {"workload": "batched FP64 PR-ADI, 1 CFD + 1 MFD seismic sim at %dx%d cells" % (side, side),
            "value": pts / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "solver": solver,
            "solve_ms": solve_ms, "hbm_frac": hbm / peak, "hbm_achieved_gbs": hbm,
            "fma_peak_tflops": {"fp64": adi.fma_peak(adi.ADI_FP64) / 1e12,
                                "fp32": adi.fma_peak(adi.ADI_FP32) / 1e12}}


def fp64_plain(adi, side):
    """The plain one-simulation-at-a-time FP64 GPU path on the same two simulations."""
    import torch

    specs = make_specs(side, 2)
    tot_pts, tot_s = 0, 0.0
    for sp in specs:
        s = adi.Sim(sp.method, sp.nx, sp.ny, sp.h, sp.dt, sp.c, precision=adi.ADI_FP64,
                    solver=adi.ADI_SOLVER_LINE)
        s.set_source(*sp.source.as_tuple())
        s.step(1)
        s.sync()
        t0 = time.perf_counter()
        s.step(2)
        s.sync()
        tot_s += time.perf_counter() - t0
        tot_pts += 2 * sp.nx * sp.ny
        s.close()
    return {"value": tot_pts / tot_s, "unit": UNIT, "steps": 2,
            "workload": "one sim at a time, FP64, %dx%d CFD then MFD" % (side, side)}


if __name__ == "__main__":
    sys.exit(main())
