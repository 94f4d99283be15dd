#!/usr/bin/env python
"""Benchmark of the MUSTA-FORCE hot path on B300.

Workload (default): 3-D spherical blast on a 256^3 grid over [-1, 1]^3,
p = e/3, e = 10 inside r < 0.2 and 1 outside, v = 0, periodic boundaries,
minmod limiter, 2 MUSTA stages, RK2 with the Hancock half step, Strang
splitting, CFL 0.4, FP32 state.  One step = CFL rate reduction + dt + 5
directional sweeps.  Metric: cell-updates/s (cells x steps / time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload blast256_fp32|blast256_fp64|blast128_fp32|...]
                  [--launch THREADS,SEGMENTS] [--no-cpu] [--no-e2e] [--no-batch]

The default line also carries, as a nested "batch" object, the event-by-event
batch (512 events of 64^3..160^3 cells) in events/s over --batch-steps steps.

Under torchrun each rank runs its own replica of the workload on its own GPU
(the hot path has no data exchange between grids); value is the whole-job
rate, the max time over ranks.  --impl reference times the FP64 CPU oracle on
the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "blast256_fp32": dict(n=256, prec="fp32"),
    "blast256_fp64": dict(n=256, prec="fp64"),
    "blast128_fp32": dict(n=128, prec="fp32"),   # small case for ncu captures
    # the paper's production settings (Sec. 3.2): RK3 and 4 MUSTA stages
    "blast256_paper": dict(n=256, prec="fp32", rk=3, stages=4),
    # the unsplit multi-D scheme (Eq. 13 with every flux term, alpha = 3)
    "blast256_unsplit": dict(n=256, prec="fp32", unsplit=True),
}
BYTES = {"fp32": 4, "fp64": 8}
# Algorithmic floating-point operations per cell of one sweep (conformal EOS,
# RK with the Hancock half step), keyed by (limiter, MUSTA stages, RK order):
# the oracle's op-counting build (distinct add, sub, mul, div, sqrt, min, max
# on state-derived values that reach the output) on a pencil where every cell
# takes the general path.  A CPU test checks these numbers against that build.
FLOPS_PER_CELL_SWEEP = {("minmod", 2, 2): 672, ("mc", 2, 2): 704, ("superbee", 2, 2): 696,
                        ("minmod", 4, 3): 1812}
# the same count for one RK stage of the unsplit scheme (alpha 3), keyed by
# (MUSTA stages, RK order); central slopes count as many operations as Minbee
FLOPS_PER_CELL_STAGE_UNSPLIT = {(2, 2): 1016}


def flops_per_cell_sweep(rk=2, stages=2, limiter="minmod"):
    return FLOPS_PER_CELL_SWEEP.get((limiter, stages, rk))


# FP32 (non-tensor) peak from unit counts and clock: 148 SMs x 128 FP32 lanes x
# 2 flop per FMA x 2.032 GHz; FP64 from the B300's nominal 1.25 TFLOP/s.
# DRAM bytes read + written per sweep launch, mean over the five sweeps of one
# step (for the unsplit scheme: per RK stage, faces + tile kernel, mean over
# the two stages of a step), from ncu captures of the current kernels (the
# sweep and unsplit profile summaries under profiles/); None where no capture
# of the current kernels exists
SWEEP_TRAFFIC = {(256, "fp32", 2, 2, False): 595.2e6,
                 (256, "fp32", 2, 2, True): 5043.2e6}
# the event batch (FP32, minmod, k = 2, RK2): DRAM bytes per cell and sweep
# launch, the mean over one step's five sweeps of an ncu capture of 64 events
# of the batch recipe (1.10e8 cells, 3.3 GB held on the device), scaled by
# cells to the full batch (the profile summary of the batch sweep under
# profiles/); 32 B per cell is algorithmic
BATCH_TRAFFIC_PER_CELL = 45.38


def bytes_per_cell_stage_unsplit(elem):
    """Algorithmic HBM bytes of one unsplit RK stage per cell: 6 faces written
    and read (the interface fluxes stay in shared memory), the input state
    read, the RK inputs read and the result written (4 fields each)."""
    return (2 * 24 + 4 + 8 + 4) * elem


ALU_PEAK_TFLOPS = {"fp32": 148 * 128 * 2 * 2.032e9 / 1e12, "fp64": 1.25}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def host_info():
    """Host cores and CPU model, for the CPU baseline."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    return {"nproc": usable, "cpu_model": model}


def cpu_baseline_oracle(n=96, steps=1, rk=2, stages=2, unsplit=False, limiter="minmod",
                        threads=False):
    """The oracle, as it stands, on a bounded sample: the blast recipe on n^3.
    threads=True runs its OpenMP timing build (pencils of each sweep split
    over all host threads; bitwise the same result).  Returns (cell-updates/s,
    seconds, threads used, sample description)."""
    from oracle import oracle as O
    from paper_1510_06340_b300 import inputs as I
    g, prim = I.spherical_blast(n)
    o = O.Oracle(n, n, n, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, bc="periodic",
                 limiter=limiter, stages=stages, rk_order=rk, cfl=0.4,
                 alpha=3.0 if unsplit else 1.0, unsplit=int(unsplit))
    U = o.prim2cons_field(*prim)
    nthr = O.lib_omp().or_threads() if threads else 1
    t0 = time.perf_counter()
    o.run(U, steps, threads=threads)
    el = time.perf_counter() - t0
    # the unsplit scheme has no OpenMP split: it runs on one thread either way
    if unsplit:
        nthr = 1
    return (n ** 3 * steps / el, el, nthr,
            f"blast recipe on {n}^3 (same physics, smaller grid), {steps} step(s)")


def cpu_baseline_block(rk=2, stages=2, unsplit=False, limiter="minmod"):
    """cpu_baseline of the blast lines: the oracle on all host threads (the
    value) and on one thread, with the host described."""
    nb1 = 96 if (rk, stages) == (2, 2) else 64   # about 2 s of one core
    v1, el1, _, s1 = cpu_baseline_oracle(nb1, 1, rk, stages, unsplit, limiter)
    host = host_info()
    nbt = 128 if (rk, stages) == (2, 2) and not unsplit else nb1
    vt, elt, thr, st = cpu_baseline_oracle(nbt, 2, rk, stages, unsplit, limiter, threads=True)
    return {"value": vt, "unit": "cell-updates/s", "cores": thr, "kind": "oracle",
            "sample": st + f", {elt:.1f} s, OpenMP over pencils",
            "single_thread": {"value": v1, "cores": 1, "sample": s1 + f", {el1:.1f} s"},
            "host": host}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    n = 96
    for _ in range(args.warmup):
        cpu_baseline_oracle(n, 1, threads=True)
    total, thr = 0.0, 1
    for _ in range(args.steps):
        r, el, thr, sample = cpu_baseline_oracle(n, 1, threads=True)
        total += el
    value = n ** 3 * args.steps / total
    line = {"impl": "reference", "metric": "cell_updates_per_s", "value": value,
            "unit": "cell-updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "3D spherical blast, p=e/3, minmod, "
                                            "2 MUSTA stages, RK2+Hancock, Strang, periodic; "
                                            f"oracle sample {n}^3 per step"},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": thr,
                             "kind": "oracle",
                             "sample": f"blast recipe on {n}^3, 1 step per timed step, "
                                       "OpenMP over pencils on all host threads",
                             "host": host_info()},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1510_06340_b300 import build, hydro
    from paper_1510_06340_b300 import inputs as I
    if rank == 0:
        build.build(verbose=False)
    if world > 1:
        dist.barrier()
    wl = WORKLOADS[args.workload]
    n, prec = wl["n"], wl["prec"]
    rk, stages = wl.get("rk", 2), wl.get("stages", 2)
    unsplit = wl.get("unsplit", False)
    flops_cell_sweep = flops_per_cell_sweep(rk, stages, args.limiter)
    dt_np = np.float64 if prec == "fp64" else np.float32
    g, prim = I.spherical_blast(n)
    prim = [np.ascontiguousarray(a, dtype=dt_np) for a in prim]
    stream = torch.cuda.Stream()
    grid = hydro.make_grid(n, n, n, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, bc="periodic",
                           prec=prec, cfl=0.4, rk_order=rk, unsplit=unsplit)
    h = hydro.Hydro(grid, limiter=args.limiter, stages=stages, stream=stream)
    h.set_primitives(*prim)
    cells = n ** 3
    if args.launch:
        th, sg = (int(x) for x in args.launch.split(","))
        for ax in range(3):
            h.force_launch(ax, th, sg)

    # warm-up (first call also autotunes the launch shapes)
    h.step(args.warmup)
    torch.cuda.synchronize()

    # timed region: device-resident state (2 x state > L2), per-sweep CUDA events
    h.set_kernel_timing(True)
    h.kernel_timing()   # reset
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t_sim0 = h.time()
    with Clocks(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        h.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = e0.elapsed_time(e1)
    t_sim = h.time() - t_sim0
    (sweep_ms, other_ms), (n_sweep, n_other) = h.kernel_timing()
    shapes = [h.get_launch(ax) for ax in range(3)]
    h.set_kernel_timing(False)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * cells * args.steps / (ms * 1e-3)

    # e2e through the public API with host buffers: upload initial primitives
    # from pinned memory, step, read each step's conservation sums, read back
    # the final primitives.
    e2e_value = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(a).pin_memory() for a in prim]
        result = [torch.empty(a.shape, dtype=pinned[0].dtype).pin_memory() for a in prim]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.set_primitives(*[p.numpy() for p in pinned])
        for _ in range(args.steps):
            h.step(1)
            h.conservation_sums()
        h.get_primitives(out=result)
        torch.cuda.synchronize()
        e2e_value = world * cells * args.steps / (time.perf_counter() - t0)
    state_bytes = 4 * cells * BYTES[prec]

    hbm, src = peaks()
    avg_sweep_ms = sweep_ms / max(n_sweep, 1)
    if unsplit:
        # a timed group is one RK stage: faces, then fluxes + update per tile
        bytes_per_sweep = bytes_per_cell_stage_unsplit(BYTES[prec]) * cells
        fpc = FLOPS_PER_CELL_STAGE_UNSPLIT.get((stages, rk))
        launches = 2 * n_sweep + n_other
        kernel_name = "unsplit RK stage (k_us_faces, k_us_tile)"
    else:
        bytes_per_sweep = 2 * 4 * BYTES[prec] * cells      # read + write of 4 fields
        fpc = flops_cell_sweep
        # per step: 5 sweeps + k_dt (the CFL rate is fused into the last sweep)
        launches = n_sweep + n_other
        kernel_name = "k_sweep (one directional sweep, all RK stages)"
    flops_per_group = fpc * cells if fpc else None
    achieved = bytes_per_sweep / (avg_sweep_ms * 1e-3) / 1e9
    alu_peak = ALU_PEAK_TFLOPS[prec]
    flops_achieved = flops_per_group / (avg_sweep_ms * 1e-3) / 1e12 if fpc else None
    traffic = (SWEEP_TRAFFIC.get((n, prec, rk, stages, unsplit))
               if args.limiter == "minmod" else None)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline_block(rk, stages, unsplit, args.limiter)
    batch = None
    if rank == 0 and world == 1 and not args.no_batch and not unsplit:
        del h
        torch.cuda.empty_cache()
        batch = batch_measure(args.events, args.batch_steps, 3, stream, local, args.no_cpu)
    if rank == 0:
        line = {
            "metric": "cell_updates_per_s", "value": value, "unit": "cell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": f"3D spherical blast {n}^3 on [-1,1]^3, p=e/3, "
                                   f"{prec.upper()}, {args.limiter}, {stages} MUSTA stages, "
                                   f"RK{rk}+Hancock, "
                                   f"{'unsplit, alpha 3' if unsplit else 'Strang'}, periodic, "
                                   "CFL 0.4",
                       "cells": cells, "parallelism": f"replicas x{world}",
                       "launch_threads_segments_xyz": shapes,
                       "l2": "inputs larger than L2 (two state copies of "
                             f"{state_bytes / 1e6:.0f} MB)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "kernel": kernel_name,
                         "algorithmic_bytes_per_launch": bytes_per_sweep,
                         "avg_launch_ms": avg_sweep_ms,
                         "peak_source": f"{src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
            "roofline_alu": {"bound": "alu", "achieved": flops_achieved, "peak": alu_peak,
                             "unit": "TFLOP/s",
                             "frac": flops_achieved / alu_peak if fpc else None,
                             "kernel": kernel_name,
                             "algorithmic_flops_per_cell": fpc,
                             "algorithmic_flops_per_launch": flops_per_group,
                             "flops_source": "oracle op-counting build (distinct add, sub, mul, "
                                             "div, sqrt, min, max reaching the output)",
                             "avg_launch_ms": avg_sweep_ms,
                             "peak_source": "derived: 148 SM x 128 lanes x 2 x 2.032 GHz "
                                            "(fp32); nominal 1.25 TFLOP/s (fp64)"},
            "kernel_ms": {"sweeps": sweep_ms, "sweep_launches": n_sweep,
                          "rate_dt": other_ms, "rate_dt_groups": n_other},
            "gpu_launches": launches,
            "physical_time_per_s": t_sim / (ms * 1e-3),
            "e2e": {"value": e2e_value, "unit": "cell-updates/s",
                    "h2d_bytes_per_step": state_bytes / args.steps,
                    "d2h_bytes_per_step": 32 + state_bytes / args.steps},
            "clocks": clk.summary(),
        }
        if cpu:
            line["cpu_baseline"] = cpu
        if batch:
            line["batch"] = batch
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def batch_cpu_baseline(mean_cells):
    """The oracle (OpenMP timing build, all host threads) on one 64^3 event of
    the batch recipe (hot spots + jet, outflow, FP64) for 2 steps; events/s
    extrapolated as cell-updates/s / (mean cells per event x 100 steps)."""
    from oracle import oracle as O
    from paper_1510_06340_b300 import inputs as I
    n = 64
    g = I.event_grid(n, 0.1)
    prim = I.hotspot_primitives(g, I.hotspots(0))
    o = O.Oracle(n, n, n, dx=0.1, x0=g["x0"], y0=g["y0"], z0=g["z0"], bc="outflow",
                 limiter="minmod", stages=2, rk_order=2, cfl=0.4, jet=I.jet(0))
    U = o.prim2cons_field(*prim)
    t0 = time.perf_counter()
    o.run(U, 2, threads=True)
    el = time.perf_counter() - t0
    rate = n ** 3 * 2 / el
    return {"value": rate / (mean_cells * 100), "unit": "events/s (100 steps each)",
            "cores": O.lib_omp().or_threads(), "kind": "oracle",
            "sample": f"one {n}^3 event of the batch recipe, 2 steps, {el:.1f} s, OpenMP over "
                      f"pencils; {rate:.3g} cell-updates/s extrapolated to the batch's mean "
                      f"event of {mean_cells:.3g} cells and 100 steps",
            "host": host_info()}


def batch_measure(nev, steps, warmup, stream, gpu, no_cpu=False):
    """The event-by-event batch on one GPU, as a nested object of the default
    line: nev events (grids uniform on 64^3..160^3, dx = 0.1 fm) of 416 Gaussian
    hot spots plus a jet, FP32, minmod, 2 MUSTA stages, RK2 + Hancock, Strang,
    outflow, one launch per sweep over all events, steps replayed as a CUDA
    graph.  Metric: events/s (events x steps / 100 per second)."""
    import torch
    from paper_1510_06340_b300 import hydro
    from paper_1510_06340_b300 import inputs as I
    sizes = I.event_sizes(nev)
    grids, spots, jets = [], [], []
    for e, n in enumerate(sizes):
        g = I.event_grid(int(n), 0.1)
        grids.append(hydro.make_grid(int(n), int(n), int(n), dx=0.1, x0=g["x0"], y0=g["y0"],
                                     z0=g["z0"], bc="outflow", prec="fp32", cfl=0.4))
        spots.append(I.hotspots(e))
        jets.append(I.jet(e))
    spots, jets = np.stack(spots), np.stack(jets)
    cells = int(sum(int(n) ** 3 for n in sizes))
    b = hydro.Batch(grids, limiter="minmod", stages=2, stream=stream)
    t0 = time.perf_counter()
    b.init_hotspots(spots, I.SPOT_SIGMA, I.E_BACKGROUND)
    b.set_jets(jets)
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    b.step(warmup)                 # the first call also autotunes the launch shapes
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(gpu) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        b.step(steps)              # CUDA graph of two steps, replayed
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # per-kernel durations: a short eager pass with CUDA events around each launch
    b.set_kernel_timing(True)
    b.kernel_timing()
    b.step(min(steps, 4))
    (sweep_ms, other_ms), (n_sweep, n_other) = b.kernel_timing()
    b.set_kernel_timing(False)
    status = b.event_status()
    value = nev * steps / 100.0 / (ms * 1e-3)
    hbm, src = peaks()
    bytes_per_sweep = 2 * 4 * 4 * cells
    avg = sweep_ms / max(n_sweep, 1)
    achieved = bytes_per_sweep / (avg * 1e-3) / 1e9
    fpc = flops_per_cell_sweep(2, 2, "minmod")
    flops = fpc * cells / (avg * 1e-3) / 1e12
    # per step: 5 sweeps + k_dt + k_jet (the CFL rate is fused into the last sweep)
    launches_per_step = (n_sweep + 2 * n_other) / max(n_other, 1)
    # end to end through the public API on the same handle (launch shapes
    # already tuned): a new batch from host hot-spot lists and jets, every
    # step's per-event conservation sums read back, final event status read
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.init_hotspots(spots, I.SPOT_SIGMA, I.E_BACKGROUND)
    b.set_jets(jets)
    for _ in range(steps):
        b.step(1)
        b.conservation_sums()
    b.event_status()
    torch.cuda.synchronize()
    e2e = nev * steps / 100.0 / (time.perf_counter() - t0)
    h2d = (spots.nbytes + jets.nbytes) / steps
    d2h = nev * 4 * 8 + nev * 4 / steps
    del b
    torch.cuda.empty_cache()
    out = {"metric": "events_per_s", "value": value, "unit": "events/s (100 steps each)",
           "events": nev, "steps": steps, "warmup": warmup, "ms_per_step": ms / steps,
           "cell_updates_per_s": cells * steps / (ms * 1e-3),
           "config": {"workload": f"{nev} events, grids uniform on 64^3..160^3, dx 0.1 fm, "
                                  "416 Gaussian hot spots + jet, FP32, minmod, 2 MUSTA stages, "
                                  "RK2+Hancock, Strang, outflow, CFL 0.4, CUDA graph of steps",
                      "cells": cells, "l2": "inputs larger than L2",
                      "steps_note": "a reduced number of the 100 steps of an event; events/s "
                                    "scales the measured steps to 100"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                        "frac": achieved / hbm, "traffic": BATCH_TRAFFIC_PER_CELL * cells,
                        "traffic_note": "scaled by cells from an ncu capture of 64 events",
                        "kernel": "k_sweep over all events (persistent grid)",
                        "algorithmic_bytes_per_launch": bytes_per_sweep, "avg_launch_ms": avg,
                        "peak_source": src},
           "roofline_alu": {"bound": "alu", "achieved": flops,
                            "peak": ALU_PEAK_TFLOPS["fp32"], "unit": "TFLOP/s",
                            "frac": flops / ALU_PEAK_TFLOPS["fp32"],
                            "algorithmic_flops_per_cell": fpc},
           "kernel_ms": {"sweeps": sweep_ms, "sweep_launches": n_sweep, "rate_dt_jet": other_ms,
                         "groups": n_other,
                         "kernel_timing": "separate eager pass of min(steps, 4) steps"},
           "gpu_launches": int(round(launches_per_step * steps)),
           "e2e": {"value": e2e, "unit": "events/s (100 steps each)",
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "path": "hydro_batch_init_hotspots + hydro_batch_set_jets from host arrays, "
                           "hydro_batch_step(1) and hydro_batch_conservation_sums per step, "
                           "hydro_batch_event_status"},
           "init_s": init_s, "events_nonfinite": int((status == 6).sum()),
           "events_repaired": int((status == 4).sum()),
           "clocks": clk.summary()}
    if not no_cpu:
        out["cpu_baseline"] = batch_cpu_baseline(cells / nev)
    return out


def run_batch(args):
    """512 events (grids uniform on 64^3..160^3, dx = 0.1 fm) of 416 Gaussian hot
    spots plus a jet, FP32, minmod, 2 MUSTA stages, RK2 + Hancock, Strang,
    outflow; one launch per sweep over all events, CUDA graph of the steps.
    Metric: events/s (events x steps / 100 per second)."""
    import torch
    from paper_1510_06340_b300 import build, dist as D, hydro
    from paper_1510_06340_b300 import inputs as I
    world, rank, local = D.world()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    if rank == 0:
        build.build(verbose=False)
    D.barrier()
    nev = args.events
    ids = D.rank_events(nev, rank)
    sizes = I.event_sizes(nev * world)[ids]
    grids, spots, jets = [], [], []
    for e, n in zip(ids, sizes):
        g = I.event_grid(int(n), 0.1)
        grids.append(hydro.make_grid(int(n), int(n), int(n), dx=0.1, x0=g["x0"], y0=g["y0"],
                                     z0=g["z0"], bc="outflow", prec="fp32", cfl=0.4))
        spots.append(I.hotspots(e))
        jets.append(I.jet(e))
    cells = int(sum(int(n) ** 3 for n in sizes))
    stream = torch.cuda.Stream()
    b = hydro.Batch(grids, limiter="minmod", stages=2, stream=stream)
    t0 = time.perf_counter()
    b.init_hotspots(np.stack(spots), I.SPOT_SIGMA, I.E_BACKGROUND)
    b.set_jets(np.stack(jets))
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    b.step(args.warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        D.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        b.step(args.steps)          # CUDA graph of two steps, replayed
        e1.record(stream)
        torch.cuda.synchronize()
        D.barrier()
    ms = D.max_over_ranks(e0.elapsed_time(e1), device="cuda")
    # per-kernel durations: a short eager pass with CUDA events around each launch
    b.set_kernel_timing(True)
    b.kernel_timing()
    b.step(min(args.steps, 4))
    (sweep_ms, other_ms), (n_sweep, n_other) = b.kernel_timing()
    b.set_kernel_timing(False)
    # per step: 5 sweeps + k_dt + k_jet (the CFL rate is fused into the last sweep)
    launches_per_step = (n_sweep + 2 * n_other) / max(n_other, 1)
    status = b.event_status()
    value = world * nev * args.steps / 100.0 / (ms * 1e-3)
    hbm, src = peaks()
    bytes_per_sweep = 2 * 4 * 4 * cells
    avg = sweep_ms / max(n_sweep, 1)
    achieved = bytes_per_sweep / (avg * 1e-3) / 1e9
    if rank == 0:
        line = {"metric": "events_per_s", "value": value, "unit": "events/s (100 steps each)",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"{nev} events per GPU, grids uniform on 64^3..160^3, "
                                       "dx 0.1 fm, 416 Gaussian hot spots + jet, FP32, minmod, "
                                       "2 MUSTA stages, RK2+Hancock, Strang, outflow, CFL 0.4",
                           "cells_per_gpu": cells, "parallelism": f"event shards x{world}",
                           "l2": "inputs larger than L2"},
                "cell_updates_per_s": world * cells * args.steps / (ms * 1e-3),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                             "frac": achieved / hbm, "traffic": None,
                             "kernel": "k_sweep over all events",
                             "algorithmic_bytes_per_launch": bytes_per_sweep,
                             "avg_launch_ms": avg, "peak_source": src},
                "kernel_ms": {"sweeps": sweep_ms, "sweep_launches": n_sweep,
                              "rate_dt_jet": other_ms, "groups": n_other},
                "gpu_launches": int(round(launches_per_step * args.steps)),
                "kernel_timing": "separate eager pass of min(steps, 4) steps",
                "init_s": init_s, "events_nonfinite": int((status == 6).sum()),
           "events_repaired": int((status == 4).sum()),
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    return 0


def run_learned(args):
    """Tabulated non-conformal EOS: 128 events on 128^3 hot-spot grids, FP32
    batch with cons->prim by Newton seeded by the trained MLP, against the
    same batch with the plain seeds and against the plain FP64 per-event path
    (one event at a time, FP64, v0 = 0).  Metric: events/s (100 steps each)."""
    import torch
    from paper_1510_06340_b300 import build, hydro
    from paper_1510_06340_b300 import inputs as I

    def rel_l1(a, b):
        a = np.asarray(a, dtype=np.float64)
        b = np.asarray(b, dtype=np.float64)
        fl = 1e-3 * np.abs(b[0]).sum()
        return [float(np.abs(a[q] - b[q]).sum() / max(np.abs(b[q]).sum(), fl)) for q in range(4)]
    from paper_1510_06340_b300 import learned
    torch.cuda.set_device(0)
    build.build(verbose=False)
    tab = I.eos_table()
    # the network is trained on cells of solver runs in its range (E above
    # where the EOS departs from p = e/3), labelled by the plain Newton solve
    t0 = time.perf_counter()
    U_train, emin = learned.harvest_states(tab, n=64, events=(0, 1), steps=4)
    X, Y, _ = learned.solver_pairs(tab, U_train)
    params, hist = learned.train_seed(X, Y, epochs=150)
    train_s = time.perf_counter() - t0
    loss = float(hist[-1])
    U_in, _ = learned.harvest_states(tab, n=64, events=(7,), steps=4)
    U_all, _ = learned.harvest_states(tab, n=64, events=(7,), steps=4, keep_all=True)
    iters_states = {"network_range": learned.seed_iterations(tab, params, U_in, "fp32")[0],
                    "all_cells": learned.seed_iterations(tab, params, U_all, "fp32")[0],
                    "states": f"cells of a 64^3 hot-spot event after 4 steps (event 7, not "
                              f"trained on); network range E > {emin:.3g}: {U_in.shape[1]} "
                              f"of {U_all.shape[1]} cells"}
    nev, n = args.events, 128
    g0 = I.event_grid(n, 0.1)
    spots = np.stack([I.hotspots(e) for e in range(nev)])
    stream = torch.cuda.Stream()

    def batch(seed, steps, prec="fp32", events=nev, counters=False):
        grids = [hydro.make_grid(n, n, n, dx=0.1, x0=g0["x0"], y0=g0["y0"], z0=g0["z0"],
                                 bc="outflow", prec=prec, cfl=0.4) for _ in range(events)]
        b = hydro.Batch(grids, hydro.make_eos(tab, seed=seed, mlp_params=params),
                        limiter="minmod", stages=2, stream=stream)
        b.init_hotspots(spots[:events], I.SPOT_SIGMA, I.E_BACKGROUND)
        b.step(args.warmup)
        torch.cuda.synchronize()
        if counters:
            b.enable_counters(True)
            b.step(1)
            c = b.counters()
            return None, c["newton_iters"] / max(c["newton_calls"], 1), b
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        return events * steps / 100.0 / (ms * 1e-3), None, b

    res = {}
    with Clocks(0) as clk:
        for seed in ("mlp", "zero", "conformal"):
            res[seed] = batch(seed, args.steps)[0]
    iters = {seed: batch(seed, 1, events=4, counters=True)[1] for seed in ("mlp", "zero", "conformal")}
    # plain FP64 per-event path: one event, v0 = 0, timed over 2 steps
    h = hydro.Hydro(hydro.make_grid(n, n, n, dx=0.1, x0=g0["x0"], y0=g0["y0"], z0=g0["z0"],
                                    bc="outflow", prec="fp64", cfl=0.4),
                    hydro.make_eos(tab, seed="zero"), limiter="minmod", stages=2, stream=stream)
    h.init_hotspots(spots[0], I.SPOT_SIGMA, I.E_BACKGROUND)
    h.step(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h.step(2)
    torch.cuda.synchronize()
    fp64_event_s = (time.perf_counter() - t0) / 2 * 100
    # error of the learned FP32 batch against the FP64 path after the same steps
    k = 4
    _, _, bl = batch("mlp", 0, events=1)
    bl.step(k)
    h2 = hydro.Hydro(hydro.make_grid(n, n, n, dx=0.1, x0=g0["x0"], y0=g0["y0"], z0=g0["z0"],
                                     bc="outflow", prec="fp64", cfl=0.4),
                     hydro.make_eos(tab, seed="zero"), limiter="minmod", stages=2, stream=stream)
    h2.init_hotspots(spots[0], I.SPOT_SIGMA, I.E_BACKGROUND)
    h2.step(args.warmup + k)
    err = rel_l1(bl.get_conserved(0), h2.get_conserved())
    line = {"metric": "events_per_s", "value": res["mlp"], "unit": "events/s (100 steps each)",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{nev} events on 128^3, tabulated EOS (4096 nodes), "
                                   "hot spots, FP32, minmod, 2 MUSTA stages, RK2+Hancock, Strang, "
                                   "Newton cons->prim seeded by the BF16 tensor-core MLP"},
            "events_per_s_by_seed": res,
            "newton_iterations_per_solve": iters,
            "newton_iterations_on_run_states_fp32": iters_states,
            "mlp_training": f"{U_train.shape[1]} cells of 2 hot-spot events after 4 steps, "
                            "E in the network range, targets from the plain FP64 Newton solve",
            "fp64_per_event_events_per_s": 1.0 / fp64_event_s,
            "learned_fp32_vs_fp64_rel_l1": err,
            "mlp_final_loss": loss, "mlp_train_s": train_s,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_table(args):
    """One 128^3 event (dx 0.1 fm) of 416 hot spots with flow |u| <= 0.5,
    outflow, the tabulated non-conformal EOS (4096 nodes), FP32, minmod,
    2 MUSTA stages, RK2 + Hancock, Strang; cons->prim by Newton from the
    seed --seed (zero or conformal).  Metric: cell-updates/s; with the
    Newton iterations per solve from a counting step."""
    import torch
    from paper_1510_06340_b300 import build, hydro
    from paper_1510_06340_b300 import inputs as I
    torch.cuda.set_device(0)
    build.build(verbose=False)
    n = 128
    g = I.event_grid(n, 0.1)
    spots = I.hotspots(0, flow_max=0.5)
    tab = I.eos_table()
    stream = torch.cuda.Stream()
    grid = hydro.make_grid(n, n, n, dx=0.1, x0=g["x0"], y0=g["y0"], z0=g["z0"], bc="outflow",
                           prec="fp32", cfl=0.4)
    h = hydro.Hydro(grid, hydro.make_eos(tab, seed=args.seed), limiter="minmod", stages=2,
                    stream=stream)
    h.init_hotspots(spots, I.SPOT_SIGMA, I.E_BACKGROUND)
    if args.launch:
        th, sg = (int(x) for x in args.launch.split(","))
        for ax in range(3):
            h.force_launch(ax, th, sg)
    h.step(args.warmup)
    torch.cuda.synchronize()
    h.set_kernel_timing(True)
    h.kernel_timing()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        h.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    (sweep_ms, other_ms), (n_sweep, n_other) = h.kernel_timing()
    h.set_kernel_timing(False)
    shapes = [h.get_launch(ax) for ax in range(3)]
    h.enable_counters(True)
    h.step(1)
    c = h.counters()
    cells = n ** 3
    hbm, src = peaks()
    avg = sweep_ms / max(n_sweep, 1)
    bps = 2 * 4 * 4 * cells
    line = {"metric": "cell_updates_per_s", "value": cells * args.steps / (ms * 1e-3),
            "unit": "cell-updates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "128^3 hot spots with flow |u| <= 0.5, outflow, tabulated EOS "
                                   f"(4096 nodes), Newton seed {args.seed}, FP32, minmod, "
                                   "2 MUSTA stages, RK2+Hancock, Strang", "cells": cells,
                       "launch_threads_segments_xyz": shapes},
            "roofline": {"bound": "hbm", "achieved": bps / (avg * 1e-3) / 1e9, "peak": hbm,
                         "unit": "GB/s", "frac": bps / (avg * 1e-3) / 1e9 / hbm,
                         "avg_launch_ms": avg, "peak_source": src},
            "newton_iterations_per_solve": c["newton_iters"] / max(c["newton_calls"], 1),
            "newton_solves_per_cell_sweep": c["newton_calls"] / (5 * cells),
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_mixed(args):
    """Single 512^3 event (dx 0.1 fm) of hot spots with random flow |u| <= 0.95,
    outflow, mixed precision (FP32 state and fluxes, FP64 cons->prim for
    |v| > 0.99, FP64 sums), minmod, 2 MUSTA stages, RK2 + Hancock, Strang.
    Metric: cell-updates/s.  Per-field relative L1 error against an FP64 run
    from the same initial state after a few steps."""
    import torch
    from paper_1510_06340_b300 import build, hydro
    from paper_1510_06340_b300 import inputs as I
    torch.cuda.set_device(0)
    build.build(verbose=False)
    n = 512
    g = I.event_grid(n, 0.1)
    spots = I.hotspots(0, flow_max=0.95)
    stream = torch.cuda.Stream()
    mk = lambda prec: hydro.make_grid(n, n, n, dx=0.1, x0=g["x0"], y0=g["y0"], z0=g["z0"],
                                      bc="outflow", prec=prec, cfl=0.4)
    h = hydro.Hydro(mk("mixed"), limiter="minmod", stages=2, stream=stream)
    h.init_hotspots(spots, I.SPOT_SIGMA, I.E_BACKGROUND)
    U0 = h.get_conserved()
    h.step(args.warmup)
    torch.cuda.synchronize()
    h.set_kernel_timing(True)
    h.kernel_timing()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        h.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    (sweep_ms, other_ms), (n_sweep, n_other) = h.kernel_timing()
    h.set_kernel_timing(False)
    sums = h.conservation_sums()
    # error against FP64 from the same initial state
    k = 3
    hm = hydro.Hydro(mk("mixed"), limiter="minmod", stages=2, stream=stream)
    hm.set_conserved(U0)
    hm.enable_counters(True)
    hm.step(k)
    redo = hm.counters()["f64_redo"]
    Um = hm.get_conserved().astype(np.float64)
    del hm
    hd = hydro.Hydro(mk("fp64"), limiter="minmod", stages=2, stream=stream)
    hd.set_conserved(U0.astype(np.float64))
    hd.step(k)
    Ud = hd.get_conserved()
    del hd
    fl = 1e-3 * np.abs(Ud[0]).sum()
    err = [float(np.abs(Um[q] - Ud[q]).sum() / max(np.abs(Ud[q]).sum(), fl)) for q in range(4)]
    hbm, src = peaks()
    cells = n ** 3
    avg = sweep_ms / max(n_sweep, 1)
    bps = 2 * 4 * 4 * cells
    line = {"metric": "cell_updates_per_s", "value": cells * args.steps / (ms * 1e-3),
            "unit": "cell-updates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "512^3 hot spots with random flow |u| <= 0.95, outflow, "
                                   "mixed precision, minmod, 2 MUSTA stages, RK2+Hancock, Strang",
                       "cells": cells},
            "roofline": {"bound": "hbm", "achieved": bps / (avg * 1e-3) / 1e9, "peak": hbm,
                         "unit": "GB/s", "frac": bps / (avg * 1e-3) / 1e9 / hbm,
                         "avg_launch_ms": avg, "peak_source": src},
            "rel_l1_vs_fp64_after_3_steps": dict(zip(("E", "Mx", "My", "Mz"), err)),
            "fp64_redo_cons2prim_in_3_steps": redo,
            "fp64_sums": list(sums), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="blast256_fp32",
                    choices=sorted(WORKLOADS) + ["batch512", "learned128", "mixed512",
                                                 "table128"])
    ap.add_argument("--seed", default="conformal", choices=["zero", "conformal"],
                    help="Newton seed of the table128 workload")
    ap.add_argument("--events", type=int, default=512, help="events per GPU (batch512)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--launch", default="", help="force 'threads,segments' for every axis")
    ap.add_argument("--limiter", default="minmod", choices=["minmod", "mc", "superbee"],
                    help="slope limiter of the blast workloads")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer e2e pass")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the nested event-batch measurement of the default line")
    ap.add_argument("--batch-steps", type=int, default=10,
                    help="timed steps of the nested event-batch measurement")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch512":
        return run_batch(args)
    if args.workload == "table128":
        return run_table(args)
    if args.workload == "mixed512":
        return run_mixed(args)
    if args.workload == "learned128":
        if args.events == 512:
            args.events = 128
        return run_learned(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
