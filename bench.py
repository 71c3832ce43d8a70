#!/usr/bin/env python
"""Benchmark: zone-updates/s of the RK2 finite-volume step on the oblique
3D Riemann problem at 256^3 (Sod states split by the plane normal to
(1,1,1) through the cube centre, gamma 1.4, outflow, CFL 0.4).

One step = ComputeTimeStep (CFL min-reduction, one 32-byte device-to-host
read) + the full RK2 step (one fused kernel and a ghost fill per substep);
one zone-update = one interior cell advanced by one step.  The timed region
starts from the initial state already resident in HBM and covers K steps of
the workload.  Prints one JSON line (rank 0).

  python bench.py [--steps K] [--warmup W] [--precision fp64|fp64_fma]
  python bench.py --impl reference      # the CPU oracle on a bounded sample
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "zone-updates/s per RK2 step at 256^3 (FP64 vs FP32) and % of HBM roofline"
CFL = 0.4
N = 256
# FP64 issue rate measured on this GPU: 2 DFMA lane-operations per SM per
# clock; 2 flops per DFMA.
DFMA_PER_SM_CLK = 2.0
# Algorithmic FP64 flops of the method (divide and square root count one
# each), from the operation counts of the definition:
#   per face: two sides x (cons 11 + sound speed 3 + flux 6) + wave bounds 4
#             + HLL denominator and product 3 + 5 components x 7 = 82
#   per cell and axis: differences 5 + limited slopes 5x4 + face states 5x4
#             + one face 82 = 127
#   divergence: x 2, y 3, z 3 per component; z adds dt* (1) and the RK
#             combine (stage 1: 1 add, stage 2: 2 adds + 1 multiply).
FLOPS_SWEEP = {"sweep_x": 127 + 5 * 2, "sweep_y": 127 + 5 * 3,
               "sweep_z": 127 + 5 * 3 + 5 * 1 + 5 * 2}     # z: stage average of RK
# Of these, 127 per cell belong to its face (differences, slopes, face states,
# HLL flux); a face whose flux is reused (a run of equal cells) skips them,
# so the FP64 flops executed are 127 per evaluated face plus the rest per cell.
FLOPS_FACE = 127
FLOPS_PRIM = 12          # per cell converted to primitives
FLOPS_DT = 23            # per interior cell
# The fused substep per cell and launch, besides its faces: the primitives of
# the cell and of its share of the tile's two-cell halo (32 x 8 tiles: 1.69
# conversions per cell), the divergence (40) and the RK combine (average 10).
FLOPS_FUSED_CELL = round(FLOPS_PRIM * (36 * 12) / (32 * 8)) + 40 + 10
# Algorithmic HBM bytes per zone-update for a fused step with in-place
# stage 2: stage 1 reads U^n, writes U^1 (80 B); stage 2 reads U^1, U^n and
# writes U^{n+1} (120 B).
BYTES_PER_ZONE_UPDATE = 200
# The float-float form (FV_PREC_FP64_FF) works on the FP32 pipe: its
# algorithmic FP32 operations (each FP32 add, multiply, fused multiply-add,
# reciprocal or reciprocal square root counted once; comparisons, sign
# tests and the FP64 <-> float-float conversions not counted), from the
# operation counts of its formulas (TwoSum 6, Fast2Sum 3, TwoProd 2;
# float-float add 11, multiply 7, reciprocal 11, inverse square root 17):
#   per face: the two face states 110; per side kinetic and total energy and
#     sound speed 122 (x2); wave bounds, 1 / (a+ + a-), a+ a-, normal mass
#     fluxes 87; the five HLL components 61 + 289 + 97 -> 888;
#   per cell and axis (one per face): the two one-sided differences of the
#     five primitives 110 and the half monotonised-central slopes 95 (theta
#     = 2, the default: theta d is exact doubling) -> 205;
#   per cell and launch: the float-float divergence 380.
FF_OPS_FACE = 888 + 205
FF_OPS_CELL = 380
# DRAM bytes (read + write) per launch of the fused kernels on the 256^3
# oblique problem (mean of stage 1 and 2, second step) from ncu captures
# (`--metrics dram__bytes_read.sum,dram__bytes_write.sum` of
# `python -m paper_1812_07977_gb300.run_case PRECISION 256 oblique 3`) of the
# kernels as they are now; None where the kernel has changed since.
FUSED_TRAFFIC = {
    "fp32_bulk": (1.736e9, "ncu capture 2026-12-04 of k_stage32<., 16, 8, 4, 1> (equal-state "
                           "skip): 1.418 GB (stage 1) and 2.054 GB (stage 2)"),
    "fp64_ff": (2.011e9, "ncu capture 2026-12-04 of k_stageff<., MC, 16, 16, 2, plane skip> "
                         "with one z chunk per column (the early steps' launch shape): 1.659 GB "
                         "(stage 1) and 2.364 GB (stage 2); with 37-plane chunks (later steps) "
                         "1.611 and 2.307 GB"),
    "fp64_fma": None,
    "fp64": None,
}


def fp64_probe():
    """Live issue rates from the library's probe (DFMA, DADD, DMUL, divide,
    square root, FFMA per second) on the current GPU, or None."""
    exe = os.path.join(ROOT, "paper_1812_07977_gb300", "_build", "fp64_probe")
    try:
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        return json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except Exception:
        return None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        self.proc.wait()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return summarize_clocks(lines)


def summarize_clocks(lines):
    """Median SM clock under load (samples above half the maximum), the
    maximum clock and the throttle reasons seen Active, from nvidia-smi's
    `ClockSampler.FIELDS` rows (csv, no header, no units)."""
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = set()
    sm, smax = [], None
    for line in lines:
        r = [p.strip() for p in line.split(",")]
        if len(r) != 8:
            continue
        try:
            clock, top = float(r[0]), float(r[1])
        except ValueError:
            continue
        sm.append(clock)
        smax = top
        for k, name in enumerate(names):
            if r[4 + k].lower() == "active":
                reasons.add(name)
    loaded = [s for s in sm if smax and s > 0.5 * smax] or sm
    return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": smax,
            "samples": len(sm), "reasons": sorted(reasons)}


def _dist():
    """(rank, world, local_rank) from torchrun's environment; init the group."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = os.environ.get("FV_BENCH_BACKEND", "nccl")
        dist.init_process_group(backend=backend)
    return rank, world, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x: float, world: int, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _oracle_slab(args):
    """One process of the oracle timing: the oracle as it stands on planes
    k0 .. k0+S-1 of the 256^3 oblique problem (its own slab, outflow at the
    cut), `warmup` untimed RK2 steps, then `steps` timed ones (each with
    ComputeTimeStep), or, with steps = 0, as many as fit in `seconds` (at most
    50).  Returns (cells, timed steps, seconds)."""
    k0, S, warmup, steps, seconds = args
    import oracle
    from paper_1812_07977_gb300 import problems

    U = problems.riemann_oblique(N, N, N, planes=(k0, k0 + S))
    m = oracle.mesh(N, N, S, lz=S / N)
    Ug = oracle.ghosted_from_interior(m, U)
    for _ in range(warmup):
        dt, _, _ = oracle.reduce_dt(m, Ug, CFL)
        oracle.step(m, Ug, dt)
    n, t0 = 0, time.perf_counter()
    while True:
        dt, _, _ = oracle.reduce_dt(m, Ug, CFL)
        oracle.step(m, Ug, dt)
        n += 1
        el = time.perf_counter() - t0
        if (steps and n >= steps) or (not steps and (el >= seconds or n >= 50)):
            break
    return N * N * S, n, el


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_on_cores(procs, S, warmup=0, steps=0, seconds=10.0):
    """The oracle on `procs` host cores: one process per core (started with
    `spawn`, so a process that has used the GPU can start them), each
    advancing its own S-plane slab of the workload (slabs side by side
    through the centre).  Returns (zone-updates/s summed over the
    processes, the longest process's seconds, its timed steps)."""
    import multiprocessing as mp

    import oracle
    oracle.build()                      # once, before the processes load it
    S = max(1, min(S, N // procs)) if procs > 1 else S
    first = max(0, N // 2 - procs * S // 2)
    starts = [min(first + i * S, N - S) for i in range(procs)]
    if procs == 1:
        res = [_oracle_slab((starts[0], S, warmup, steps, seconds))]
    else:
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_oracle_slab, [(k0, S, warmup, steps, seconds) for k0 in starts])
    rate = sum(c * n / el for c, n, el in res)
    slow = max(res, key=lambda r: r[2])
    return rate, slow[2], slow[1], S


def cpu_baseline(seconds_target: float = 10.0):
    """The oracle as it stands on bounded samples of the workload: one
    process on one core (a 256 x 256 x 8 slab through the centre), and one
    process per host core, each on its own 256 x 256 x S slab (the slabs
    side by side through the centre), about `seconds_target` of steps each."""
    one, el1, n1, _ = oracle_on_cores(1, 8, seconds=seconds_target)
    cores = host_cores()
    allc, el, n, S = oracle_on_cores(cores, 8, seconds=seconds_target)
    return {"value": allc, "unit": "zone-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes (one per host core), each running RK2 steps (with "
                      f"ComputeTimeStep) of its own 256x256x{S} slab of the 256^3 oblique "
                      f"problem for ~{seconds_target:.0f} s ({n} steps, {el:.1f} s in the "
                      f"slowest); value = sum of the processes' rates",
            "single_core": {"value": one, "cores": 1,
                            "sample": f"{n1} RK2 steps of a 256x256x8 slab through the "
                                      f"centre, one process, {el1:.1f} s"}}


def run_reference(args):
    """--impl reference: the CPU oracle on the arm's workload on every host
    core, each step a bounded sample (one 256 x 256 x 4 slab of the same mesh
    per core, slabs side by side through the centre)."""
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    cores = host_cores()
    rate, el, steps, S = oracle_on_cores(cores, 4, warmup=args.warmup, steps=args.steps)
    sample = (f"each step: one RK2 step of a 256x256x{S} slab of the 256^3 oblique problem "
              f"in each of {cores} processes (one per host core); value = sum of the "
              f"processes' rates")
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "zone-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "oblique Riemann 256^3 (sampled slabs)", "sample": sample},
            "cpu_baseline": {"value": rate, "unit": "zone-updates/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": "zone-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _timed_run(m, U0_dev, steps, warmup, world, dev, rank, sample_clocks):
    """Warm up, restart the workload from U0, time `steps` steps with CUDA
    events on the current stream; returns (ms_max, ms_local, profile, clocks)."""
    import torch

    def step():
        m.step(m.reduce_dt(CFL))

    m.set_state(U0_dev)
    for _ in range(warmup):
        step()
    m.set_state(U0_dev)
    torch.cuda.synchronize()
    m.profile(True)
    m.read_profile()
    sampler = ClockSampler(dev.index)
    if rank == 0 and sample_clocks:
        sampler.start()
    _barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(steps):
        step()
    ev1.record()
    torch.cuda.synchronize()
    _barrier(world)
    clocks = sampler.stop() if (rank == 0 and sample_clocks) else None
    ms = ev0.elapsed_time(ev1)
    prof = m.read_profile()
    m.profile(False)
    faces = m.face_counts()          # evaluated, defined over the timed steps
    return _max_over_ranks(ms, world, dev), ms, prof, clocks, faces


def run_batched(args, world, dev, rank):
    """The batched workload: 96 meshes, axis lengths uniform in
    {16, 24, ..., 128}, each a random Riemann problem (FP32-bulk), one
    persistent launch per substep, the whole step replayed from a CUDA graph,
    launch configuration from the library's autotuner."""
    import torch

    from paper_1812_07977_gb300 import problems
    from paper_1812_07977_gb300.fv import Batch

    spec = problems.batched_riemann(seed=12345, count=96)
    stream = torch.cuda.Stream()          # capturable; events are recorded on it
    b = Batch([s["shape"] for s in spec], stream=stream)
    for m, s in enumerate(spec):
        b.set_state(m, torch.from_numpy(s["U0"]).to(dev))
    kc, occ, tile_y, tune_ms = b.autotune(CFL)
    per_class = {f"class{c} ({('nx<=24', 'nx<=64', 'nx>64')[c]})": b.class_tuning(c)
                 for c in range(3)}
    for _ in range(args.warmup):
        b.step(CFL, use_graph=True)
    for m, s in enumerate(spec):
        b.set_state(m, torch.from_numpy(s["U0"]).to(dev))
    nmesh, cells, items = b.info()
    torch.cuda.synchronize()
    _barrier(world)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.batch_steps):
        b.step(CFL, use_graph=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    el = _max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world, dev)
    bad, fb = b.counters()
    b.close()
    return {"value": world * cells * args.batch_steps / el, "unit": "zone-updates/s",
            "ms_per_step": 1e3 * el / args.batch_steps, "steps": args.batch_steps,
            "meshes": nmesh, "cells": cells, "work_items": items,
            "autotuned": {"per_class": per_class, "ms_per_step": tune_ms},
            "timing": "CUDA events on the batch's stream around the graph launches",
            "nonphysical": bad}


def run_learned(args):
    """The learned-correction workload: periodic shear layers (rho 1 and 2,
    vx +-0.5, vy = A sin(4 pi x), p = 2.5, gamma 1.4), fine 256^3 FP64 runs
    block-averaged 4x onto a 64^3 coarse mesh; training by the library's
    kernels (with input-noise injection); evaluation on a held-out amplitude
    against the averaged fine run, with and without the correction."""
    from paper_1812_07977_gb300 import learned
    r = learned.run(fine_n=args.learned_fine, factor=4, train_amps=(0.01, 0.04, 0.07, 0.1),
                    val_amp=0.085, test_amp=0.055, samples=args.learned_samples, every=2,
                    epochs=args.learned_epochs, lr=1e-3, eval_steps=args.learned_eval_steps,
                    val_steps=args.learned_eval_steps, noise=args.learned_noise)
    out = {k: v for k, v in r.items() if not isinstance(v, list)}
    out["l1_rho_plain_mean"] = float(np.mean(r["l1_rho_plain"]))
    out["l1_rho_learned_mean"] = float(np.mean(r["l1_rho_learned"]))
    out["l1_rho_plain_final"] = r["l1_rho_plain"][-1]
    out["l1_rho_learned_final"] = r["l1_rho_learned"][-1]
    out["gain"] = out["l1_rho_plain_mean"] / max(out["l1_rho_learned_mean"], 1e-300)
    return out


def run_shear(args, dev):
    """512^3 periodic shear layer (rho 2/1, vx +-0.5, p 2.5, gamma 5/3, an
    8-mode seeded perturbation of amplitude 0.01 on vy and vz): the FP32-bulk
    fused step replayed from a CUDA graph (a batch of one mesh) versus the
    FP64-class step of --precision (held to the FP64 oracle), `shear_steps`
    steps each with its own CFL time steps, with the mass and energy drift of
    each."""
    import torch

    from paper_1812_07977_gb300 import problems
    from paper_1812_07977_gb300.fv import Batch, Mesh
    n, K, g53 = args.shear_n, args.shear_steps, 5.0 / 3.0
    U0 = problems.shear_layer_device(n, 0.01, gamma=g53, modes=8, seed=2024, device=dev)
    m64 = Mesh(n, n, n, gamma=g53, bc=("periodic",) * 3, precision=args.precision)
    m64.set_state(U0)
    s0 = m64.conserved_sums()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    dts = []
    ev[0].record()
    for _ in range(K):
        dt = m64.reduce_dt(CFL)
        dts.append(dt)
        m64.step(dt)
    ev[1].record()
    torch.cuda.synchronize()
    ms64 = ev[0].elapsed_time(ev[1]) / K
    s64 = m64.conserved_sums()
    rho64 = m64.get_state()[0].clone()
    stream = torch.cuda.Stream()
    b = Batch([(n, n, n)], gamma=g53, bc=("periodic",) * 3, stream=stream)
    b.set_state(0, U0)
    ev[2].record(stream)
    for _ in range(K):                 # its own CFL dt each step, from a graph
        b.step(CFL, use_graph=True)
    ev[3].record(stream)
    torch.cuda.synchronize()
    ms32 = ev[2].elapsed_time(ev[3]) / K
    U32 = b.get_state(0)
    b.close()
    m64.set_state(U32)                 # the library's pairwise sums of the FP32 run
    s32 = m64.conserved_sums()
    drho = float((U32[0] - rho64).abs().mean() / rho64.abs().mean())
    m64.close()
    scale = [float(v) for v in U0.abs().reshape(5, -1).sum(1) / U0[0].numel()]
    return {"cells": n ** 3, "steps": K,
            args.precision: {"ms_per_step": ms64, "value": n ** 3 / (ms64 / 1e3),
                     "mass_drift": abs(s64[0] - s0[0]) / scale[0],
                     "energy_drift": abs(s64[4] - s0[4]) / scale[4]},
            "fp32_graph": {"ms_per_step": ms32, "value": n ** 3 / (ms32 / 1e3),
                           "mass_drift": abs(s32[0] - s0[0]) / scale[0],
                           "energy_drift": abs(s32[4] - s0[4]) / scale[4]},
            "rho_l1_rel_fp32_vs_" + args.precision: drho,
            "note": "drifts relative to the mean |U| per cell; the FP32 run takes its own "
                    "CFL steps, so the two end times agree to the dt difference"}


def _fused_roofline(prof, faces, zones, bytes_per_launch_cell, peak_tflops, hbm, flops,
                    per_face=FLOPS_FACE, per_cell=FLOPS_FUSED_CELL):
    """The fused substep kernel's figures: the operations executed per launch
    (per_face per evaluated face + per_cell per cell: FP64 flops for the FP64
    kernels, FP32 operations for the float-float one) against the peak of
    that pipe, and its algorithmic HBM bytes against the copy bandwidth."""
    ms, launches = prof["fused"]
    launches = max(launches, 1)
    evaluated, defined = faces
    sec = ms / 1e3
    out = {"kernel_ms": ms, "launches": launches, "avg_launch_ms": ms / launches,
           "faces_evaluated": evaluated, "faces_defined": defined,
           "faces_evaluated_fraction": evaluated / max(defined, 1)}
    b = bytes_per_launch_cell * zones
    out["hbm"] = {"achieved": b * launches / sec / 1e9 if sec > 0 else None, "peak": hbm,
                  "unit": "GB/s", "bytes_per_launch": b,
                  "frac": b * launches / sec / 1e9 / hbm if sec > 0 else None}
    if flops:
        executed = evaluated * per_face + per_cell * zones * launches
        method = defined * per_face + per_cell * zones * launches
        out["alu"] = {"achieved": executed / sec / 1e12 if sec > 0 else None,
                      "peak": peak_tflops, "unit": "TFLOP/s",
                      "frac": executed / sec / 1e12 / peak_tflops if sec > 0 else None,
                      "flops_per_launch": executed / launches,
                      "method_flops_per_launch": method / launches,
                      "effective_tflops": method / sec / 1e12 if sec > 0 else None}
    return out


def run_ours(args):
    import numpy as np
    import torch

    from paper_1812_07977_gb300 import problems
    from paper_1812_07977_gb300.fv import Mesh

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    probe = fp64_probe() if rank == 0 else None
    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    n = args.n
    zones = n ** 3
    U0 = problems.riemann_oblique(n, n, n)
    U0_dev = torch.from_numpy(U0).to(dev)
    m = Mesh(n, n, n, precision=args.precision)
    ms_max, ms, prof, clocks, faces = _timed_run(m, U0_dev, args.steps, args.warmup, world, dev,
                                                 rank, True)
    value = world * zones * args.steps / (ms_max / 1e3)

    def step():
        m.step(m.reduce_dt(CFL))

    # end to end through the public API with host buffers: each step copies
    # the state in from pinned host memory and the result back out
    host = torch.from_numpy(U0.copy()).pin_memory()
    m.set_state(host)
    step()
    m.get_state(host)
    host.copy_(torch.from_numpy(U0))
    _barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        m.set_state(host)
        step()
        m.get_state(host)
    torch.cuda.synchronize()
    e2e_s = _max_over_ranks(time.perf_counter() - t0, world, dev)
    state_bytes = 5 * zones * 8
    e2e = {"value": world * zones * args.e2e_steps / e2e_s, "unit": "zone-updates/s",
           "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes + 32,
           "steps": args.e2e_steps}
    m.close()

    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    derived_peak = DFMA_PER_SM_CLK * 2.0 * sms * sm_max * 1e6 / 1e12     # TFLOP/s
    if probe and probe.get("dfma_per_s"):
        fp64_peak = 2.0 * probe["dfma_per_s"] / 1e12
        peak_source = ("FP64 peak measured live by paper_1812_07977_gb300/_build/fp64_probe "
                       "(DFMA rate x 2 flops), of measured")
    else:
        fp64_peak = derived_peak
        peak_source = (f"FP64 issue rate 2 DFMA/SM/clk x {sms} SMs x {sm_max:.0f} MHz "
                       "(MEASURED_PEAKS sm_max_mhz)")

    # the float-float kernel's pipe: FP32 lane operations per second, measured
    # live (FFMA rate of the probe) or 128 per SM and clock
    derived_fp32 = 128.0 * sms * sm_max * 1e6 / 1e12
    if probe and probe.get("ffma_per_s"):
        fp32_peak = probe["ffma_per_s"] / 1e12
        fp32_source = ("FP32 operation rate measured live by paper_1812_07977_gb300/_build/"
                       "fp64_probe (FFMA lane operations per second), of measured")
    else:
        fp32_peak = derived_fp32
        fp32_source = f"128 FP32 lanes per SM and clock x {sms} SMs x {sm_max:.0f} MHz"

    def variant(prec, U0v, nsteps, bc=("outflow",) * 3):
        U0v_dev = torch.from_numpy(U0v).to(dev) if isinstance(U0v, np.ndarray) else U0v
        fused = prec.endswith("_fused")
        mv = Mesh(n, n, n, precision=prec[:-len("_fused")] if fused else prec, bc=bc)
        if fused:
            mv.set_tuning("fp64_fused", 1)
        vms_max, _, vprof, _, vfaces = _timed_run(mv, U0v_dev, nsteps, args.warmup, world, dev,
                                                  rank, False)
        mv.close()
        vval = world * zones * nsteps / (vms_max / 1e3)
        out = {"value": vval, "unit": "zone-updates/s", "ms_per_step": vms_max / nsteps,
               "steps": nsteps,
               "kernel_ms_per_step": {c: v[0] / nsteps for c, v in vprof.items()},
               "faces_evaluated_fraction": vfaces[0] / max(vfaces[1], 1),
               "hbm_roofline_whole_step": {
                   "achieved": BYTES_PER_ZONE_UPDATE * vval / 1e9, "peak": hbm, "unit": "GB/s",
                   "frac": BYTES_PER_ZONE_UPDATE * vval / 1e9 / hbm}}
        if vprof["fused"][1] > 0:
            if prec == "fp64_ff":
                out["fused_kernel"] = _fused_roofline(vprof, vfaces, zones, 100, fp32_peak, hbm,
                                                      True, FF_OPS_FACE, FF_OPS_CELL)
            else:
                out["fused_kernel"] = _fused_roofline(vprof, vfaces, zones, 100, fp64_peak, hbm,
                                                      not prec.startswith("fp32"))
            cap = FUSED_TRAFFIC.get(prec)
            if cap and U0v is U0 and n == N:
                out["fused_kernel"]["hbm"]["traffic"] = cap[0]
                out["fused_kernel"]["hbm"]["traffic_note"] = cap[1]
        return out

    # the other arithmetic variants on the same workload, fewer steps each,
    # and every variant on a state with no equal neighbours (a seeded smooth
    # periodic 256^3 state: every face evaluated, nothing reused)
    variants = {}
    for prec in args.variants:
        if prec != args.precision:
            variants[prec] = variant(prec, U0, args.variant_steps)
    if args.noreuse_steps > 0:
        smooth = problems.random_smooth_periodic(n, n, n, seed=12345)
        for prec in [args.precision] + [p for p in args.variants if p != args.precision]:
            variants[prec + "_no_reuse"] = variant(prec, smooth, args.noreuse_steps,
                                                   bc=("periodic",) * 3)
            variants[prec + "_no_reuse"]["workload"] = (
                "seeded smooth periodic 256^3 state (3 random Fourier modes per field, rho and "
                "p within 20% of 1, |v| <= 0.5): no two neighbouring cells equal")
        del smooth

    if args.batch_steps > 0:
        variants["batched_fp32"] = run_batched(args, world, dev, rank)
    if args.learned_epochs > 0 and rank == 0:
        variants["learned_correction"] = run_learned(args)
    if args.shear_steps > 0 and rank == 0:
        variants["shear_layer_512"] = run_shear(args, dev)

    if rank != 0:
        return 0

    hbm_achieved = BYTES_PER_ZONE_UPDATE * zones * args.steps / (ms / 1e3) / 1e9
    launches = sum(v[1] for v in prof.values())
    ff = args.precision == "fp64_ff"
    if ff:
        fused = _fused_roofline(prof, faces, zones, 100, fp32_peak, hbm, True, FF_OPS_FACE,
                                FF_OPS_CELL)
        kernel, peak, src, dpeak = ("k_stageff (fused substep, float-float faces)", fp32_peak,
                                    fp32_source, derived_fp32)
        ops = (f"FP32 operations of the float-float arithmetic: {FF_OPS_FACE} per evaluated "
               f"face + {FF_OPS_CELL} per cell and launch (each add, multiply or FMA once)")
    else:
        fused = _fused_roofline(prof, faces, zones, 100, fp64_peak, hbm, True)
        kernel, peak, src, dpeak = ("k_stage64 (fused FP64 substep)", fp64_peak, peak_source,
                                    derived_peak)
        ops = (f"FP64 flops executed: {FLOPS_FACE} per evaluated face + {FLOPS_FUSED_CELL} "
               f"per cell and launch")
    alu = fused["alu"]
    cap = FUSED_TRAFFIC.get(args.precision) if n == N else None
    traffic = args.traffic if args.traffic else (cap[0] if cap else None)
    roofline = {"bound": "alu", "kernel": kernel,
                "achieved": alu["achieved"], "peak": peak, "unit": "TFLOP/s",
                "frac": alu["frac"], "traffic": traffic,
                "traffic_note": (cap[1] if cap and not args.traffic else
                                 "DRAM bytes per launch from an ncu capture of this kernel "
                                 "(null: no capture of the current kernel)"),
                "peak_source": src, "derived_peak": dpeak,
                "avg_launch_ms": fused["avg_launch_ms"],
                "flops": ops,
                "flops_per_launch": alu["flops_per_launch"],
                "method_flops_per_launch": alu["method_flops_per_launch"],
                "effective_tflops": alu["effective_tflops"],
                "faces_evaluated": fused["faces_evaluated"],
                "faces_defined": fused["faces_defined"],
                "faces_evaluated_fraction": fused["faces_evaluated_fraction"],
                "hbm_view": fused["hbm"]}
    line = {
        "metric": METRIC, "value": value, "unit": "zone-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 state; float-float (2 x f32) face arithmetic" if ff else "f64",
        "data": "synthetic",
        "config": {"workload": "oblique Riemann problem 256^3 (Sod states, plane normal "
                               "(1,1,1), gamma 1.4, outflow, CFL 0.4), steps 1..K",
                   "precision": args.precision, "cells": zones,
                   "l2": "inputs larger than L2 (0.70 GB per ghosted state, 1.4 GB resident)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roofline,
        "hbm_roofline": {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm, "unit": "GB/s",
                         "frac": hbm_achieved / hbm,
                         "bytes_per_zone_update": BYTES_PER_ZONE_UPDATE,
                         "note": "whole step vs the algorithmic minimum traffic, of measured"},
        "kernel_ms_per_step": {c: v[0] / args.steps for c, v in prof.items()},
        "variants": variants,
        # the same precision with every face evaluated (nothing to reuse): the
        # kernels' rate without the workload's uniform regions
        "every_face_evaluated": ({k: variants[args.precision + "_no_reuse"].get(k)
                                  for k in ("value", "unit", "ms_per_step", "steps",
                                            "faces_evaluated_fraction", "workload")}
                                 if args.precision + "_no_reuse" in variants else None),
        "gpu_launches": launches,
        "fp64_probe": probe,
        "e2e": e2e,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64_ff", choices=["fp64", "fp64_fma", "fp64_ff"],
                    help="FP64 arithmetic of the headline line (fp32_bulk is reported as a "
                         "variant)")
    ap.add_argument("--variants", nargs="*",
                    default=["fp64", "fp64_fma", "fp64_fused", "fp32_bulk"],
                    help="other precisions timed beside the headline one")
    ap.add_argument("--variant-steps", type=int, default=50)
    ap.add_argument("--noreuse-steps", type=int, default=10,
                    help="steps of each precision on a 256^3 state without equal neighbours "
                         "(0: skip)")
    ap.add_argument("--batch-steps", type=int, default=50,
                    help="steps of the 96-mesh batched workload (0: skip)")
    ap.add_argument("--learned-epochs", type=int, default=16,
                    help="training epochs of the learned correction (0: skip)")
    ap.add_argument("--learned-fine", type=int, default=256)
    ap.add_argument("--learned-samples", type=int, default=16)
    ap.add_argument("--learned-eval-steps", type=int, default=32)
    ap.add_argument("--learned-noise", type=float, default=0.5,
                    help="training-input noise, in units of each field's standard deviation")
    ap.add_argument("--shear-n", type=int, default=512)
    ap.add_argument("--shear-steps", type=int, default=100,
                    help="steps of the 512^3 shear-layer FP32-graph vs FP64 comparison (0: skip)")
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per fused-kernel launch from an ncu capture of it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
