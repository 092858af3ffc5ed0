"""Benchmark: boosted-frame LWFA stage (3D, 128 x 128 x 1024 cells, 2 electrons per cell
= 33,554,432 particles, quadratic shape, 3-pass binomial filter, Vay pusher, FP32 storage
with the FP64 gamma solve), synthetic lab-frame inputs transformed to gamma_boost = 13.

Prints one JSON line: particle-steps/s of the whole step (gather + push + deposit +
filter + Maxwell), the fused particle kernel against the HBM roofline, the FP64 CPU
oracle on a bounded sample of the same workload, and an end-to-end figure through the C
ABI with host buffers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) the one 128 x 128 x 1024 instance is split along z into N slabs,
one per rank (paper_0909_5603_gb300.slab: ghost planes of J, E and B exchanged every
step, particles moved every MIGRATE_EVERY steps, all staged through host memory over a
gloo group); rank 0 prints particle-steps/s of the whole instance over the slowest
rank's time (strong scaling).  --replicas instead runs N independent copies (weak
scaling, no exchange).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import synth  # noqa: E402  (seeded input recipes, shared with the tests)

METRIC = "particle-steps/s (gather+Vay push+deposit) & % HBM roofline, FP32 vs FP64"

# ---- workload: lab-frame inputs of the boosted LWFA stage (normalised units, lambda0 = 1)
GAMMA_B = 13.0
LAMBDA0 = 1.0
N_GRID = (128, 128, 1024)
PPC = 2


def workload(nz=N_GRID[2]):
    return synth.lwfa_stage((N_GRID[0], N_GRID[1], nz), GAMMA_B, PPC, seed=3, lambda0=LAMBDA0)


# DRAM traffic of the particle kernel, from one ncu capture of a 128x128x128 slab of the
# same workload (profiles/k_particles_lwfa_128x128x128.md), valid while the kernel's
# sources are the ones that were captured
PROFILE = os.path.join(ROOT, "profiles", "k_particles_lwfa_128x128x128.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_0909_5603_gb300", "csrc", f)
                  for f in ("k_particles.cuh", "pic_device.cuh", "k_push.cuh", "k_push_f32.cu", "pic_instance.h")]


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_value(key):
    """A per-particle figure of the particle kernel's ncu capture, or None when the capture
    is absent or the kernel sources changed since it was taken."""
    try:
        with open(PROFILE) as f:
            kv = dict(line.split(":", 1) for line in f if line.startswith((key, "kernel_source_sha256")))
        if kv.get("kernel_source_sha256", "").strip() != kernel_source_hash():
            return None
        return float(kv[key])
    except (OSError, ValueError, KeyError):
        return None


def profiled_traffic(particles):
    """DRAM bytes per launch scaled from the capture, or None when the kernel changed."""
    per = profiled_value("dram_bytes_per_particle")
    return None if per is None else per * particles


def issue_roofline(kern_ms, particles, clocks):
    """The bound that applies to the particle kernel, instruction issue: warp instructions
    per launch (the capture's count per particle times the particles) over the measured
    launch time, against 4 warp instructions per SM-cycle on 152 SMs at the sampled SM
    clock (2070 MHz when no sample).  None when the capture is stale or absent."""
    per = profiled_value("warp_instructions_per_particle")
    if per is None or not kern_ms or kern_ms <= 0:
        return None
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    achieved = per * particles / (kern_ms * 1e-3) / 1e9
    peak = 152 * 4 * mhz * 1e-3
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "G warp-instructions/s",
            "frac": achieved / peak, "warp_instructions_per_particle": per, "sm_mhz": mhz}


def smem_roofline(kern_ms, particles, clocks):
    """The shared-memory pipe of the particle kernel (gather loads, deposit atomics, tile
    folds): shared-memory wavefronts per launch (the capture's count per particle times
    the particles) over the measured launch time, against one wavefront per SM-cycle on
    152 SMs at the sampled SM clock.  None when the capture is stale or absent."""
    per = profiled_value("shared_wavefronts_per_particle")
    if per is None or not kern_ms or kern_ms <= 0:
        return None
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    achieved = per * particles / (kern_ms * 1e-3) / 1e9
    peak = 152 * mhz * 1e-3
    return {"bound": "shared-memory wavefronts", "achieved": achieved, "peak": peak, "unit": "G wavefronts/s",
            "frac": achieved / peak, "wavefronts_per_particle": per, "sm_mhz": mhz}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("PIC_BENCH_GLOO") is None else "gloo"
        dist.init_process_group(backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------------ oracle (CPU)
def _oracle_worker(args):
    """One process: the FP64 oracle on a 128 x 128 x nz slab of the workload, `warmup`
    untimed then `steps` timed steps.  Returns (particle-steps, start, end, particles)."""
    nz, steps, warmup = args
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle
    import synth as synth_

    w = synth_.lwfa_stage((N_GRID[0], N_GRID[1], nz), GAMMA_B, PPC, seed=3, lambda0=LAMBDA0)
    s = oracle.Sim(3, w["n"], (1, 1, 1), w["dx"], w["dt"], order=2, filter_passes=3, tile=(8, 8, 8))
    p = w["plasma"]
    s.load_lab_frame(GAMMA_B, laser=w["laser"], plasma=[p[0], p[1], p[2], p[3], *p[4], p[5]])
    np0 = s.num_particles()
    s.step(warmup)
    t0 = time.time()
    done = 0.0
    for _ in range(steps):
        before = s.num_particles()
        s.step(1)
        done += 0.5 * (before + s.num_particles())
    return done, t0, time.time(), np0


def oracle_sample(steps, nz_sample=8, warmup=0, workers=1):
    """The FP64 oracle as it stands on a bounded sample of the workload: the same lab-frame
    plasma and grid spacing on a 128 x 128 x nz_sample slab, `steps` timed steps, in
    `workers` independent processes at once (one per host core for the all-core figure;
    the oracle itself is single-threaded).  Returns (particle-steps/s, sample, cores):
    the processes' particle-steps over the span from the first start to the last end."""
    import oracle

    oracle.build()
    if workers <= 1:
        res = [_oracle_worker((nz_sample, steps, warmup))]
    else:
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_oracle_worker, [(nz_sample, steps, warmup)] * workers)
    done = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    sample = (f"128x128x{nz_sample} slab of the same lab-frame plasma and spacing ({res[0][3]} particles), "
              f"{steps} timed steps after {warmup} untimed, "
              + ("single thread" if workers <= 1 else f"{workers} independent processes, one per host core"))
    oracle_sample.ms_per_step = 1e3 * span / max(steps, 1)
    return done / span, sample, max(1, workers)


def workload_name(nz):
    """The workload both arms report (the precision is the line's dtype and precision)."""
    return (f"boosted LWFA stage (3D laser wakefield), gamma_boost 13, 128x128x{nz} cells, "
            f"2 ppc = {2 * 128 * 128 * nz:,} particles, order-2 shape, 3-pass 1-2-1 filter, Vay")


def run_reference(args, rank, world):
    """The FP64 CPU oracle as it stands, each step a bounded sample of the workload."""
    if rank != 0:
        return
    v, sample, cores = oracle_sample(steps=args.steps, nz_sample=4, warmup=args.warmup, workers=os.cpu_count() or 1)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "particle-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": oracle_sample.ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.nz), "precision": "FP64 (the oracle)", "sample": sample},
            "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU arm
def run_ours(args, rank, world):
    import torch

    import paper_0909_5603_gb300 as pic

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local % max(torch.cuda.device_count(), 1))
    pic.build()
    w = workload(args.nz)
    ncell = w["n"][0] * w["n"][1] * w["n"][2]
    sim = pic.Simulation(3, w["n"], (1, 1, 1), w["dx"], w["dt"], gamma_boost=GAMMA_B, order=2,
                         precision=pic.PIC_PREC_FP32, pusher=pic.PIC_PUSHER_VAY, filter_passes=3, tile=(8, 8, 8),
                         track_ids=False)
    sim.load_lab_frame(laser=w["laser"], plasma=w["plasma"])
    n0 = sim.num_particles()
    stream = sim.stream
    sim.step(args.warmup)
    sim.synchronize()

    # ---- timed region: K steps through pic_step's CUDA graph (profiling off), CUDA events
    # on the library's stream
    nb = sim.num_particles()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1)
    na = sim.num_particles()
    psteps = 0.5 * (nb + na) * args.steps
    ms_max = allreduce_max(ms, world)
    psteps_all = allreduce_sum(psteps, world)
    value = psteps_all / (ms_max * 1e-3)

    # ---- phase split and the particle kernel's launch time: a separate pass of K steps
    # launched directly with CUDA events around every phase (pic_set_profiling)
    sim.set_profiling(True, reset=True)
    nb_p = sim.num_particles()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    sim.step(args.steps)
    p1.record(stream)
    torch.cuda.synchronize()
    tm = sim.timings()
    sim.set_profiling(False)
    na_p = sim.num_particles()
    ms_profiled = p0.elapsed_time(p1)

    # ---- roofline of the fused particle kernel
    peaks, peak_kind = measured_peaks()
    bytes_particle = 32 + 32     # read cell + 3 off + 3 u + w (FP32), write the same
    bytes_cell = 24 + 12         # E, B tile read; J tile flush
    kern_ms = tm["ms_particles"] / max(tm["steps"], 1)
    algo_bytes = 0.5 * (nb_p + na_p) * bytes_particle + ncell * bytes_cell
    achieved = algo_bytes / (kern_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": profiled_traffic(0.5 * (nb_p + na_p)), "peak_kind": peak_kind,
            "kernel": "k_particles_one<3,2,float,Vay>", "kernel_ms": kern_ms,
            "bytes_per_launch": algo_bytes,
            "kernel_timing": "CUDA events around each launch in a second pass of the same K steps (direct launches)"}

    # ---- FP64 path (the plain FP64 one-instance baseline at the same accuracy)
    fp64 = None
    if not args.skip_fp64:
        del sim
        torch.cuda.empty_cache()
        s64 = pic.Simulation(3, w["n"], (1, 1, 1), w["dx"], w["dt"], gamma_boost=GAMMA_B, order=2,
                             precision=pic.PIC_PREC_FP64, filter_passes=3, tile=(8, 8, 8), track_ids=False)
        s64.load_lab_frame(laser=w["laser"], plasma=w["plasma"])
        s64.step(2)
        s64.synchronize()
        s64.set_profiling(True, reset=True)
        k64 = max(2, args.steps // 4)
        nb64 = s64.num_particles()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(s64.stream)
        s64.step(k64)
        f1.record(s64.stream)
        torch.cuda.synchronize()
        t64 = s64.timings()
        na64 = s64.num_particles()
        fp64 = {"value": 0.5 * (nb64 + na64) * k64 / (f0.elapsed_time(f1) * 1e-3), "unit": "particle-steps/s",
                "steps": k64, "particle_kernel_ms": t64["ms_particles"] / max(t64["steps"], 1)}
        del s64
        torch.cuda.empty_cache()

    # ---- end to end through the C ABI with host buffers
    e2e = None if args.skip_e2e else end_to_end(pic, w, args, torch)
    scan = None if args.skip_scan else batched_scan(pic, torch)

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.skip_cpu:
        ncores = os.cpu_count() or 1
        v1, sample1, _ = oracle_sample(steps=20, nz_sample=8, warmup=1)
        v, sample, cores = oracle_sample(steps=20, nz_sample=8, warmup=1, workers=ncores)
        cpu = {"value": v, "unit": "particle-steps/s", "cores": cores, "kind": "oracle", "sample": sample,
               "host_cores": ncores, "single_thread": {"value": v1, "cores": 1, "sample": sample1}}
    line = {"metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args.nz), "precision": "FP32 storage + FP64 gamma solve",
                       "particles": n0, "cells": ncell, "l2": (f"inputs larger than L2 ({n0 * 32 / 1e9:.2f} GB of particles per buffer, L2 0.13 GB)"
                              if n0 * 32 > 129e6 else f"inputs of {n0 * 32 / 1e9:.3f} GB fit in L2"),
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "cell_updates_per_s": ncell * args.steps * world / (ms_max * 1e-3),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "fp64": fp64, "batched_scan": scan,
            "gpu_launches": int(round(tm["launches"] / max(tm["steps"], 1) * args.steps)),
            "phase_ms_per_step": {k: tm[k] / max(tm["steps"], 1) for k in
                                  ("ms_particles", "ms_scan", "ms_filter", "ms_maxwell", "ms_other")},
            "profiled_pass_ms_per_step": ms_profiled / args.steps,
            "clocks": clk.summary()}
    line["issue_roofline"] = issue_roofline(kern_ms, 0.5 * (nb_p + na_p), line["clocks"])
    line["smem_roofline"] = smem_roofline(kern_ms, 0.5 * (nb_p + na_p), line["clocks"])
    print(json.dumps(line), flush=True)


MIGRATE_EVERY = 8


def run_slabs(args, rank, world):
    """The instance split into `world` z slabs (one per rank); every rank loads the whole
    instance once, keeps its slab and frees the rest."""
    import torch
    import torch.distributed as dist

    import paper_0909_5603_gb300 as pic
    from paper_0909_5603_gb300 import slab as S

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local % max(torch.cuda.device_count(), 1))
    pic.build()
    w = workload(args.nz)
    n = w["n"]
    kw = dict(bc=(1, 1, 1), dx=w["dx"], dt=w["dt"], gamma_boost=GAMMA_B, order=2, precision=pic.PIC_PREC_FP32,
              pusher=pic.PIC_PUSHER_VAY, filter_passes=3, tile=(8, 8, 8), track_ids=False)
    whole = pic.Simulation(3, n, **kw)
    whole.load_lab_frame(laser=w["laser"], plasma=w["plasma"])
    n_whole = whole.num_particles()
    slabs = S.plan(n[2], world, False, ghost=S.ghost_planes(3, MIGRATE_EVERY))
    sim = S.split_gpu(whole, slabs, [rank], **kw)[rank]
    del whole
    torch.cuda.empty_cache()
    group = dist.new_group(backend="gloo")
    run = S.SlabRun(slabs, {rank: S.GpuShard(sim)}, S.Distributed(slabs[rank], group), n[0], n[1],
                    migrate_every=MIGRATE_EVERY)
    shard = run.shards[rank]
    run.step(args.warmup)
    sim.synchronize()
    nb = sim.num_particles()
    calls0 = shard.plane_launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(sim.stream)
        run.step(args.steps)
        e1.record(sim.stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1)
    psteps = 0.5 * (nb + sim.num_particles()) * args.steps
    ms_max = allreduce_max(ms, world)
    value = allreduce_sum(psteps, world) / (ms_max * 1e-3)
    plane_launches = shard.plane_launches - calls0
    # the step's own launches, counted by the library over one more (profiled) step
    sim.set_profiling(True, reset=True)
    run.step(1)
    sim.synchronize()
    step_launches = sim.timings()["launches"]
    sim.set_profiling(False)
    if rank != 0:
        return
    ncell = n[0] * n[1] * n[2]
    line = {"metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args.nz), "precision": "FP32 storage + FP64 gamma solve",
                       "particles": n_whole, "cells": ncell,
                       "l2": f"inputs larger than L2 ({n_whole * 32 / world / 1e9:.2f} GB of particles per slab)",
                       "parallelism": f"z slabs x{world}, {slabs[0].ghost} ghost planes, particles moved every "
                                      f"{MIGRATE_EVERY} steps, exchange through host memory (gloo)"},
            "cell_updates_per_s": ncell * args.steps / (ms_max * 1e-3),
            "roofline": None, "cpu_baseline": None, "e2e": None,
            "gpu_launches": int(step_launches * args.steps + plane_launches),
            "note": "per-kernel roofline, CPU baseline and end-to-end figures come from the 1-GPU run; "
                    "gpu_launches counts rank 0's phase and plane pack/unpack launches (not the relayouts "
                    "of moved particles)",
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def end_to_end(pic, w, args, torch):
    """Same metric through the public API with host buffers: the particle state is
    uploaded from pinned host memory in the storage precision (FP32, the run's own), K
    steps run, each step's diagnostics are read back and the final particles are copied
    into pinned host arrays allocated beforehand, all inside the timed region."""
    src = pic.Simulation(3, w["n"], (1, 1, 1), w["dx"], w["dt"], gamma_boost=GAMMA_B, order=2,
                         precision=pic.PIC_PREC_FP32, filter_passes=3, tile=(8, 8, 8), track_ids=False)
    src.load_lab_frame(laser=w["laser"], plasma=w["plasma"])
    p = src.get_particles(stored=True)
    ex, by = src.get_field(pic.PIC_EX), src.get_field(pic.PIC_BY)
    del src
    torch.cuda.empty_cache()

    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    # pinned host copies of the inputs, pinned room for the outputs
    hp = {k: pinned(p[k]) for k in ("cell", "off", "u", "w")}
    hex_, hby = pinned(ex), pinned(by)
    npart = hp["cell"].size
    out = {k: pinned(np.empty_like(v)) for k, v in p.items()}
    sim = pic.Simulation(3, w["n"], (1, 1, 1), w["dx"], w["dt"], gamma_boost=GAMMA_B, order=2,
                         precision=pic.PIC_PREC_FP32, filter_passes=3, tile=(8, 8, 8), track_ids=False)
    k = args.steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.load_particles(hp["cell"], hp["off"], hp["u"], hp["w"])
    sim.set_field(pic.PIC_EX, hex_)
    sim.set_field(pic.PIC_BY, hby)
    nb = sim.num_particles()
    for _ in range(k):
        sim.step(1)
        sim.diagnostics()
    res = sim.get_particles(stored=True, out=out)
    t1 = time.perf_counter()
    na = res["cell"].size
    h2d = npart * (4 + 12 + 12 + 4) + 2 * hex_.size * 8
    d2h = k * 64 + na * (4 + 12 + 12 + 4 + 4)
    del sim
    torch.cuda.empty_cache()
    return {"value": 0.5 * (nb + na) * k / (t1 - t0), "unit": "particle-steps/s",
            "h2d_bytes_per_step": int(h2d / k), "d2h_bytes_per_step": int(d2h / k),
            "seconds": t1 - t0, "includes": "host validation and tile sort of 33.5M FP32 particles and their "
                                            "upload (plus the library's 4 B/particle slot array), two FP64 "
                                            "field uploads, K steps with per-step diagnostics read-back, final "
                                            "FP32 particle read-back into pinned arrays"}


def batched_scan(pic, torch, count=256, steps=10, steps64=3, warmup=3):
    """The batched 2D3V boosted-frame scan: `count` independent instances (seeded recipe
    tests/synth.py scan_instance: N x N with log2 N in [6, 9], 1-16 electrons per cell,
    gamma_b in [1, 50], n/n_c in [1e-4, 1e-2]) advanced as one batch in FP32 with the FP64
    gamma solve (one launch per phase over all instances, replayed from one CUDA graph),
    against the same instances in FP64 stepped one at a time on one stream."""
    ds = [synth.scan_instance(i) for i in range(count)]

    def make(d, prec, stream=None):
        s = pic.Simulation(2, d["n"], (0, 0, 0), d["dx"], d["dt"], gamma_boost=d["gamma_boost"], order=2,
                           precision=prec, filter_passes=3, tile=(16, 1, 16), track_ids=False, stream=stream)
        s.load_lab_frame(laser=d["laser"], plasma=d["plasma"])
        return s

    t = time.perf_counter()
    sims = [make(d, pic.PIC_PREC_FP32) for d in ds]
    load_s = time.perf_counter() - t
    cells = sum(d["n"][0] * d["n"][2] for d in ds)
    batch = pic.Batch(sims)
    batch.step(warmup)
    batch.synchronize()
    nb = sum(s.num_particles() for s in sims)
    stream = sims[0].stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    batch.step(steps)
    e1.record(stream)
    batch.synchronize()
    ms = e0.elapsed_time(e1) / steps
    na = sum(s.num_particles() for s in sims)
    out = {"instances": count, "particles": int(nb), "cells": int(cells), "steps": steps,
           "load_seconds": round(load_s, 2), "ms_per_step": ms,
           "particle_steps_per_s": 0.5 * (nb + na) / (ms * 1e-3),
           "cell_updates_per_s": cells / (ms * 1e-3), "dtype": "f32",
           "launch": "per-phase kernels over all instances, one CUDA graph replay per step"}
    # the same batch as one persistent launch per call (every step of the call)
    batch.set_persistent(True)
    batch.step(1)
    batch.synchronize()
    nbp = sum(s.num_particles() for s in sims)
    e0.record(stream)
    batch.step(steps)
    e1.record(stream)
    batch.synchronize()
    msp = e0.elapsed_time(e1) / steps
    nap = sum(s.num_particles() for s in sims)
    out["persistent"] = {"ms_per_step": msp, "particle_steps_per_s": 0.5 * (nbp + nap) / (msp * 1e-3),
                         "launch": f"one persistent launch for the {steps} steps"}
    batch.close()
    del sims, batch
    torch.cuda.empty_cache()
    # FP64, one instance after the other on one stream (each its own launches and graph)
    common = torch.cuda.Stream()
    sims64 = [make(d, pic.PIC_PREC_FP64, common) for d in ds]
    for s in sims64:
        s.step(1)
    torch.cuda.synchronize()
    n64 = sum(s.num_particles() for s in sims64)
    e0.record(common)
    for _ in range(steps64):
        for s in sims64:
            s.step(1)
    e1.record(common)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1) / steps64
    out["fp64_one_at_a_time"] = {"ms_per_step": ms64, "particle_steps_per_s": n64 / (ms64 * 1e-3),
                                 "steps": steps64}
    del sims64
    torch.cuda.empty_cache()
    return out


def precision_sweep(pic, torch, args):
    """The LWFA stage at scale for several boosts (256 x 256 x 2048 cells, 4 electrons per
    cell, about 5.4e8 particles): the FP32 path (FP64 gamma solve) against the all-FP64 GPU
    path after `--sweep-steps` steps.  Reports per boost the normwise relative difference
    of the wake field E_z and of E_x, the relative difference of the field and kinetic
    energies, and both paths' particle-steps/s."""
    out = []
    gammas = [float(g) for g in args.sweep_gammas.split(",")]
    for gb in gammas:
        w = synth.lwfa_stage((256, 256, 2048), gb, 4, seed=4 + gammas.index(gb))
        res = {"gamma_boost": gb}
        fields, diags = {}, {}
        for prec, name in ((pic.PIC_PREC_FP32, "fp32"), (pic.PIC_PREC_FP64, "fp64")):
            sim = pic.Simulation(3, w["n"], (1, 1, 1), w["dx"], w["dt"], gamma_boost=gb, order=2, precision=prec,
                                 filter_passes=3, tile=(8, 8, 8), track_ids=False)
            sim.load_lab_frame(laser=w["laser"], plasma=w["plasma"])
            n = sim.num_particles()
            sim.step(2)
            sim.synchronize()
            sim.set_profiling(True, reset=True)
            sim.step(args.sweep_steps - 2)
            sim.synchronize()
            t = sim.timings()
            ms = sum(t[k] for k in ("ms_particles", "ms_scan", "ms_filter", "ms_maxwell", "ms_other")) / t["steps"]
            res[name] = {"particles": n, "ms_per_step": ms, "particle_steps_per_s": n / (ms * 1e-3),
                         "particle_kernel_ms": t["ms_particles"] / t["steps"]}
            fields[name] = {c: sim.get_field(c) for c in (pic.PIC_EZ, pic.PIC_EX)}
            diags[name] = sim.diagnostics()
            del sim
            torch.cuda.empty_cache()
        for c, key in ((pic.PIC_EZ, "Ez"), (pic.PIC_EX, "Ex")):
            a, b = fields["fp32"][c], fields["fp64"][c]
            res[f"rel_err_{key}"] = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
        for k in ("field_energy", "kinetic_energy"):
            res[f"rel_err_{k}"] = abs(diags["fp32"][k] - diags["fp64"][k]) / max(abs(diags["fp64"][k]), 1e-300)
        res["steps"] = args.sweep_steps
        out.append(res)
        print(json.dumps(res), flush=True)
    return out


def instability_study(pic, torch, args):
    """Boosted-frame numerical instability (Sec. 2: a short-wavelength instability whose
    growth rises with the boost and the inverse resolution, controlled with low-dispersion
    solvers and low-pass filtering): the LWFA stage downscaled to 32 x 32 x 256 cells with
    a 2-period laser, cold plasma with its ions, FP32, for each boost, solver and number of
    filter passes; reports max |E| after `--study-steps` steps over its value after 10
    steps (the laser's), and the field energy ratio.  Yee runs at dt = dz/2 capped at 0.9
    of its Courant limit; the low-dispersion solver at dt = 0.9 min(dx, dz)."""
    rows = []
    for gb in [float(g) for g in args.sweep_gammas.split(",")]:
        w = synth.lwfa_stage((32, 32, 256), gb, 2)
        lz = w["n"][2] * w["dx"][2]
        doppler = gb * (1 + math.sqrt(1 - 1 / gb ** 2))
        laser = (2.0, 1.0, 20.0, 2.0, 0.5 * lz / doppler)
        for solver, name in ((pic.PIC_SOLVER_YEE, "yee"), (pic.PIC_SOLVER_CK, "ck")):
            dt = w["dt"] if solver == pic.PIC_SOLVER_YEE else 0.9 * min(w["dx"][0], w["dx"][2])
            for passes in (0, 3):
                sim = pic.Simulation(3, w["n"], (1, 1, 1), w["dx"], dt, gamma_boost=gb, order=2,
                                     precision=pic.PIC_PREC_FP32, filter_passes=passes, tile=(8, 8, 8),
                                     track_ids=False, solver=solver, absorb_cells=8)
                sim.load_lab_frame(laser=laser, plasma=w["plasma"])
                sim.step(10)
                e0 = max(np.abs(sim.get_field(c)).max() for c in (pic.PIC_EX, pic.PIC_EY, pic.PIC_EZ))
                f0 = sim.diagnostics()["field_energy"]
                sim.step(args.study_steps - 10)
                e1 = max(np.abs(sim.get_field(c)).max() for c in (pic.PIC_EX, pic.PIC_EY, pic.PIC_EZ))
                f1 = sim.diagnostics()["field_energy"]
                row = {"gamma_boost": gb, "solver": name, "filter_passes": passes, "dt": dt,
                       "steps": args.study_steps, "max_E_growth": e1 / e0, "field_energy_ratio": f1 / f0}
                rows.append(row)
                print(json.dumps(row), flush=True)
                del sim
                torch.cuda.empty_cache()
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-scan", action="store_true", help="skip the 256-instance batched scan")
    ap.add_argument("--precision-sweep", action="store_true",
                    help="instead of the benchmark: FP32 vs FP64 on the LWFA stage at 256x256x2048, 4 ppc, per boost")
    ap.add_argument("--sweep-gammas", default="2,5,13,30,100")
    ap.add_argument("--sweep-steps", type=int, default=100)
    ap.add_argument("--instability-study", action="store_true",
                    help="instead of the benchmark: field growth per boost, solver and filter passes")
    ap.add_argument("--study-steps", type=int, default=400)
    ap.add_argument("--replicas", action="store_true",
                    help="with N > 1: N independent copies of the instance instead of N z slabs of one")
    ap.add_argument("--nz", type=int, default=N_GRID[2],
                    help="cells along z (a shorter slab of the same workload, for profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world = dist_init()
    if args.instability_study:
        import torch

        import paper_0909_5603_gb300 as pic
        pic.build()
        print(json.dumps({"instability_study": instability_study(pic, torch, args)}))
    elif args.precision_sweep:
        import torch

        import paper_0909_5603_gb300 as pic
        pic.build()
        print(json.dumps({"precision_sweep": precision_sweep(pic, torch, args)}))
    elif args.impl == "reference":
        run_reference(args, rank, world)
    elif world > 1 and not args.replicas:
        run_slabs(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
