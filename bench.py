#!/usr/bin/env python3
"""Throughput benchmark of the GB300 WaterLily time step (libwl.so through its C ABI).

One "step" is one full time step (simstep!: two convection-diffusion + BDIM stages,
two multigrid projections to Poisson tol 1e-6, the CFL time step) of the whole
domain.  The metric is cells*steps/s; V-cycles/s and the roofline fraction of the
dominant kernel are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

N > 1 is launched by torchrun, one rank per GPU; every rank advances an independent
replica of the workload (the method has no data exchange between replicas), the
value is all ranks' cells*steps divided by the slowest rank's time.
The reference arm is the FP64 CPU oracle timed on the host cores on a bounded
sample of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # 3-D flow past a sphere, radius 16 cells, Re = 3700 (diameter based), uniform inflow
    "sphere512": dict(dims=(512, 256, 256), nu=32.0 / 3700.0, U=(1.0, 0.0, 0.0),
                      body=dict(kind=1, center=(128.0, 128.0, 128.0), radius=16.0), periodic=0, ic=0,
                      desc="3-D flow past a sphere R=16, Re=3700, 512x256x256 cells, uniform inflow, tol 1e-6"),
    "sphere256": dict(dims=(256, 128, 128), nu=32.0 / 3700.0, U=(1.0, 0.0, 0.0),
                      body=dict(kind=1, center=(64.0, 64.0, 64.0), radius=16.0), periodic=0, ic=0,
                      desc="3-D flow past a sphere R=16, Re=3700, 256x128x128 cells, uniform inflow, tol 1e-6"),
    # the same sphere on a 3/4-scale grid (14.2 M cells, one FP32 field 57 MB): larger than
    # L2 in what each kernel touches, small enough for multi-pass profiler captures
    "sphere384": dict(dims=(384, 192, 192), nu=32.0 / 3700.0, U=(1.0, 0.0, 0.0),
                      body=dict(kind=1, center=(96.0, 96.0, 96.0), radius=16.0), periodic=0, ic=0,
                      desc="3-D flow past a sphere R=16, Re=3700, 384x192x192 cells, uniform inflow, tol 1e-6"),
    "tgv128": dict(dims=(128, 128, 128), nu=(128.0 / (2 * 3.141592653589793)) / 1600.0, U=(0.0, 0.0, 0.0),
                   body=None, periodic=7, ic=1,
                   desc="3-D Taylor-Green vortex, 128^3 periodic, Re=1600, tol 1e-6"),
    # the paper's donut: a torus (axis along the flow) in an N = (2^(p+1), 2^p, 2^p) box,
    # Re = 1000 on the ring diameter; ring radius 2^p/8 and tube radius 2^p/32 centred a
    # quarter of the way down the box (the paper shows the shape, not its dimensions)
    "donut256": dict(dims=(256, 128, 128), nu=32.0 / 1000.0, U=(1.0, 0.0, 0.0),
                     body=dict(kind=2, center=(64.0, 64.0, 64.0), radius=16.0, radius2=4.0), periodic=0, ic=0,
                     desc="3-D flow past a torus R=16 r=4 (axis along the flow), Re=1000, 256x128x128 cells, tol 1e-6"),
    "donut512": dict(dims=(512, 256, 256), nu=64.0 / 1000.0, U=(1.0, 0.0, 0.0),
                     body=dict(kind=2, center=(128.0, 128.0, 128.0), radius=32.0, radius2=8.0), periodic=0, ic=0,
                     desc="3-D flow past a torus R=32 r=8 (axis along the flow), Re=1000, 512x256x256 cells, tol 1e-6"),
    "cyl128x64": dict(dims=(128, 64), nu=0.064, U=(1.0, 0.0), body=dict(kind=1, center=(32.0, 32.0), radius=8.0),
                      periodic=0, ic=0, desc="2-D flow past a circle R=8, Re=250, 128x64 cells, tol 1e-6"),
    # the paper's own benchmark shape: Taylor-Green vortex at Re = 1e5 on N^3 (N = 2^p,
    # 2^21 and 2^24 cells), length scale N/(2 pi)
    "tgv128re1e5": dict(dims=(128, 128, 128), nu=(128.0 / (2 * 3.141592653589793)) / 1e5, U=(0.0, 0.0, 0.0),
                        body=None, periodic=7, ic=1, desc="3-D Taylor-Green vortex, 128^3 periodic, Re=1e5, tol 1e-6"),
    "tgv256re1e5": dict(dims=(256, 256, 256), nu=(256.0 / (2 * 3.141592653589793)) / 1e5, U=(0.0, 0.0, 0.0),
                        body=None, periodic=7, ic=1, desc="3-D Taylor-Green vortex, 256^3 periodic, Re=1e5, tol 1e-6"),
}

# Algorithmic bytes per fine-level cell of one launch of each kernel class (D
# dimensions, FP32 fields, double-float fine pressure), each array read or written
# once:
#   sweep_fine : mean of the 4 sweeps of a cycle: first (coarse correction 4/2^D +
#                rhs 4 + faces 4D + out 4), two middle (in 4 + rhs 4 + faces 4D +
#                out 4), last (in 4 + rhs 4 + faces 4D + pressure hi/lo read and
#                written 16)
#   resid_fine : residual: pressure 8 + rhs 4 + faces 4D + residual out 4 +
#                restricted 4/2^D; the projection's first pass also reads the
#                velocity 4D and writes the rhs instead of reading it (same count)
#   stage      : stage 1 reads u 4D + mu0 4D, writes 4D; stage 2 also reads u0 4D
#   correct    : u 4D + faces 4D + pressure 8 in, u 4D out
# Where the fine level splits its tiles (wl_level_split), the tiles away from the body
# form their face coefficients instead of reading them: the 4D face bytes of the sweep
# and the residual count only for the band_fraction of tiles that read them.
def algo_bytes(cls, D, n_div=0, n_res=0, band_fraction=1.0):
    f = 4.0 * D
    if cls in ("sweep_fine", "resid_fine"):
        f *= band_fraction
    if cls == "sweep_fine":
        first = 4.0 / 2**D + 4 + f + 4
        mid = 4 + 4 + f + 4
        last = 4 + 4 + f + 16
        return (first + 2 * mid + last) / 4
    if cls == "resid_fine":
        res = 8 + 4 + f + 4 + 4.0 / 2**D
        div = res + f
        return (n_div * div + n_res * res) / max(n_div + n_res, 1)
    if cls == "stage":
        return (3 * f + 4 * f) / 2
    if cls == "correct":
        return 3 * f + 8
    raise KeyError(cls)


KERNEL_NAMES = {"sweep_fine": "k_sweep_tma<3> (fine level)", "resid_fine": "k_resid_tma (fine level)",
                "stage": "k_stage<3>", "correct": "k_correct3"}


def kernel_name(cls, D, periodic, dims=None):
    """The kernels behind a class on this grid: tiles across a periodic x or y side sweep
    in the staged kernel's wrapping variant when those sides are whole 64 x 8 tiles away
    from the body (every periodic workload here is body-free), else in the table kernel
    k_sweep; the fine residual of a periodic grid is k_residual."""
    name = KERNEL_NAMES[cls].replace("<3>", f"<{D}>")
    whole = dims is not None and (not periodic & 1 or dims[0] % 64 == 0) and (not periodic & 2 or dims[1] % 8 == 0)
    if cls == "sweep_fine" and periodic & 3 and not whole:
        name = f"k_sweep_tma<{D}> + k_sweep<{D}> (fine level; k_sweep: tiles across a periodic side)"
    if cls == "resid_fine" and (periodic or D == 2):
        name = f"k_residual<{D}> (fine level)"
    if cls == "correct" and D == 2:
        name = "k_correct<2>"
    return name
KERNEL_SRC = {"sweep_fine": "wl_sweep_tma.cu", "resid_fine": "wl_sweep_tma.cu", "stage": "wl_momentum.cu",
              "correct": "wl_poisson.cu", "sweep_fine_uni": "wl_sweep_tma.cu", "resid_fine_uni": "wl_sweep_tma.cu"}
# the kernel classes of wl_profile_step that partition a step (the *_uni / *_bandt classes
# time the fine level's split launches again, one by one)
BASE_CLASSES = ("stage", "band", "resid_fine", "restrict", "sweep_fine", "sweep_coarse", "coarsest", "correct",
                "control")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _src_sha(name):
    path = os.path.join(ROOT, "paper_2304_08159_gb300", "csrc", name)
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _traffic(cls, ncell, n_div=0, n_res=0):
    """DRAM bytes per launch of a kernel class from the committed ncu capture on the
    512x256x256 grid (per fine cell, scaled to this workload's cells), averaged like
    algo_bytes: the 4 sweeps of a V-cycle, divergence and residual passes in the
    profiled step's proportion; None when the kernel source changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            t = json.load(f)[cls]
        if t["src_sha"] != _src_sha(KERNEL_SRC[cls]):
            return None
        if cls in ("resid_fine", "resid_fine_uni"):
            per = (n_div * t["divergence"] + n_res * t["residual"]) / max(n_div + n_res, 1)
        else:
            per = t["bytes_per_cell"]
        return per * ncell
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group("nccl")
        return dist, dist.get_rank(), ws, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


def reduce_replicas(dist, t, vcycles, device):
    """Slowest rank's time and all ranks' V-cycles (t and vcycles of this rank)."""
    if dist is None:
        return t, vcycles
    import torch

    mx = torch.tensor([t], dtype=torch.float64, device=device)
    sm = torch.tensor([float(vcycles)], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx.item(), sm.item()


def job_value(world, ncell, steps, tmax):
    """Whole-job cells*steps/s: every replica's cells*steps over the slowest time."""
    return world * ncell * steps / tmax


def _launches_per_step(nlev, post, has_body):
    """Kernels one graph step launches outside the V-cycles, and per V-cycle."""
    fixed = 2 * (1 + (1 if has_body else 0))  # stages (+ band)
    fixed += 2 * 2  # per projection: divergence/residual + decision
    fixed += 2 + 1  # corrections + step end
    # restrictions, coarsest solve, sweeps of every level but the coarsest, fine
    # residual, decision; a single-level hierarchy: solve, fold into the pressure,
    # residual, decision
    per_cycle = (nlev - 2) + 1 + (nlev - 1) * post + 2 if nlev > 1 else 4
    return fixed, per_cycle


def cpu_oracle_step_rate(w, steps=1):
    """The FP64 oracle (as it is) on the host cores: setup, then `steps` timed full
    time steps with multigrid projections at tol 1e-6.  Returns (cells*steps/s, s, cores)."""
    import oracle as O

    o = O.Oracle(w["dims"], w["nu"], U=w["U"], periodic=w["periodic"], body=w["body"])
    o.set_ic(w["ic"], 1.0)
    t0 = time.perf_counter()
    o.step(steps, tol=1e-6, maxit=32, solver=1)
    t = time.perf_counter() - t0
    ncell = 1
    for d in w["dims"]:
        ncell *= d
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return ncell * steps / t, t, cores


def bench_config(args, w, ws):
    """The workload's `config` dict, the same in both arms."""
    ncell = 1
    for d in w["dims"]:
        ncell *= d
    field_mb = 4.0 * ncell / 1e6
    if field_mb > 129.0:
        l2 = "inputs larger than L2 (one FP32 field of the grid is %.0f MB, L2 129 MB)" % field_mb
    else:
        l2 = ("fields smaller than L2 (one FP32 field %.1f MB): steps run back to back, L2 not flushed; "
              "a table row, not the headline" % field_mb)
    return {"workload": args.workload, "desc": w["desc"], "cells": ncell, "dims": list(w["dims"]),
            "poisson_tol": args.tol, "replicas": ws, "l2": l2}


def run_reference(args, w, rank, ws):
    if rank != 0:
        return 0
    ncell = 1
    for d in w["dims"]:
        ncell *= d
    steps = max(1, min(args.steps, args.ref_steps))
    if args.warmup > 0 and args.ref_warmup > 0:
        cpu_oracle_step_rate(w, 1)
    rate, t, cores = cpu_oracle_step_rate(w, steps)
    sample = (f"{steps} full time step(s) of the {args.workload} workload by the FP64 oracle "
              f"(multigrid V(0,4) projections to tol 1e-6) after its setup; the arm's --steps is capped "
              f"at {args.ref_steps} to bound CPU time")
    line = {"impl": "reference", "metric": "cells*steps/s", "value": rate, "unit": "cell*step/s",
            "n_gpus": ws, "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(args, w, ws),
            "cpu_baseline": {"value": rate, "unit": "cell*step/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": "cell*step/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, w, dist, rank, ws, lrank):
    import numpy as np
    import torch

    from paper_2304_08159_gb300 import Sim, wl

    torch.cuda.set_device(lrank)
    ncell = int(np.prod(w["dims"]))
    D = len(w["dims"])
    sim = Sim(w["dims"], w["nu"], w["U"], body=w["body"], periodic=w["periodic"], tol=args.tol)
    if w["ic"]:
        sim.set_ic(w["ic"], 1.0)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    sim.step(args.warmup)
    _, _, vc_warm, _ = sim.status()  # the V-cycle total is cumulative since creation
    barrier()
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(lrank).uuid)
    except Exception:
        gpu_id = str(lrank)
    clocks = ClockSampler(gpu_id)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    barrier()
    ck = clocks.stop()
    t = e0.elapsed_time(e1) / 1e3
    rc, last, vc_end, worst = sim.status()
    vcycles = vc_end - vc_warm  # the timed steps' V-cycles
    tmax, vtot = reduce_replicas(dist, t, vcycles, "cuda")
    value = job_value(ws, ncell, args.steps, tmax)
    nlev = len(sim.levels())
    try:  # the captured step graph's own kernel nodes (per step, per V-cycle)
        fixed, per_cycle = sim.graph_kernels()
    except Exception:
        fixed, per_cycle = _launches_per_step(nlev, 4, w["body"] is not None)
    launches = args.steps * fixed + vcycles * per_cycle

    # ---- per-kernel device time (host-driven steps with events around each launch)
    # an NVTX range around the host-driven steps lets ncu select their launches
    # (--nvtx --nvtx-include "wl_profile_step/"); the timed graph steps hide theirs
    torch.cuda.nvtx.range_push("wl_profile_step")
    prof = sim.profile_step(args.prof_steps)
    torch.cuda.nvtx.range_pop()
    prof_steps = args.prof_steps
    peak, peak_kind = _peaks()
    cls = max(("sweep_fine", "resid_fine", "stage", "correct"), key=lambda k: prof[k][0])
    ms_tot, n = prof[cls]
    nd = min(2 * prof_steps, n)
    split, band_fraction = sim.level_split(0)
    step_ms = sum(prof[k][0] for k in BASE_CLASSES)
    uni = cls + "_uni"
    if uni in prof and prof[uni][1] == n and n > 0:
        # the fine level splits into two launches, the uniform tiles' kernel on the sim's
        # stream and the band tiles' beside it: the dominant kernel is the uniform one,
        # timed on its own stream; its bytes are those of the uniform tiles' cells, which
        # form their face coefficients instead of reading them
        bytes_launch = algo_bytes(cls, D, nd, n - nd, 0.0) * ncell * (1.0 - band_fraction)
        avg_s = prof[uni][0] / n / 1e3
        name = kernel_name(cls, D, w["periodic"], w["dims"]) + ", uniform-tile launch"
        traffic = _traffic(uni, ncell, nd, n - nd)
        pair = {"pair_avg_launch_ms": ms_tot / n, "band_tile_launch_ms": prof[cls + "_bandt"][0] / n}
    else:
        bytes_launch = algo_bytes(cls, D, nd, n - nd, band_fraction) * ncell
        avg_s = ms_tot / n / 1e3
        name = kernel_name(cls, D, w["periodic"], w["dims"])
        traffic = _traffic(cls, ncell, nd, n - nd)
        pair = {}
    achieved = bytes_launch / avg_s / 1e9
    roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
            "algorithmic_bytes_per_launch": bytes_launch, "avg_launch_ms": avg_s * 1e3,
            "coefficients_read_by_fraction_of_tiles": band_fraction,
            "share_of_step": ms_tot / step_ms, **pair}
    kern = {k: {"ms_per_step": v[0] / prof_steps, "launches_per_step": v[1] / prof_steps} for k, v in prof.items()}

    # ---- end to end through the C ABI with pinned host buffers: state in, step, state out
    host_u = torch.empty(D * ncell, dtype=torch.float32, pin_memory=True)
    sim_u = sim.get(wl.WL_FIELD_U, device=True).reshape(-1)
    host_u.copy_(sim_u)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sim._check(wl.wl_set_field(sim.h, wl.WL_FIELD_U, host_u.data_ptr(), 0), "wl_set_field")
        sim.step(1)
        sim._check(wl.wl_get_field(sim.h, wl.WL_FIELD_U, host_u.data_ptr(), 0), "wl_get_field")
    barrier()
    te = time.perf_counter() - t0
    te, _ = reduce_replicas(dist, te, 0, "cuda")
    e2e = {"value": job_value(ws, ncell, e2e_steps, te), "unit": "cell*step/s", "h2d_bytes_per_step": 4 * D * ncell,
           "d2h_bytes_per_step": 4 * D * ncell, "steps": e2e_steps}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, tcpu, cores = cpu_oracle_step_rate(w, 1)
        cpu = {"value": rate, "unit": "cell*step/s", "cores": cores, "kind": "oracle",
               "sample": f"1 full time step of the {args.workload} workload by the FP64 oracle (multigrid "
                         f"V(0,4) projections to tol 1e-6) after its setup, {tcpu:.1f} s"}

    mixed = None
    if rank == 0 and ws == 1 and not args.no_mixed:
        sim.close()
        try:
            mixed = mixed_bench(w, args)
        except Exception as e:  # reported, not fatal: the main measurement stands
            mixed = {"error": f"{type(e).__name__}: {e}"}

    adjoint = None
    if rank == 0 and ws == 1 and not args.no_adjoint:
        try:
            adjoint = adjoint_bench(args.tol)
        except Exception as e:  # reported, not fatal: the main measurement stands
            adjoint = {"error": f"{type(e).__name__}: {e}"}

    serving = None
    if rank == 0 and ws == 1 and not args.no_serve:
        try:
            serving = serving_bench(args.serve_requests, args.tol)
        except Exception as e:  # reported, not fatal: the main measurement stands
            serving = {"error": f"{type(e).__name__}: {e}"}

    # whole-step roofline: algorithmic bytes per cell per step of the model (3-D: 196 B
    # fixed + 142 B per V-cycle; 2-D: 136 B + 187 B), with the V-cycles actually run
    nv = vcycles / args.steps
    bstep = (196.0 + 142.0 * nv) if D == 3 else (136.0 + 187.0 * nv)
    at_peak = peak * 1e9 / bstep
    step_roof = {"bytes_per_cell_step": bstep, "vcycles_per_step": nv, "cells_steps_per_s_at_peak": at_peak,
                 "frac": value / ws / at_peak, "peak": peak, "peak_kind": peak_kind}

    if rank == 0:
        line = {"metric": "cells*steps/s", "value": value, "unit": "cell*step/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": bench_config(args, w, ws),
                "vcycles_per_s": vtot / tmax, "vcycles_per_step": vcycles / args.steps,
                "converged": rc == 0, "worst_residual": worst,
                "roofline": roof, "step_roofline": step_roof, "kernels": kern, "cpu_baseline": cpu, "e2e": e2e,
                "mixed_precision": mixed, "adjoint": adjoint, "serving": serving, "clocks": ck,
                "gpu_launches": int(ws * launches)}
        print(json.dumps(line), flush=True)
    sim.close()
    return 0


def mixed_bench(w, args):
    """The same workload with the multigrid levels between the fine and the coarsest
    one stored in BF16 and in FP16 (FP32 arithmetic; fine residual, pressure and FP64
    coarsest solve unchanged), timed like the main line over up to 100 steps, and its
    velocity and pressure after warm-up + those steps against an FP32 run of the same
    steps (relative L2; the pressure with its mean removed)."""
    import numpy as np
    import torch

    from paper_2304_08159_gb300 import Sim

    steps = max(1, min(args.steps, 100))
    stream = torch.cuda.current_stream()

    def run(cp):
        sim = Sim(w["dims"], w["nu"], w["U"], body=w["body"], periodic=w["periodic"], tol=args.tol,
                  coarse_precision=cp)
        if w["ic"]:
            sim.set_ic(w["ic"], 1.0)
        sim.step(args.warmup)
        _, _, vc0, _ = sim.status()  # cumulative since creation
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        rc, last, vc1, worst = sim.status()
        vc = vc1 - vc0
        u, p = sim.get(0, device=True).double(), sim.get(1, device=True).double()
        sim.close()
        return t, vc, rc, worst, u, p - p.mean()

    ncell = int(np.prod(w["dims"]))
    t32, vc32, _, _, u32, p32 = run("fp32")
    out = {"steps": steps, "poisson_tol": args.tol,
           "fp32": {"value": ncell * steps / t32, "unit": "cell*step/s", "vcycles_per_step": vc32 / steps}}
    for cp in ("bf16", "fp16"):
        t, vc, rc, worst, u, p = run(cp)
        out[cp] = {"value": ncell * steps / t, "unit": "cell*step/s", "vcycles_per_step": vc / steps,
                   "converged": rc == 0, "worst_residual": worst, "speedup_vs_fp32": t32 / t,
                   "rel_l2_u_vs_fp32": float(torch.linalg.norm(u - u32) / torch.linalg.norm(u32)),
                   "rel_l2_p_vs_fp32": float(torch.linalg.norm(p - p32) / torch.linalg.norm(p32))}
        del u, p
    return out


def adjoint_bench(tol):
    """The adjoint configuration: 2-D cylinder 256x128, R = 12 at (64, 64), Re = 200 on the
    diameter, U = 1, fixed dt 0.1, mean drag coefficient over 50 steps differentiated with
    respect to (R, cx, cy) by the hand-written adjoint with checkpoints every 10 steps.
    Wall time of the recorded forward rollout and of the backward pass (segment
    recomputation + adjoint): step graphs, the adjoint solves' V-cycles in WHILE nodes,
    one synchronisation at the end of each pass (graph builds included)."""
    import numpy as np

    from paper_2304_08159_gb300 import Sim

    nsteps, every, R = 50, 10, 12.0

    def run():
        sim = Sim((256, 128), 24.0 / 200.0, (1.0, 0.0), body=dict(kind=1, center=(64.0, 64.0), radius=R), tol=tol,
                  dt_fixed=0.1)
        t0 = time.perf_counter()
        F = sim.grad_forward(nsteps, every)
        t1 = time.perf_counter()
        g = np.zeros_like(F)
        g[:, 0] = 1.0 / (nsteps * R)
        tb = sim.grad_backward(g)
        t2 = time.perf_counter()
        ws = sim.grad_workspace.numel()
        sim.close()
        J = F[:, 0].mean() / R
        tb[0] -= J / R
        return t1 - t0, t2 - t1, J, tb, ws

    run()  # warm-up (module load, first kernel launches)
    tf, tbk, J, tb, ws = run()
    ncell = 256 * 128
    return {"workload": "2-D cylinder 256x128, R=12, Re=200, 50 steps at dt=0.1, checkpoints every 10",
            "forward_ms": 1e3 * tf, "backward_ms": 1e3 * tbk, "backward_over_forward": tbk / tf,
            "forward_cells_steps_per_s": ncell * nsteps / tf,
            "mean_drag_coefficient": J, "dCD_dtheta": [float(v) for v in tb], "theta": ["R", "cx", "cy"],
            "gradient_workspace_mb": ws / 1e6, "poisson_tol": tol}


def serving_bench(n_req, tol, batch_cells=1 << 18):
    """The serving mix (seeded Poisson stream of 2-D cylinder and 3-D sphere cases of
    different sizes) served batched (continuous batching: one wl_step_batch per round, each
    resident's own step graph; and one wl_batch_step per round, the residents of at most
    batch_cells cells in one batched graph per dimension) and one request at a time on the
    same GPU; wall time includes admission and simulation setup in all three."""
    import numpy as np
    from paper_2304_08159_gb300 import serve

    reqs = serve.request_stream(n_req)
    warm = serve.request_stream(2, seed=1)
    serve.serve_gpu(warm, tol=tol)
    serve.serve_gpu(warm, tol=tol, batch_cells=batch_cells)
    serve.sequential_gpu(warm, tol=tol)
    stats, lat = serve.serve_gpu(reqs, tol=tol)
    bstats, blat = serve.serve_gpu(reqs, tol=tol, batch_cells=batch_cells)
    small, large = serve.class_latencies_ms(bstats)
    t_seq, cs_seq, lat_seq = serve.sequential_gpu(reqs, tol=tol)
    occ = [n for n, _, _ in stats["rounds"]]
    b = stats["cells_steps"] / stats["wall_s"]
    bb = bstats["cells_steps"] / bstats["wall_s"]
    q = cs_seq / t_seq
    nsmall = sum(1 for r in reqs if r.cells <= batch_cells)

    def pct(v, p):
        return float(np.percentile(v, p)) if v else None
    return {"requests": n_req, "mix": "seeded Poisson stream (seed 20230417, 2 per round): 2-D cylinder N^2 "
                                      "N 64-512, 3-D sphere N^3 N 32-192, R 4-24, Re 100-1000, 20-200 steps",
            "batched": {"value": b, "unit": "cell*step/s", "wall_s": stats["wall_s"],
                        "step_latency_ms_p50": float(np.percentile(lat, 50)),
                        "step_latency_ms_p99": float(np.percentile(lat, 99)),
                        "rounds": len(lat), "mean_resident": float(np.mean(occ)), "max_resident": int(max(occ)),
                        "peak_workspace_gb": stats["peak_bytes"] / 1e9},
            "small_batched": {"batch_cells": batch_cells, "small_requests": nsmall,
                              "value": bb, "unit": "cell*step/s", "wall_s": bstats["wall_s"],
                              "step_latency_ms_p50": pct(blat, 50), "step_latency_ms_p99": pct(blat, 99),
                              "small_step_latency_ms_p50": pct(small, 50), "small_step_latency_ms_p99": pct(small, 99),
                              "large_step_latency_ms_p50": pct(large, 50), "large_step_latency_ms_p99": pct(large, 99),
                              "over_sequential": bb / q,
                              "how": "requests of at most batch_cells cells step together in one batched graph per "
                                     "dimension (wl_batch_step: every kernel of the step launched once for all of "
                                     "them over a device descriptor table); the others with their own graphs"},
            "sequential": {"value": q, "unit": "cell*step/s", "wall_s": t_seq,
                           "step_latency_ms_p50": float(np.percentile(lat_seq, 50)),
                           "step_latency_ms_p99": float(np.percentile(lat_seq, 99))},
            "batched_over_sequential": b / q, "poisson_tol": tol}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="sphere512", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--prof-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--ref-steps", type=int, default=2)
    ap.add_argument("--ref-warmup", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=32)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        return run_reference(args, w, rank, ws)
    dist, rank, ws, lrank = _dist()
    try:
        return run_ours(args, w, dist, rank, ws, lrank)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
