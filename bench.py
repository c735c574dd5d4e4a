#!/usr/bin/env python
"""Benchmark of the FLA hot path on one GB300.

Workload (the 512^2 planar-jet configuration): a 512 x 512 mesh on [0,1]^2, a
Gaussian jet (centre speed 1, width 0.05) with 8 Lamb-Oseen vortices carried
by it, 256 releases of 1,024 FLA seeds at the inlet over 1,000 RK4 steps of
dt = 1e-3, St0 ~ U[0.2, 2] per release, d^2-law evaporation (delta = -0.2),
the carrier re-sampled and the kernel-regression sources deposited every 10
steps (100 deposits onto 262,144 cells), FP32 with FP64 det J.

One step = one whole run of the path over that input: 100 windows of
{carrier sample, fused 10-step advance, cell keys, radix sort, bin starts,
records, kernel-regression gather}.  The run is captured once in a CUDA graph
and replayed; the cloud is reset to its seeds (device-to-device copy) and L2 is
flushed (a 256 MB write) before each timed step, outside the step's events.

Reported: source-term cells/s (cells x deposits / step time) as the headline,
droplet-steps/s from the device's own counter, the PSI-CELL reference run
(2^24 parcels, same flow) as a separately timed leg, per-phase CUDA-event
times from an instrumented eager run, the roofline of the dominant kernel, the
end-to-end number with host buffers, and the FP64 CPU oracle on a bounded
sample as the CPU baseline.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "source-term cells/s (kernel-regression deposit, with droplet-steps/s) at rel-L2 <= 1e-4 vs FP64 oracle"
UNIT = "cells/s"
WORKLOADS = {
    # name: (description, dtype name, has PSI-CELL reference)
    "jet_vortex_2d": ("jet_vortex_2d: 512^2 cells, 262,144 FLA seeds (256 releases x 1,024), 1,000 RK4 steps, "
                      "100 deposits", "F32", True),
    "taylor_green_2d": ("taylor_green_2d: 64^2 cells, 4,096 FLA seeds, 200 RK4 steps, 20 deposits, FP64", "F64", True),
    "abc_jet_3d": ("abc_jet_3d: 128^3 cells, 2,097,152 FLA seeds in a cone, 500 RK4 steps, 50 deposits, "
                   "J-scaled anisotropic kernel", "F32", False),
}
WORKLOAD = WORKLOADS["jet_vortex_2d"][0]


def make_workload(name, with_lpt):
    from paper_2512_20829_gb300 import inputs as I
    if name == "jet_vortex_2d":
        return I.jet_vortex_2d(lpt_per_batch=65_536 if with_lpt else 0)
    if name == "taylor_green_2d":
        wl = I.taylor_green_2d()
        if not with_lpt:
            wl.lpt = None
        return wl
    return I.abc_jet_3d()

# Floating-point operations per droplet step of the fused advance, counted from the
# kernel's operation list (FMA = 2).  2D: four stages of bilinear interpolation of 6
# node values (58) and the right-hand side (28), the RK4 combinations (156), St(t)
# (13) and the window sums (20).  3D: trilinear interpolation of 12 values (217) and
# the right-hand side (78) per stage, combinations (312), St(t) and sums (40).
FLOPS_PER_STEP = {2: 533, 3: 1532}
# Operations per (cell, droplet) pair inside the truncated kernel, the paper's
# form of the weight (one ex2 per pair besides these).  2D spherical: 2 differences,
# r^2 (3), exponent (1), prefactor (1), 4 FMA sums (8).  3D spherical: 3 differences,
# r^2 (5), exponent and prefactor (2), sums (9).  3D J-scaled: 3 differences,
# P d (15), d.(P d) (5), exponent (2), sums (9).
FLOPS_PER_PAIR = {(2, 0): 15, (3, 0): 19, (2, 1): 24, (3, 1): 34}
FP64_PEAK_TFLOPS = 1.25   # GB300 FP64, per the hardware description
# DRAM bytes (read + write) of one k_gather2d_items launch from an ncu capture
# (profiles/gather2d_jet512_window81.md); None once the kernel changes.
GATHER_TRAFFIC = {
    (2, 0, False): (6245888, "ncu dram__bytes_read+write of k_gather2d_items, jet 512^2 deposit 81"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="jet_vortex_2d",
                    help="configuration to run (the headline metric is quoted on jet_vortex_2d)")
    ap.add_argument("--no-psicell", action="store_true", help="skip the PSI-CELL reference leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--clocks-dir", default=tempfile.gettempdir(),
                    help="where the nvidia-smi clock samples of the timed region are written")
    ap.add_argument("--no-variants", action="store_true", help="skip the other precision forms")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-clouds leg")
    ap.add_argument("--form", choices=["mixed", "plain", "fold", "learned"], default="mixed",
                    help="precision form of the headline path (the default is the mixed form)")
    ap.add_argument("--profile-batch", action="store_true",
                    help="one run of the 64-cloud batch with plain launches (no graph), for external profilers")
    ap.add_argument("--profile-only", action="store_true",
                    help="one eager run of the whole path, nothing else (for external profilers)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, directory: str):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(directory, f"clocks_rank{device_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(r[1] for r in rows)),
                "samples": len(rows), "reasons": reasons}


# --------------------------------------------------------------------------- GPU path

class JetPath:
    """Device buffers and the issue order of one whole run of a workload."""

    def __init__(self, ctx, wl, fla, with_fla=True, with_lpt=False, dtype=None, precision=None,
                 fold_guard=False, mlp=None):
        import torch
        self.fla, self.ctx, self.wl = fla, ctx, wl
        self.dtype = fla.F32 if dtype is None else dtype
        self.precision = fla.PREC_MIXED if precision is None else precision
        self.m = fla.mesh(wl.dim, wl.n_cells_axis)
        self.desc = fla.carrier_desc(wl.carrier)
        self.nodes = fla.nodes_buffer(self.m, self.dtype)
        self.mlp = mlp
        self.cfg = fla.deposit_cfg(wl.kernel, wl.h_min, wl.h_max, wl.window * wl.dt, wl.p, precision=self.precision,
                                   mlp=mlp)
        self.cloud = fla.DeviceCloud.from_seeds(wl.fla, wl.dim, wl.delta, wl.dt, self.dtype) if with_fla else None
        if self.cloud is not None and self.dtype == fla.F32 and self.precision == fla.PREC_MIXED and fold_guard:
            self.cloud.enable_fold()   # double-precision J, W near fold caustics
        self.lpt = fla.DeviceCloud.from_seeds(wl.lpt, wl.dim, wl.delta, wl.dt, self.dtype) if with_lpt else None
        n = max(c.n for c in (self.cloud, self.lpt) if c is not None)
        self.ws = fla.aligned_ws(fla.workspace(self.m, self.dtype, wl.kernel, n))
        self.out = fla.SourceFields(self.m, self.dtype) if with_fla else None
        self.psi = fla.PsicellFields(self.m, self.dtype) if with_lpt else None
        self.pristine = [(c.state.clone(), c.meta.clone()) for c in (self.cloud, self.lpt) if c is not None]

    def clouds(self):
        return [c for c in (self.cloud, self.lpt) if c is not None]

    def reset(self):
        for c, (s, m) in zip(self.clouds(), self.pristine):
            c.state.copy_(s)
            c.meta.copy_(m)

    def issue(self):
        """Enqueue the whole run on the current stream (capturable)."""
        fla, wl, m = self.fla, self.wl, self.m
        for s in range(0, wl.nsteps, wl.window):
            if s == 0 or not wl.carrier.steady:   # a steady carrier is sampled once per run
                fla.carrier_sample(self.ctx, self.desc, m, 0.0 if wl.carrier.steady else s * wl.dt, self.dtype,
                                   self.nodes)
            for c in self.clouds():
                fla.advance(self.ctx, c, m, self.nodes, s, wl.window, wl.dt, reset_acc=True)
            if self.cloud is not None:
                fla.deposit_sources(self.ctx, self.cloud, m, self.cfg, self.out, self.ws)
            if self.lpt is not None:
                fla.psicell(self.ctx, self.lpt, m, wl.window * wl.dt, self.psi, self.ws)


def batch_leg(ctx, fla, I, flush, steps):
    """64 clouds of uneven size and mesh, 100 steps (10 deposits) per run: the
    batched launches of fla_batch_run (one graph) against the same clouds
    issued one by one through the per-cloud calls (also one graph)."""
    import torch
    wls = I.batch_clouds()
    b = fla.Batch(ctx, wls)
    s = torch.cuda.Stream()
    windows = wls[0].nsteps // wls[0].window
    with torch.cuda.stream(s):
        b.run(windows, stream=s)            # tuning windows, then the graph
        torch.cuda.synchronize()
        b.reset(s)
        b.run(windows, stream=s)            # the graph of a whole run
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            b.reset(s)
            flush.add_(1.0)
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(s)
            b.run(windows, stream=s)
            eb.record(s)
            torch.cuda.synchronize()
            times.append(ea.elapsed_time(eb))
    batched = float(np.median(times))
    tun = b.tuning()
    del b
    torch.cuda.empty_cache()
    # the same clouds through the per-cloud calls
    paths = [JetPath(ctx, wl, fla, with_fla=True, dtype=fla.F32) for wl in wls]

    class _All:
        def __init__(self, ps):
            self.ps, self.ctx = ps, ctx

        def reset(self):
            for p in self.ps:
                p.reset()

        def issue(self):
            for p in self.ps:
                p.issue()
    allp = _All(paths)
    g, launches = capture(allp)
    ut = []
    for _ in range(steps):
        allp.reset()
        flush.add_(1.0)
        torch.cuda.synchronize()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record()
        g.replay()
        eb.record()
        torch.cuda.synchronize()
        ut.append(ea.elapsed_time(eb))
    unbatched = float(np.median(ut))
    del g, paths, allp
    torch.cuda.empty_cache()
    cells = sum(w.n_cells for w in wls)
    return {"workload": f"{len(wls)} clouds (seed 4): {sum(w.fla.n for w in wls):,} seeds, 1e3-5e5 per cloud, "
                        f"2D 32^2-256^2 spherical / 3D 32^3-64^3 J-scaled, {windows} windows of 10 steps",
            "cells": cells, "ms_per_run": round(batched, 4), "cells_per_s": cells * windows / (batched * 1e-3),
            "unbatched_ms_per_run": round(unbatched, 4), "speedup_vs_unbatched": round(unbatched / batched, 3),
            "launches_per_run": tun["launches_per_window"] * windows, "unbatched_launches_per_run": launches,
            "tuning": tun}


def capture(path):
    import torch
    path.reset()
    path.issue()                     # eager warm-up (sets kernel attributes once)
    torch.cuda.synchronize()
    path.reset()
    torch.cuda.synchronize()
    path.ctx.profile(False, reset=True)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        path.issue()
    torch.cuda.synchronize()
    launches = sum(v["launches"] for v in path.ctx.profile_read().values())
    return g, launches


def timed_replays(path, g, steps, flush, events=True):
    import torch
    times = []
    for _ in range(steps):
        path.reset()
        flush.add_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        times.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in times]


def roofline_entry(phase_name, prof, peaks, status_pairs, droplet_steps_per_run, dim, kernel, f64):
    """Roofline of the dominant phase from the instrumented run's CUDA-event times
    (one call = the phase's kernel launches for one window)."""
    p = prof[phase_name]
    calls = max(p["calls"], 1)
    ms_per_call = p["ms"] / calls
    sm_max = 2070.0
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12          # TFLOP/s at the maximum SM clock
    mufu_pairs = 152 * 16 * sm_max * 1e6                     # ex2 per second
    if phase_name == "advance":
        flops = droplet_steps_per_run * FLOPS_PER_STEP[dim] / calls
        ach = flops / (ms_per_call * 1e-3) / 1e12
        peak = FP64_PEAK_TFLOPS if f64 else fp32_peak
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "kernel": "k_advance",
                "peak_basis": ("GB300 FP64 rate (derived)" if f64 else
                               "152 SM x 128 FP32 lanes x 2 x 2070 MHz (derived, max clock)")}
    if phase_name == "gather":
        fpp = FLOPS_PER_PAIR[(dim, kernel)]
        flops = status_pairs / calls * fpp
        ach = flops / (ms_per_call * 1e-3) / 1e12
        peak = FP64_PEAK_TFLOPS if f64 else min(fp32_peak, mufu_pairs * fpp / 1e12)
        traffic = GATHER_TRAFFIC.get((dim, kernel, f64))
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": traffic[0] if traffic else None,
                "traffic_basis": traffic[1] if traffic else None,
                "kernel": "kernel-regression gather (all launches of one deposit)",
                "peak_basis": ("GB300 FP64 rate (derived)" if f64 else
                               f"min(FP32 152x128x2, MUFU ex2 152x16 per pair x {fpp} flops) at 2070 MHz (derived)")}
    # HBM-bound phases: algorithmic bytes
    return {"bound": "hbm", "achieved": None, "peak": peaks.get("hbm_gbs"), "unit": "GB/s", "frac": None,
            "traffic": None, "kernel": phase_name}


def max_over_ranks(value: float, world: int, device: str = "cuda") -> float:
    """The largest of the ranks' values (all ranks receive it); world 1 returns value."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(world: int, cells: int, deposits: int, steps: int, total_ms: float) -> float:
    """Whole-job cells/s: every rank deposits its own replica's cells each window,
    timed by the slowest rank."""
    return world * cells * deposits * steps / (total_ms * 1e-3)


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2512_20829_gb300 import fla, inputs as I

    rank, local, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    ctx = fla.Context(local)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    desc, dname, has_psi = WORKLOADS[args.workload]
    dtype = getattr(fla, dname)
    wl = make_workload(args.workload, has_psi and not args.no_psicell)
    cells = wl.n_cells
    deposits = wl.nsteps // wl.window

    form_mlp = None
    if args.form == "learned":
        form_mlp = fla.LearnedCorrection(ctx, fla.init_mlp_params(0, 0.5, zero_last=True))
    path = JetPath(ctx, wl, fla, with_fla=True, dtype=dtype,
                   precision=fla.PREC_PLAIN if args.form == "plain" else fla.PREC_MIXED,
                   fold_guard=args.form == "fold", mlp=form_mlp)
    if args.profile_batch:
        b = fla.Batch(ctx, I.batch_clouds())
        b.set_tuning(128, 4, 1)
        b.run(b.workloads[0].nsteps // b.workloads[0].window)   # legacy stream: plain launches
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_batch": True, "launches_per_window": b.tuning()["launches_per_window"]}))
        return
    if args.profile_only:
        # one eager run of the whole path (no graph), for external profilers
        path.reset()
        path.issue()
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_only": True, "workload": desc}))
        return
    g, launches_per_run = capture(path)
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        path.reset()
        g.replay()
    torch.cuda.synchronize()

    # ---------------- timed region (graph replays)
    ctx.sync_status(reset=True)
    sampler = ClockSampler(local, args.clocks_dir)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    times = timed_replays(path, g, args.steps, flush)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    st = ctx.sync_status(reset=True)
    total_ms = max_over_ranks(float(sum(times)), world)
    ms_per_step = total_ms / args.steps
    droplet_steps_per_run = st.droplet_steps / args.steps
    value = weak_value(world, cells, deposits, args.steps, total_ms)

    # ---------------- instrumented eager run: per-phase CUDA-event times
    path.reset()
    ctx.sync_status(reset=True)
    ctx.profile(True, reset=True)
    path.issue()
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False, reset=True)
    stp = ctx.sync_status(reset=True)
    dominant = max(prof, key=lambda k: prof[k]["ms"])
    roof = roofline_entry(dominant, prof, peaks, stp.pairs, droplet_steps_per_run, wl.dim, wl.kernel,
                          dtype == fla.F64)
    phases = {k: {"ms_per_run": round(v["ms"], 4), "launches_per_run": v["launches"]} for k, v in prof.items()
              if v["calls"]}

    # ---------------- end to end: pinned host seeds in, final source fields out
    host_state = path.pristine[0][0].cpu().pin_memory()
    host_meta = path.pristine[0][1].cpu().pin_memory()
    out_host = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in (path.out.s_mass, path.out.s_mom,
                                                                              path.out.dsum)]
    h2d = host_state.numel() * host_state.element_size() + host_meta.numel() * host_meta.element_size()
    d2h = sum(t.numel() * t.element_size() for t in out_host)
    e2e = []
    for k in range(max(2, args.steps // 2)):
        flush.add_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        path.cloud.state.copy_(host_state, non_blocking=True)
        path.cloud.meta.copy_(host_meta, non_blocking=True)
        g.replay()
        for dst, src in zip(out_host, (path.out.s_mass, path.out.s_mom, path.out.dsum)):
            dst.copy_(src, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        e2e.append(a.elapsed_time(b))
    e2e_ms = float(np.mean(e2e))

    # ---------------- the other precision forms of the same path, timed the same way:
    # plain single precision (det J and n in FP32) and mixed with the advance's fold guard
    precision = None
    if dtype == fla.F32 and not args.no_variants:
        variants = {}
        learned = None
        if wl.kernel == fla.KERNEL_ISO:
            # zero last layer: the same h as the plain method, so the difference is the network's cost
            learned = fla.LearnedCorrection(ctx, fla.init_mlp_params(0, 0.5, zero_last=True))
        forms = [("plain_fp32", fla.PREC_PLAIN, False, None), ("mixed_fold_guard", fla.PREC_MIXED, True, None)]
        if learned is not None:
            forms.append(("learned_tensor_core_mlp", fla.PREC_MIXED, False, learned))
        for name, prec, guard, mlp in forms:
            vp = JetPath(ctx, wl, fla, with_fla=True, dtype=dtype, precision=prec, fold_guard=guard, mlp=mlp)
            vg, _ = capture(vp)
            vg.replay()
            torch.cuda.synchronize()
            ctx.sync_status(reset=True)
            vt = timed_replays(vp, vg, 3, flush)
            vst = ctx.sync_status(reset=True)
            variants[name] = {"ms_per_step": round(float(np.mean(vt)), 4),
                              "cells_per_s": cells * deposits / (float(np.mean(vt)) * 1e-3),
                              "fold_steps_per_run": vst.fold_steps / 3}
            del vg, vp
        precision = {"headline": "mixed: FP32 trajectories and kernels, det J and n in FP64 where det J cancels",
                     "variants": variants}

    # ---------------- PSI-CELL reference leg (2^24 parcels, same flow, same windows)
    psi = None
    if not args.no_psicell and wl.lpt is not None and rank == 0:
        del g
        ppath = JetPath(ctx, wl, fla, with_fla=False, with_lpt=True, dtype=dtype)
        pg, plaunch = capture(ppath)
        pg.replay()
        torch.cuda.synchronize()
        ctx.sync_status(reset=True)
        pt = timed_replays(ppath, pg, 2, flush)
        pst = ctx.sync_status(reset=True)
        pms = float(np.mean(pt))
        psi = {"parcels": wl.lpt.n, "ms_per_run": round(pms, 3),
               "cells_per_s": cells * deposits / (pms * 1e-3),
               "parcel_steps_per_s": pst.droplet_steps / 2 / (pms * 1e-3),
               "gpu_launches_per_run": plaunch,
               "fla_speedup_vs_psicell": round(pms / ms_per_step, 2)}
        del pg, ppath

    batch = None
    if rank == 0 and not args.no_batch and args.workload == "jet_vortex_2d":
        batch = batch_leg(ctx, fla, I, flush, max(3, args.steps // 2))

    cpu = None
    if rank == 0 and not args.no_cpu and args.workload == "jet_vortex_2d":
        cpu = cpu_baseline(wl)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (f64 det J)" if dtype == fla.F32 else "f64",
            "data": "synthetic (seeded, " + args.workload + ")",
            "config": {"workload": desc, "form": args.form, "global_batch": world * wl.fla.n, "cells": cells,
                       "deposits_per_step": deposits, "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"replicas x{world} (independent clouds, no collective)"},
            "droplet_steps_per_s": world * droplet_steps_per_run * args.steps / (total_ms * 1e-3),
            "gpu_launches": launches_per_run * args.steps,
            "clocks": clocks,
            "roofline": roof,
            "phases": phases,
            "e2e": {"value": world * cells * deposits / (e2e_ms * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms},
            "forms": precision,
            "psicell_reference": psi,
            "batch": batch,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------- CPU oracle

def cpu_baseline(wl, seeds=8192, cells_a=256, cells_b=4096, track=256):
    """The FP64 oracle, single-threaded, on a bounded sample of the same workload,
    scaled to the whole run from separately timed parts:
      carrier  one node re-sample, times the number of carrier steps;
      advance  cost per droplet step from `seeds` seeds of the first release over
               two windows (their two re-samples subtracted), times the run's active
               droplet steps, counted from `track` random seeds integrated through the
               whole run with the analytic carrier;
      deposit  cell-list deposit of a cloud state of the workload's size and shape at
               cells_a and cells_b cells: fixed part (cell list and records) plus the
               per-cell slope times all cells, times the number of deposits."""
    from oracle import oracle as O
    from paper_2512_20829_gb300 import inputs as I
    rng = np.random.default_rng(0)
    n, nsteps, win = wl.fla.n, wl.nsteps, wl.window
    deposits = nsteps // win
    wall0 = time.perf_counter()
    # carrier
    t0 = time.perf_counter()
    O.carrier_nodes(wl.carrier, 0.0, wl.n_cells_axis)
    t_node = time.perf_counter() - t0
    t_car = t_node * (1 if wl.carrier.steady else deposits)
    # advance cost per droplet step
    first = np.nonzero(wl.fla.batch == 0)[0][:seeds]
    sub = I.Cloud(kind=wl.fla.kind, x0=wl.fla.x0[first], batch=wl.fla.batch[first], step_start=wl.fla.step_start,
                  St0=wl.fla.St0, n0=wl.fla.n0, h0=wl.fla.h0)
    adv = O.Advancer(wl, sub)
    st = O.initial_state(sub, wl.dim)
    t0 = time.perf_counter()
    adv.advance(st, 0, win, reset_acc=True)
    adv.advance(st, win, win, reset_acc=True)
    t_two = time.perf_counter() - t0
    per_step = max(t_two - 2 * t_node, 1e-9) / (len(first) * 2 * win)
    # active droplet steps of the whole run (fraction from tracked seeds, analytic carrier)
    idx = np.sort(rng.choice(n, track, replace=False))
    tr = I.Cloud(kind=wl.fla.kind, x0=wl.fla.x0[idx], batch=wl.fla.batch[idx], step_start=wl.fla.step_start,
                 St0=wl.fla.St0, n0=wl.fla.n0, h0=wl.fla.h0)
    adv2 = O.Advancer(wl, tr, use_mesh=False)
    st2 = O.initial_state(tr, wl.dim)
    active_steps = 0
    for s in range(0, nsteps, win):
        adv2.advance(st2, s, win, reset_acc=True)
        active_steps += win * int((st2.status == O.ACTIVE).sum())
    droplet_steps = active_steps * n / track
    # deposit: fixed + per-cell
    s_ = I.synthetic_state(2, n, wl.n_cells_axis, seed=31, band=(0.4, 0.6), h0_cells=2.0, jac_spread=0.3)
    D = O.dep_struct(wl)
    band = np.arange(int(0.4 * wl.n_cells_axis), int(0.6 * wl.n_cells_axis))
    times = []
    for c in (cells_a, cells_b):
        cells = rng.choice(band, c) * wl.n_cells_axis + rng.integers(0, wl.n_cells_axis, c)
        t0 = time.perf_counter()
        O.nw_deposit_celllist(D, s_.x, s_.J, s_.acc, s_.status, s_.batch, s_.n0, s_.h0, cells=cells)
        times.append(time.perf_counter() - t0)
    per_cell = max(times[1] - times[0], 1e-9) / (cells_b - cells_a)
    fixed = max(times[0] - per_cell * cells_a, 0.0)
    t_dep = fixed + per_cell * wl.n_cells
    t_run = t_car + per_step * droplet_steps + deposits * t_dep
    return {"value": wl.n_cells * deposits / t_run, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"carrier re-sample x{1 if wl.carrier.steady else deposits}; {len(first)} seeds x {2 * win} "
                       f"steps ({per_step * 1e6:.2f} us per droplet step) x {droplet_steps:.3g} active droplet "
                       f"steps (from {track} tracked seeds); cell-list deposit at {cells_a}/{cells_b} cells of a "
                       f"{n}-droplet state ({per_cell * 1e6:.1f} us per cell + {fixed:.2f} s fixed) x {deposits}"),
            "est_seconds_per_run": round(t_run, 1), "sample_seconds": round(time.perf_counter() - wall0, 2),
            "cpu": platform_cpu()}


def platform_cpu():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip() + f" x{os.cpu_count()}"
    except Exception:
        pass
    return f"{os.uname().machine} x{os.cpu_count()}"


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    from paper_2512_20829_gb300 import inputs as I
    wl = I.jet_vortex_2d(lpt_per_batch=0)
    per_step = []
    last = None
    for k in range(args.warmup + args.steps):
        last = cpu_baseline(wl, seeds=256, cells_a=32, cells_b=96, track=32)
        if k >= args.warmup:
            per_step.append(wl.n_cells * (wl.nsteps // wl.window) / last["value"])
    ms = 1e3 * float(np.mean(per_step))
    value = wl.n_cells * (wl.nsteps // wl.window) / (ms * 1e-3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded jet + vortices)",
            "config": {"workload": WORKLOAD, "cells": wl.n_cells},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "per step: " + last["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
