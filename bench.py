#!/usr/bin/env python
"""Benchmark of the FLA hot path on one GB300.

Headline workload (the largest single-GPU configuration): the 3D spray cone,
a 128^3 mesh on [0,1]^3, ABC flow (1, 0.7, 0.43) at wavenumber 2 pi plus a
round jet of radius 0.05, 2,097,152 FLA seeds on a volume-preserving lattice
in a cone, St0 = 1, d^2-law evaporation (delta = -0.2), 500 RK4 steps of
dt = 1e-3, the J-scaled anisotropic kernel truncated at 3 sigma, sources
deposited every 10 steps (50 deposits onto 2,097,152 cells), in the
compensated precision form (double-float trajectories and carrier, single-
precision deposit, det J in double): the form that keeps the sources within
rel-L2 1e-4 of the FP64 oracle over every cell, fold caustics included.

One step = one whole run of the path over that input: per window {carrier
sample (once for a steady carrier), fused 10-step advance, cell keys, radix
sort, bin starts, records, kernel-regression gather}.  The run is captured
once in a CUDA graph and replayed; the cloud is reset to its seeds (device-to-
device copy) and L2 is flushed (a 256 MB write) before each timed step,
outside the step's events.

Reported beside the headline: droplet-steps/s from the device's own counter;
per-phase CUDA-event times of an instrumented eager run and a roofline entry
per phase; the end-to-end number through the C-ABI with pinned host buffers;
the single-precision forms of the same workload (their cells/s and, from the
CPU-baseline leg, the rel-L2 each form reaches on the reduced configuration);
the planar-jet and Taylor-Green configurations as secondary legs (the jet with
its 2^24-parcel PSI-CELL reference); the 64-cloud batched leg; and the FP64 CPU
oracle on a bounded sample, on one host core and on all of them.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "source-term cells/s (kernel-regression deposit, with droplet-steps/s) at rel-L2 <= 1e-4 vs FP64 oracle"
UNIT = "cells/s"
# name: (description, headline form)
WORKLOADS = {
    "abc_jet_3d": ("abc_jet_3d: 128^3 cells, 2,097,152 FLA seeds in a cone, ABC + round jet, 500 RK4 steps, "
                   "50 deposits, J-scaled anisotropic kernel (3 sigma)", "compensated"),
    "jet_vortex_2d": ("jet_vortex_2d: 512^2 cells, 262,144 FLA seeds (256 releases x 1,024), 1,000 RK4 steps, "
                      "100 deposits, spherical kernel", "compensated"),
    "taylor_green_2d": ("taylor_green_2d: 64^2 cells, 4,096 FLA seeds, 200 RK4 steps, 20 deposits, spherical kernel",
                        "fp64"),
}
# The precision forms: (cloud dtype name, deposit precision, fold guard, learned correction)
FORMS = {
    "compensated": ("F32X2", "PREC_MIXED", False, False),
    "mixed": ("F32", "PREC_MIXED", False, False),
    "plain": ("F32", "PREC_PLAIN", False, False),
    "fold": ("F32", "PREC_MIXED", True, False),
    "learned": ("F32", "PREC_MIXED", False, True),
    "fp64": ("F64", "PREC_MIXED", False, False),
}
FORM_TEXT = {
    "compensated": "double-float trajectories and carrier nodes, single-precision deposit, det J and n in FP64",
    "mixed": "FP32 trajectories and kernels, det J and n in FP64 where det J cancels",
    "plain": "FP32 throughout",
    "fold": "mixed + FP64 J, W while |det J| < 1e-2",
    "learned": "mixed + tensor-core bandwidth MLP fused into the records (zero last layer: same h)",
    "fp64": "FP64 throughout",
}


def make_workload(name, with_lpt=False, scale=1):
    from paper_2512_20829_gb300 import inputs as I
    if name == "jet_vortex_2d":
        return I.jet_vortex_2d(scale=scale, lpt_per_batch=65_536 if with_lpt else 0)
    if name == "taylor_green_2d":
        wl = I.taylor_green_2d(scale=scale)
        if not with_lpt:
            wl.lpt = None
        return wl
    return I.abc_jet_3d(scale=scale)


# Floating-point operations per droplet step of the advance's algorithm, counted from the
# single-precision kernel's operation list (FMA = 2).  2D: four stages of bilinear
# interpolation of 6 node values (58) and the right-hand side (28), the RK4 combinations
# (156), St(t) (13) and the window sums (20).  3D: trilinear interpolation of 12 values
# (217) and the right-hand side (78) per stage, combinations (312), St(t) and sums (40).
# The compensated form performs the same algorithm in double-float arithmetic (about
# 6.5 FP32 instructions per algorithmic operation); its roofline is taken on these
# algorithmic operations against the FP32 peak.
FLOPS_PER_STEP = {2: 533, 3: 1532}
# Operations per (cell, droplet) pair inside the truncated kernel, the paper's form of the
# weight (one ex2 per pair besides these).  2D spherical: 2 differences, r^2 (3), exponent
# (1), prefactor (1), 4 FMA sums (8).  3D spherical: 3 differences, r^2 (5), exponent and
# prefactor (2), sums (9).  3D J-scaled: 3 differences, P d (15), d.(P d) (5), exponent
# (2), sums (9).
FLOPS_PER_PAIR = {(2, 0): 15, (3, 0): 19, (2, 1): 24, (3, 1): 34}
FP64_PEAK_TFLOPS = 1.25   # GB300 FP64, per the hardware description
SM_COUNT, FP32_LANES, MUFU_LANES, SM_MAX_MHZ = 152, 128, 16, 2070.0
# Carrier: double-precision operations per node, counted from the evaluation (the
# double-float form samples in FP64; a steady carrier is sampled once per run).
# Jet + 8 vortices x 3 periodic images: ~22 per image (far field, no exponential) + jet.
# ABC + round jet: ~40 plus six sin/cos and one exponential.
CARRIER_FLOPS_PER_NODE = {"jet_vortex_2d": 24 * 22 + 12, "abc_jet_3d": 60, "taylor_green_2d": 30}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="abc_jet_3d",
                    help="configuration to run (the headline is the largest single-GPU one, abc_jet_3d)")
    ap.add_argument("--form", choices=sorted(FORMS), default=None,
                    help="precision form of the headline path (default: the workload's form that meets 1e-4)")
    ap.add_argument("--no-psicell", action="store_true", help="skip the PSI-CELL reference leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-variants", action="store_true", help="skip the other precision forms")
    ap.add_argument("--no-secondary", action="store_true", help="skip the other configurations")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-clouds leg")
    ap.add_argument("--clocks-dir", default=tempfile.gettempdir(),
                    help="where the nvidia-smi clock samples of the timed region are written")
    ap.add_argument("--profile-batch", action="store_true",
                    help="one run of the 64-cloud batch with plain launches (no graph), for external profilers")
    ap.add_argument("--batch-persistent", action="store_true",
                    help="with --profile-batch: the windows as the persistent kernel")
    ap.add_argument("--profile-only", action="store_true",
                    help="one eager run of the whole path, nothing else (for external profilers)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    def __init__(self, device_index: int, directory: str):
        self.dev = device_index
        self.path = os.path.join(directory, f"bench_clocks_{os.getpid()}.csv")
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for name, v in zip(names, p[3:7]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(np.max(smax)), "samples": len(sm),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- GPU path

class RunPath:
    """Device buffers and the issue order of one whole run of a workload."""

    def __init__(self, ctx, wl, fla, form, with_fla=True, with_lpt=False, parcel_deposit="psicell", ordered=True):
        dname, pname, fold_guard, learned = FORMS[form]
        self.ordered = ordered
        self.parcel_deposit = fla.psicell if parcel_deposit == "psicell" else fla.cic
        self.fla, self.ctx, self.wl, self.form = fla, ctx, wl, form
        self.dtype = getattr(fla, dname)
        self.precision = getattr(fla, pname)
        self.m = fla.mesh(wl.dim, wl.n_cells_axis)
        self.desc = fla.carrier_desc(wl.carrier)
        self.nodes = fla.nodes_buffer(self.m, self.dtype)
        self.mlp = fla.LearnedCorrection(ctx, fla.init_mlp_params(0, 0.5, zero_last=True)) if learned else None
        self.cfg = fla.deposit_cfg(wl.kernel, wl.h_min, wl.h_max, wl.window * wl.dt, wl.p, precision=self.precision,
                                   mlp=self.mlp)
        self.cloud = fla.DeviceCloud.from_seeds(wl.fla, wl.dim, wl.delta, wl.dt, self.dtype) if with_fla else None
        if self.cloud is not None and fold_guard:
            self.cloud.enable_fold()   # double-precision J, W near fold caustics
        ldt = fla.F64 if self.dtype == fla.F64 else fla.F32
        self.lpt = fla.DeviceCloud.from_seeds(wl.lpt, wl.dim, wl.delta, wl.dt, ldt) if with_lpt else None
        n = max(c.n for c in (self.cloud, self.lpt) if c is not None)
        self.ws = fla.aligned_ws(fla.workspace(self.m, self.dtype, wl.kernel, n))
        self.out = fla.SourceFields(self.m, self.dtype) if with_fla else None
        self.psi = fla.PsicellFields(self.m, ldt) if with_lpt else None
        self.lnodes = fla.nodes_buffer(self.m, ldt) if (with_lpt and ldt != self.dtype) else None
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
        binned = None   # the cloud whose cell-sorted order the workspace holds

        def order(c):
            return fla.workspace_order(self.ws, m, c.n) if self.ordered and binned is c else None

        for s in range(0, wl.nsteps, wl.window):
            if s == 0 or not wl.carrier.steady:   # a steady carrier is sampled once per run
                t = 0.0 if wl.carrier.steady else s * wl.dt
                if self.cloud is not None:
                    fla.carrier_sample(self.ctx, self.desc, m, t, self.dtype, self.nodes)
                if self.lnodes is not None or (self.cloud is None and self.lpt is not None):
                    ln = self.lnodes if self.lnodes is not None else self.nodes
                    fla.carrier_sample(self.ctx, self.desc, m, t, self.lpt.dtype, ln)
            if self.cloud is not None:
                fla.advance(self.ctx, self.cloud, m, self.nodes, s, wl.window, wl.dt, reset_acc=True,
                            order=order(self.cloud))
            if self.lpt is not None:
                ln = self.lnodes if self.lnodes is not None else self.nodes
                fla.advance(self.ctx, self.lpt, m, ln, s, wl.window, wl.dt, reset_acc=True, order=order(self.lpt))
            if self.cloud is not None:
                fla.deposit_sources(self.ctx, self.cloud, m, self.cfg, self.out, self.ws)
                binned = self.cloud
            if self.lpt is not None:
                self.parcel_deposit(self.ctx, self.lpt, m, wl.window * wl.dt, self.psi, self.ws)
                binned = self.lpt


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


def timed_replays(path, g, steps, flush):
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


def instrumented_run(path):
    """One eager run with per-phase CUDA events; returns the phase table and the
    device counters of that run."""
    import torch
    ctx = path.ctx
    path.reset()
    torch.cuda.synchronize()
    ctx.sync_status(reset=True)
    ctx.profile(True, reset=True)
    path.issue()
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False, reset=True)
    st = ctx.sync_status(reset=True)
    return prof, st


# --------------------------------------------------------------------------- rooflines

def source_sha(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2512_20829_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel_key):
    """DRAM bytes per full-size launch from profiles/traffic.json, if that figure was
    taken from the kernel's current source (the file records the source hash of the
    translation units it was measured on); None otherwise."""
    try:
        tab = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except Exception:
        return None, None
    e = tab.get(kernel_key)
    if not e:
        return None, None
    if e.get("source_sha") != source_sha(*e["sources"]):
        return None, f"stale: {kernel_key} changed since the capture"
    return e["bytes_per_launch"], e["basis"]


def rooflines(prof, st, wl, form, peaks, clocks):
    """One entry per phase: achieved algorithmic work per launch over the phase's
    average launch time (CUDA events), against the binding peak."""
    dim, kernel = wl.dim, wl.kernel
    f64 = form == "fp64"
    sm = SM_MAX_MHZ
    fp32_peak = SM_COUNT * FP32_LANES * 2 * sm * 1e6 / 1e12           # TFLOP/s
    mufu_pairs = SM_COUNT * MUFU_LANES * sm * 1e6                      # ex2 per second
    hbm = peaks.get("hbm_gbs")
    out = {}
    deposits = max(prof["records"]["calls"], 1)
    binned = st.deposited / deposits                                    # droplets binned per deposit
    n = wl.fla.n
    nn = wl.n_cells_axis + 1
    nodes = nn ** dim
    planes = (2 * dim + 2 * dim * dim + 1 + dim + 3) // 4
    elem = 8 if f64 else 4
    for name, p in prof.items():
        if not p["calls"] or p["ms"] <= 0:
            continue
        per_call = p["ms"] / p["calls"]
        e = {"ms_per_run": round(p["ms"], 4), "launches_per_run": p["launches"]}
        if name == "advance":
            flops = st.droplet_steps * FLOPS_PER_STEP[dim] / p["calls"]
            ach = flops / (per_call * 1e-3) / 1e12
            peak = FP64_PEAK_TFLOPS if f64 else fp32_peak
            e.update(bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                     work=f"{FLOPS_PER_STEP[dim]} algorithmic flop per droplet step x "
                          f"{st.droplet_steps / p['calls']:.4g} droplet steps per launch")
        elif name == "gather":
            fpp = FLOPS_PER_PAIR[(dim, kernel)]
            flops = st.pairs / p["calls"] * fpp
            ach = flops / (per_call * 1e-3) / 1e12
            peak = FP64_PEAK_TFLOPS if f64 else min(fp32_peak, mufu_pairs * fpp / 1e12)
            e.update(bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                     work=f"{fpp} flop per pair inside the truncation x {st.pairs / p['calls']:.4g} pairs per deposit")
        elif name == "carrier":
            per_node = next((v for k, v in CARRIER_FLOPS_PER_NODE.items() if wl.name.startswith(k)), 40)
            flops = per_node * nodes
            ach = flops / (per_call * 1e-3) / 1e12
            fp64_eval = form in ("compensated", "fp64")
            peak = FP64_PEAK_TFLOPS if fp64_eval else fp32_peak
            e.update(bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                     work=f"analytic carrier, {flops / nodes:.0f} flop per node x {nodes} nodes "
                          f"({'FP64' if fp64_eval else 'FP32'} evaluation)")
        else:
            # HBM phases: algorithmic bytes (each value moved once)
            if name == "sort":
                # keys, sort and bin starts (one kernel): position plane and meta read,
                # sorted keys and permutation written, bin starts written
                byts = n * (16 + 4 + 8) + wl.n_cells * 4
            elif name == "bins":
                byts = binned * 4 + wl.n_cells * 4            # sorted keys read, bin starts written
            elif name == "records":
                rec = 32 if (dim, kernel) == (2, 0) else (64 if (dim, kernel) == (3, 1) else 48)
                lo = (2 if dim == 3 else 1) * 16 if form == "compensated" else 0   # J low parts
                byts = binned * (planes * 16 * (2 if f64 else 1) + lo + 8 + rec)
            elif name == "psicell":
                byts = n * 20 + wl.n_cells * (4 + 4 * (1 + dim))
            else:
                continue
            gbs = byts / (per_call * 1e-3) / 1e9
            e.update(bound="hbm", achieved=gbs, peak=hbm, unit="GB/s", frac=gbs / hbm if hbm else None,
                     work=f"{byts / 1e6:.4g} MB algorithmic per call")
        out[name] = e
    return out


# --------------------------------------------------------------------------- legs

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


def time_form(ctx, fla, wl, form, flush, reps=3, with_lpt=False, with_fla=True, parcel_deposit="psicell"):
    """Graph-replayed whole runs of one form; median ms, device counters per run."""
    import torch
    p = RunPath(ctx, wl, fla, form, with_fla=with_fla, with_lpt=with_lpt, parcel_deposit=parcel_deposit)
    g, launches = capture(p)
    g.replay()
    torch.cuda.synchronize()
    ctx.sync_status(reset=True)
    t = timed_replays(p, g, reps, flush)
    st = ctx.sync_status(reset=True)
    ms = float(np.median(t))
    res = {"ms_per_run": round(ms, 4), "launches_per_run": launches,
           "droplet_steps_per_run": st.droplet_steps / reps}
    del g
    return p, ms, res


def reduced_outputs(ctx, fla, wl_small, forms):
    """Final sources of each form on the reduced configuration (the CPU baseline's sample)."""
    import torch
    outs = {}
    for form in forms:
        p = RunPath(ctx, wl_small, fla, form)
        p.reset()
        p.issue()
        torch.cuda.synchronize()
        outs[form] = (p.out.s_mass.double().cpu().numpy(), p.out.s_mom.double().cpu().numpy().T,
                      p.out.dsum.double().cpu().numpy())
        del p
    return outs


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
    tun.update(b.mode())
    # each window form timed the same way: one persistent kernel per window,
    # and the launch per phase and group
    forms = {}
    for name, mode in (("persistent", fla.BATCH_PERSISTENT), ("launches", fla.BATCH_LAUNCHES)):
        b.set_mode(mode)
        with torch.cuda.stream(s):
            b.reset(s)
            b.run(windows, stream=s)
            torch.cuda.synchronize()
            ft = []
            for _ in range(steps):
                b.reset(s)
                flush.add_(1.0)
                ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ea.record(s)
                b.run(windows, stream=s)
                eb.record(s)
                torch.cuda.synchronize()
                ft.append(ea.elapsed_time(eb))
        forms[name] = {"ms_per_run": round(float(np.median(ft)), 4),
                       "launches_per_run": b.tuning()["launches_per_window"] * windows}
    del b
    torch.cuda.empty_cache()
    # the same clouds through the per-cloud calls
    paths = [RunPath(ctx, wl, fla, "mixed") for wl in wls]

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
    ut = timed_replays(allp, g, steps, flush)
    unbatched = float(np.median(ut))
    del g, paths, allp
    torch.cuda.empty_cache()
    cells = sum(w.n_cells for w in wls)
    return {"workload": f"{len(wls)} clouds (seed 4): {sum(w.fla.n for w in wls):,} seeds, 1e3-5e5 per cloud, "
                        f"2D 32^2-256^2 spherical / 3D 32^3-64^3 J-scaled, {windows} windows of 10 steps, mixed form",
            "cells": cells, "ms_per_run": round(batched, 4), "cells_per_s": cells * windows / (batched * 1e-3),
            "unbatched_ms_per_run": round(unbatched, 4), "speedup_vs_unbatched": round(unbatched / batched, 3),
            "launches_per_run": tun["launches_per_window"] * windows, "unbatched_launches_per_run": launches,
            "tuning": tun, "window_forms": forms}


def two_way_leg(ctx, fla, I, flush, steps):
    """Two-way coupling (App. B) on the periodic Taylor-Green carrier: per
    window the carrier's node values, the fused 10-step advance, the
    kernel-regression deposit, and 10 carrier steps with the sources; one
    graph per run (droplets in the mixed form, the carrier in double)."""
    import torch
    case = I.two_way_taylor_green()
    wl = case.wl
    n_windows = wl.nsteps // wl.window

    class _Path:
        def __init__(self, carrier_only=False):
            self.ctx = ctx
            self.ns = fla.NavierStokes(ctx, wl.n_cells_axis, case.nu, case.diff, wl.dt, case.omega0,
                                       mean_u=case.mean_u)
            self.tw = fla.TwoWay(ctx, wl, self.ns, dtype=fla.F32)
            self.carrier_only = carrier_only

        def reset(self):
            self.tw.reset()

        def issue(self):
            if self.carrier_only:
                for _ in range(n_windows):
                    self.ns.nodes(fla.F32, self.tw.nodes)
                    self.ns.step(wl.window, self.tw.out)
            else:
                self.tw.run(n_windows)

    out = {}
    for name, only in (("coupled", False), ("carrier", True)):
        path = _Path(only)
        g, launches = capture(path)
        t = timed_replays(path, g, steps, flush)
        out[name] = (float(np.median(t)), launches)
        del g, path
        torch.cuda.empty_cache()
    ms = out["coupled"][0]
    return {"workload": f"{wl.name}: periodic carrier Re = 1000, vapour D = 1e-3, {wl.nsteps} steps, "
                        f"{n_windows} deposits, mixed-form droplets, double-precision carrier",
            "ms_per_run": round(ms, 4), "carrier_ms_per_run": round(out["carrier"][0], 4),
            "cells_per_s": wl.n_cells * n_windows / (ms * 1e-3),
            "carrier_steps_per_s": wl.nsteps / (out["carrier"][0] * 1e-3)}


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
    desc, default_form = WORKLOADS[args.workload]
    form = args.form or default_form
    wl = make_workload(args.workload)
    cells = wl.n_cells
    deposits = wl.nsteps // wl.window

    if args.profile_batch:
        b = fla.Batch(ctx, I.batch_clouds())
        b.set_tuning(128, 4, 1)
        if args.batch_persistent:
            b.set_mode(fla.BATCH_PERSISTENT)
        b.run(b.workloads[0].nsteps // b.workloads[0].window)   # legacy stream: plain launches
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_batch": True, "launches_per_window": b.tuning()["launches_per_window"]}))
        return
    path = RunPath(ctx, wl, fla, form)
    if args.profile_only:
        # one eager run of the whole path (no graph), for external profilers
        path.reset()
        path.issue()
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_only": True, "workload": desc, "form": form}))
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

    # ---------------- instrumented eager run: per-phase CUDA-event times and rooflines
    prof, stp = instrumented_run(path)
    roofs = rooflines(prof, stp, wl, form, peaks, clocks)
    dominant = max(roofs, key=lambda k: roofs[k]["ms_per_run"])
    roof = {k: roofs[dominant][k] for k in ("bound", "achieved", "peak", "unit", "frac")}
    dom_key = {"advance": "advance_x2" if form == "compensated" else "advance", "gather": "gather"}.get(dominant,
                                                                                                     dominant)
    traffic, basis = measured_traffic(f"{dom_key}:{args.workload}")
    roof.update(traffic=traffic, traffic_basis=basis, kernel=dominant,
                peak_basis=("measured HBM copy (MEASURED_PEAKS.json)" if roof["bound"] == "hbm" else
                            "152 SM x 128 FP32 lanes x 2 x 2070 MHz (derived, max clock)"))

    # ---------------- end to end: pinned host seeds in, final source fields out
    host_state = path.pristine[0][0].cpu().pin_memory()
    host_meta = path.pristine[0][1].cpu().pin_memory()
    out_host = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in (path.out.s_mass, path.out.s_mom,
                                                                              path.out.dsum)]
    h2d = host_state.numel() * host_state.element_size() + host_meta.numel() * host_meta.element_size()
    d2h = sum(t.numel() * t.element_size() for t in out_host)
    e2e = []
    for _ in range(max(2, args.steps // 2)):
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
    del g, path
    torch.cuda.empty_cache()

    # ---------------- the other precision forms of the same workload
    variants = {}
    if rank == 0 and not args.no_variants and form != "fp64":
        names = ["compensated", "mixed", "plain"]
        if wl.dim == 2 and wl.kernel == fla.KERNEL_ISO:
            names += ["fold", "learned"]
        for name in names:
            if name == form:
                continue
            p, ms, res = time_form(ctx, fla, wl, name, flush)
            res.update(form=FORM_TEXT[name], cells_per_s=cells * deposits / (ms * 1e-3))
            variants[name] = res
            del p
            torch.cuda.empty_cache()

    # ---------------- the other configurations
    secondary = {}
    if rank == 0 and not args.no_secondary:
        for wname in WORKLOADS:
            if wname == args.workload:
                continue
            w2 = make_workload(wname, with_lpt=(wname == "jet_vortex_2d" and not args.no_psicell))
            f2 = WORKLOADS[wname][1]
            leg = {"workload": WORKLOADS[wname][0], "forms": {}}
            names = [f2, "mixed"] if f2 != "fp64" else [f2]
            if wname == "jet_vortex_2d":
                names.append("learned")   # network with a zero last layer: the plain supports, the network's cost
            for name in names:
                p, ms, res = time_form(ctx, fla, w2, name, flush)
                pr, sp = instrumented_run(p)
                res.update(form=FORM_TEXT[name], cells_per_s=w2.n_cells * (w2.nsteps // w2.window) / (ms * 1e-3),
                           phases={k: round(v["ms"], 4) for k, v in pr.items() if v["calls"]})
                if name == f2:
                    res["rooflines"] = rooflines(pr, sp, w2, name, peaks, clocks)
                leg["forms"][name] = res
                del p
                torch.cuda.empty_cache()
            if wname == "jet_vortex_2d":
                # the plain method at four times the seeds, the seeding whose error the
                # learned form is compared with (tests/test_gpu_learn_gain.py)
                w4 = I.jet_vortex_2d(seeding=2, lpt_per_batch=0)
                p4, ms4, res4 = time_form(ctx, fla, w4, "mixed", flush, reps=2)
                leg["mixed_4x_seeds"] = {"seeds": w4.fla.n, "ms_per_run": round(ms4, 4),
                                         "cells_per_s": w4.n_cells * (w4.nsteps // w4.window) / (ms4 * 1e-3)}
                del p4
                torch.cuda.empty_cache()
            if w2.lpt is not None:
                pp, pms, pres = time_form(ctx, fla, w2, "mixed", flush, reps=2, with_lpt=True, with_fla=False)
                leg["psicell_reference"] = {
                    "parcels": w2.lpt.n, "ms_per_run": round(pms, 3),
                    "cells_per_s": w2.n_cells * (w2.nsteps // w2.window) / (pms * 1e-3),
                    "parcel_steps_per_s": pres["droplet_steps_per_run"] / (pms * 1e-3),
                    "gpu_launches_per_run": pres["launches_per_run"],
                    "fla_speedup_vs_psicell": round(pms / leg["forms"][f2]["ms_per_run"], 2)}
                del pp
                torch.cuda.empty_cache()
                # Cloud-In-Cell on the same parcels (the paper's C^1 alternative to PSI-CELL)
                cp, cms, cres = time_form(ctx, fla, w2, "mixed", flush, reps=2, with_lpt=True, with_fla=False,
                                          parcel_deposit="cic")
                leg["cic_reference"] = {
                    "parcels": w2.lpt.n, "ms_per_run": round(cms, 3),
                    "cells_per_s": w2.n_cells * (w2.nsteps // w2.window) / (cms * 1e-3),
                    "gpu_launches_per_run": cres["launches_per_run"]}
                del cp
                torch.cuda.empty_cache()
            secondary[wname] = leg

    batch = None
    if rank == 0 and not args.no_batch:
        batch = batch_leg(ctx, fla, I, flush, 3)
    two_way = None
    if rank == 0 and not args.no_secondary:
        two_way = two_way_leg(ctx, fla, I, flush, 3)

    cpu, forms_error = None, None
    if rank == 0 and not args.no_cpu:
        cpu, ref_src, wl_small = cpu_baseline(args.workload, wl, droplet_steps_per_run)
        gforms = [form] + [f for f in variants if f not in ("learned",)]
        outs = reduced_outputs(ctx, fla, wl_small, gforms)
        forms_error = {f: all_cell_errors(outs[f], ref_src, wl_small.dim) for f in gforms}
        forms_error["basis"] = (f"all-cell rel-L2 of each form's final sources vs the FP64 oracle on {wl_small.name} "
                                f"({wl_small.nsteps} steps), the CPU baseline's sample")
        if form in forms_error and form in ("compensated", "fp64"):
            cpu["tolerance_met"] = all(v <= 1e-4 for v in forms_error[form].values())

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"compensated": "f32x2 (double-float) advance, f32 deposit, f64 det J", "fp64": "f64",
                      "plain": "f32"}.get(form, "f32 (f64 det J)"),
            "data": "synthetic (seeded, " + args.workload + ")",
            "config": {"workload": desc, "form": form, "form_text": FORM_TEXT[form], "global_batch": world * wl.fla.n,
                       "cells": cells, "deposits_per_step": deposits, "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"replicas x{world} (independent clouds, no collective)"},
            "droplet_steps_per_s": world * droplet_steps_per_run * args.steps / (total_ms * 1e-3),
            "gpu_launches": launches_per_run * args.steps,
            "clocks": clocks,
            "roofline": roof,
            "rooflines": roofs,
            "e2e": {"value": world * cells * deposits / (e2e_ms * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms},
            "forms": {"headline": form, "variants": variants, "rel_l2_all_cells": forms_error},
            "secondary": secondary,
            "batch": batch,
            "two_way": two_way,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def all_cell_errors(g, ref, dim):
    gm, gv, gd = g
    om, ov, od = ref
    out = {}

    def rl2(a, b):
        nb = np.linalg.norm(b)
        return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))
    out["S_mass"] = rl2(gm, om)
    for c in range(dim):
        out[f"S_mom_{'xyz'[c]}"] = rl2(gv[:, c], ov[:, c])
    out["D"] = rl2(gd, od)
    return out


# --------------------------------------------------------------------------- CPU oracle

def oracle_sample(wl_small, threads, nsteps=None):
    """The FP64 oracle on a reduced configuration with `threads` host threads:
    carrier sampling, the advance over `nsteps` steps (window by window), and the
    cell-list deposit at the end.  Returns timings, active droplet steps and the
    final sources."""
    from oracle import oracle as O
    O.set_threads(threads)
    nsteps = wl_small.nsteps if nsteps is None else nsteps
    t0 = time.perf_counter()
    O.carrier_nodes(wl_small.carrier, 0.0, wl_small.n_cells_axis)
    t_car = time.perf_counter() - t0
    adv = O.Advancer(wl_small, wl_small.fla)
    st = O.initial_state(wl_small.fla, wl_small.dim)
    ds = 0
    t0 = time.perf_counter()
    s = 0
    while s < nsteps:
        k = min(wl_small.window, nsteps - s)
        adv.advance(st, s, k, reset_acc=True)
        ds += k * int((st.status == O.ACTIVE).sum())
        s += k
    t_adv = time.perf_counter() - t0
    D = O.dep_struct(wl_small)
    t0 = time.perf_counter()
    src = O.nw_deposit_celllist(D, st.x, st.J, st.acc, st.status, st.batch, wl_small.fla.n0, wl_small.fla.h0)
    t_dep = time.perf_counter() - t0
    return {"t_car": t_car, "t_adv": t_adv, "t_dep": t_dep, "droplet_steps": ds, "steps": nsteps,
            "carrier_samples": (1 if wl_small.carrier.steady else -(-nsteps // wl_small.window)),
            "state": st}, src


def oracle_deposit_seconds(wl_small, st, threads):
    """Time of the oracle's cell-list deposit of a given state on `threads` threads."""
    from oracle import oracle as O
    O.set_threads(threads)
    D = O.dep_struct(wl_small)
    t0 = time.perf_counter()
    O.nw_deposit_celllist(D, st.x, st.J, st.acc, st.status, st.batch, wl_small.fla.n0, wl_small.fla.h0)
    return time.perf_counter() - t0


def oracle_run_seconds(smp, wl_small, wl, full_droplet_steps):
    """Time of the whole configuration at the oracle's measured unit costs: per node
    sample, per droplet step, per deposited cell (the reduced configuration keeps the
    seeding density per cell, so the deposit's candidates per cell match)."""
    nodes_s = (wl_small.n_cells_axis + 1) ** wl_small.dim
    nodes = (wl.n_cells_axis + 1) ** wl.dim
    per_node = smp["t_car"] / nodes_s
    # the carrier time inside the advance (re-samples of an unsteady carrier) is removed
    adv_only = max(smp["t_adv"] - per_node * nodes_s * max(smp["carrier_samples"] - 1, 0), 1e-9)
    per_ds = adv_only / max(smp["droplet_steps"], 1)
    per_cell = smp["t_dep"] / wl_small.n_cells
    samples = 1 if wl.carrier.steady else wl.nsteps // wl.window
    deposits = wl.nsteps // wl.window
    t = per_node * nodes * samples + per_ds * full_droplet_steps + per_cell * wl.n_cells * deposits
    return t, per_ds, per_cell, per_node


def cpu_baseline(name, wl, gpu_droplet_steps=None):
    """The FP64 oracle, as it stands, on the host cores, on the reduced
    configuration of the same workload (scale 4: 1/64 of the seeds and cells in
    3D, 1/16 in 2D): all threads over the whole reduced run, one thread over its
    first windows; both scaled to the full configuration by their measured unit
    costs.  Returns the baseline entry, the reduced run's sources and workload."""
    wall0 = time.perf_counter()
    wl_small = make_workload(name, scale=4)
    nthreads = os.cpu_count() or 1
    from oracle import oracle as O
    O.build()
    smp_all, src = oracle_sample(wl_small, nthreads)
    # the full run's active droplet steps: the reduced run's per seed and step, times the full seeds
    full_ds = smp_all["droplet_steps"] * wl.fla.n / wl_small.fla.n
    t_all, per_ds_all, per_cell_all, _ = oracle_run_seconds(smp_all, wl_small, wl, full_ds)
    one_steps = max(wl_small.window, min(wl_small.nsteps, 60 if wl.dim == 3 else 200))
    smp_one, _ = oracle_sample(wl_small, 1, nsteps=one_steps)
    # the one-thread deposit is timed on the same end-of-run state as the all-thread one
    smp_one["t_dep"] = oracle_deposit_seconds(wl_small, smp_all["state"], 1)
    t_one, per_ds_one, per_cell_one, _ = oracle_run_seconds(smp_one, wl_small, wl, full_ds)
    O.set_threads(nthreads)
    deposits = wl.nsteps // wl.window
    entry = {"value": wl.n_cells * deposits / t_all, "unit": UNIT, "cores": nthreads, "kind": "oracle",
             "sample": (f"{wl_small.name}: {wl_small.nsteps} steps on {nthreads} threads "
                        f"({per_ds_all * 1e6:.3f} us per droplet step, {per_cell_all * 1e6:.1f} us per cell), "
                        f"scaled to {wl.fla.n} seeds x {full_ds / wl.fla.n:.1f} active steps and "
                        f"{wl.n_cells} cells x {deposits} deposits"),
             "est_seconds_per_run": round(t_all, 1),
             "single_thread": {"value": wl.n_cells * deposits / t_one, "unit": UNIT, "cores": 1,
                               "sample": (f"{wl_small.name}: first {one_steps} steps and the end-of-run deposit "
                                          f"on 1 thread ({per_ds_one * 1e6:.3f} us per droplet step, "
                                          f"{per_cell_one * 1e6:.1f} us per cell), scaled the same way"),
                               "est_seconds_per_run": round(t_one, 1)},
             "sample_seconds": round(time.perf_counter() - wall0, 2), "cpu": platform_cpu()}
    if gpu_droplet_steps:
        entry["full_run_active_droplet_steps"] = {"scaled_from_sample": full_ds, "gpu_counter": gpu_droplet_steps}
    return entry, src, wl_small


def platform_cpu():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip() + f" x{os.cpu_count()}"
    except Exception:
        pass
    return f"{os.uname().machine} x{os.cpu_count()}"


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores (all of them), each step
    a bounded sample of the workload (the reduced configuration's first windows and
    its end-of-run deposit), scaled to the whole configuration."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    name = args.workload
    desc, _ = WORKLOADS[name]
    wl = make_workload(name)
    wl_small = make_workload(name, scale=4)
    O.build()
    nthreads = os.cpu_count() or 1
    steps_sample = max(wl_small.window, min(wl_small.nsteps, 100 if wl.dim == 3 else 300))
    # active droplet steps of the full run from one pass over the whole reduced run
    smp_full, _ = oracle_sample(wl_small, nthreads)
    full_ds = smp_full["droplet_steps"] * wl.fla.n / wl_small.fla.n
    per_step = []
    for k in range(args.warmup + args.steps):
        smp, _ = oracle_sample(wl_small, nthreads, nsteps=steps_sample)
        t, per_ds, per_cell, _ = oracle_run_seconds(smp, wl_small, wl, full_ds)
        if k >= args.warmup:
            per_step.append(t)
    ms = 1e3 * float(np.mean(per_step))
    deposits = wl.nsteps // wl.window
    value = wl.n_cells * deposits / (ms * 1e-3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded, " + name + ")",
            "config": {"workload": desc, "cells": wl.n_cells, "deposits_per_step": deposits},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": (f"per step: {wl_small.name}, first {steps_sample} steps and their deposit "
                                        f"on {nthreads} threads ({per_ds * 1e6:.3f} us per droplet step, "
                                        f"{per_cell * 1e6:.1f} us per cell), scaled to the whole configuration")},
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
