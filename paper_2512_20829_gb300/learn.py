"""Training and evaluation of the learned bandwidth correction (the paper has no
counterpart).  Orchestration only: every deposit, gradient and update runs in
the CUDA library through fla.py.

A sample is one sparse-seeded cloud state at a deposit time together with the
sources of a densely seeded cloud (64 times the seeds) of the same flow at the
same time and the same kernel scale (the target).  The loss of fla_learn_grad is the mean over the source components
of ||S - T||^2 / ||T||^2 at the sample's training cells.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fla
from . import inputs as I


@dataclass
class Sample:
    cloud: "fla.DeviceCloud"      # sparse cloud state at the deposit (a private copy)
    m: "fla.Mesh"
    wl: I.Workload
    target: np.ndarray            # (n_cells, 1 + dim): dense sources, mass then momentum
    covered: np.ndarray           # cells where the dense reference has D > 0, away from fold caustics
    all_covered: np.ndarray       # cells where the dense reference has D > 0


TAU_CAUSTIC = 1e-2


def caustic_cells(cloud: "fla.DeviceCloud", wl: I.Workload) -> np.ndarray:
    """Cells within the largest kernel support (3 h_max) of a droplet with
    |det J| < 1e-2.  Near a fold caustic n = n0/|det J| is singular (Eq. 6):
    the few droplets closest to the fold carry n up to thousands of times the
    cloud's, a sparse and a dense seeding sample different ones, and neither
    estimate converges there; these cells are left out of the training and of
    the error."""
    h = cloud.to_host()
    d, N = wl.dim, wl.n_cells_axis
    act = h["status"] == 1
    det = np.abs(np.linalg.det(h["J"].astype(np.float64)))
    sel = act & (det < TAU_CAUSTIC) & np.all((h["x"] >= 0) & (h["x"] <= 1), axis=1)
    mark = np.zeros((N,) * d, bool)
    R = int(np.ceil(3.0 * wl.h_max * N))
    ci = np.minimum((h["x"][sel].astype(np.float64) * N).astype(np.int64), N - 1)
    for c in ci:
        lo = np.maximum(c - R, 0)
        hi = np.minimum(c + R + 1, N)
        mark[tuple(slice(lo[a], hi[a]) for a in range(d - 1, -1, -1))] = True   # axes (z,) y, x
    return mark.ravel()


def snapshot(c: "fla.DeviceCloud") -> "fla.DeviceCloud":
    """A device copy of a cloud (state, meta and release table shared read-only)."""
    s = object.__new__(fla.DeviceCloud)
    s.__dict__.update(c.__dict__)
    s.state = c.state.clone()
    s.meta = c.meta.clone()
    s.fold = None
    s.tau_fold = 0.0
    return s


def _fields(out: "fla.SourceFields") -> np.ndarray:
    return np.concatenate([out.s_mass.double().cpu().numpy()[:, None], out.s_mom.double().cpu().numpy().T], axis=1)


def flow_pair(flow: str, flow_seed: int, seeding: int = 8, matched_scale: bool = False, sparse_seeding: int = 1):
    """The sparse workload of a flow and its dense counterpart (seeding^2 = 64
    times the seeds in 2D, seeding^3 / 8 = 64 times in 3D: 2^24 droplets each).

      jet:  the 512^2 jet of the flow seed, 262,144 sparse seeds; the dense
            cloud splits each release into ``seeding`` releases of ``seeding``
            times the seeds (2^24), 1,000 steps;
      cone: the 128^3 ABC + round-jet flow of the seed (amplitudes and radius
            drawn within 10 %), a 64^3 seed lattice (2^18) against a 256^3
            one (2^24), J-scaled kernel (the correction scales its Lagrangian
            bandwidth h0), 500 steps.

    The dense cloud keeps its own smoothing length (its seed spacing): the
    target resolves what 64 times the seeds resolve, and the correction learns
    how far a sparse cloud's kernels should follow it.  With matched_scale the
    dense cloud takes the sparse one's smoothing length instead (the sparse
    method's own estimate without its sampling noise); against that target no
    bandwidth change improves on the plain method (measured: constant factors
    e^c, c in [-0.7, 1.1], and supports up to 3 h_max all leave the error at or
    above the plain one on the jet), so it is not used for training.
    sparse_seeding (jet only) multiplies the sparse cloud's seeds by its square,
    as ``seeding`` does the dense one's: the plain method at a denser seeding."""
    if flow == "jet":
        sp = I.jet_vortex_2d(scale=1, lpt_per_batch=0, flow_seed=flow_seed, seeding=sparse_seeding)
        de = I.jet_vortex_2d(scale=1, lpt_per_batch=0, flow_seed=flow_seed, seeding=seeding)
    elif flow == "cone":
        sp = I.abc_jet_3d(seeds_side=64, flow_seed=flow_seed, kernel=I.KERNEL_ANISO)
        de = I.abc_jet_3d(seeds_side=256, flow_seed=flow_seed, kernel=I.KERNEL_ANISO)
    else:
        raise ValueError(flow)
    if matched_scale:
        de.fla.h0 = np.full_like(de.fla.h0, float(sp.fla.h0[0]))
    return sp, de


def make_samples(ctx: "fla.Context", flow: str, flow_seeds, windows, matched_scale: bool = False,
                 sparse_seeding: int = 1) -> list[Sample]:
    """Runs the sparse and the dense cloud of each flow (see flow_pair) and
    keeps a sample at the end of each listed window."""
    import torch
    samples = []
    for fs in flow_seeds:
        wl_s, wl_d = flow_pair(flow, fs, matched_scale=matched_scale, sparse_seeding=sparse_seeding)
        sims = fla.Simulation(ctx, wl_s), fla.Simulation(ctx, wl_d)
        keep = set(windows)
        w = 0
        while sims[0].step < wl_s.nsteps and keep:
            dep = w in keep
            for sim in sims:
                sim.window(deposit=dep, with_psicell=False)
            if dep:
                torch.cuda.synchronize()
                target = _fields(sims[1].out)
                covered = sims[1].out.dsum.cpu().numpy() > 0
                snap = snapshot(sims[0].fla)
                samples.append(Sample(snap, sims[0].m, wl_s, target, covered & ~caustic_cells(snap, wl_s), covered))
                keep.discard(w)
            w += 1
        del sims
        torch.cuda.empty_cache()
    return samples


def sample_error(S: np.ndarray, T: np.ndarray, mask: np.ndarray) -> float:
    """Mean over components of ||S - T||^2 / ||T||^2 on the masked cells."""
    e = []
    for k in range(T.shape[1]):
        t = T[mask, k]
        nt = float(t @ t)
        if nt > 0:
            d = S[mask, k] - t
            e.append(float(d @ d) / nt)
    return float(np.mean(e))


def deposit_fields(ctx, smp: Sample, net=None) -> np.ndarray:
    import torch
    wl = smp.wl
    out = fla.SourceFields(smp.m, fla.F32)
    ws = fla.aligned_ws(fla.workspace(smp.m, fla.F32, wl.kernel, smp.cloud.n))
    cfg = fla.deposit_cfg(wl.kernel, wl.h_min, wl.h_max, wl.window * wl.dt, wl.p, mlp=net)
    fla.deposit_sources(ctx, smp.cloud, smp.m, cfg, out, ws)
    torch.cuda.synchronize()
    return _fields(out)


def evaluate(ctx, samples: list[Sample], net=None, all_cells: bool = False) -> float:
    """Mean sample error of the plain method (net None) or the learned one, on the
    covered cells away from fold caustics (all_cells: every covered cell)."""
    return float(np.mean([sample_error(deposit_fields(ctx, s, net), s.target, s.all_covered if all_cells else s.covered)
                          for s in samples]))


def train(ctx, samples: list[Sample], iters: int = 200, cells_per_sample: int = 850, lr: float = 2e-3,
          seed: int = 0, init_scale: float = 0.5, log=None, stats: dict | None = None) -> "fla.LearnedCorrection":
    """Adam on the sum of the samples' losses; the training cells of each sample
    are drawn once (seeded) from its covered cells.  stats (optional) receives
    the wall time per iteration of the loop (gradients of every sample, Adam,
    re-pack), in milliseconds."""
    import time

    import torch
    rng = np.random.default_rng(seed)
    net = fla.LearnedCorrection(ctx, fla.init_mlp_params(seed, init_scale, zero_last=True))
    bufs = []
    for s in samples:
        cov = np.nonzero(s.covered)[0]
        cells = np.sort(rng.choice(cov, min(cells_per_sample, cov.size), replace=False))
        bufs.append(fla.LearnBuffers(ctx, s.cloud, s.m, cells, s.target[cells], kernel=s.wl.kernel))
    grad = torch.zeros(fla.MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    mom, var = torch.zeros_like(grad), torch.zeros_like(grad)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(1, iters + 1):
        grad.zero_()
        loss.zero_()
        for b, s in zip(bufs, samples):
            cfg = fla.deposit_cfg(s.wl.kernel, s.wl.h_min, s.wl.h_max, s.wl.window * s.wl.dt, s.wl.p, mlp=net)
            fla.learn_grad(ctx, b, cfg, grad, loss)
        grad.mul_(1.0 / len(samples))
        fla.adam_step(ctx, net.params, grad, mom, var, it, lr=lr)
        net.pack()
        if log is not None and (it == 1 or it % 25 == 0 or it == iters):
            log(it, float(loss.item()) / len(samples))
    torch.cuda.synchronize()
    if stats is not None:
        stats["ms_per_iter"] = 1e3 * (time.perf_counter() - t0) / max(iters, 1)
    return net
