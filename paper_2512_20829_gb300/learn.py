"""Training and evaluation of the learned bandwidth correction (the paper has no
counterpart).  Orchestration only: every deposit, gradient and update runs in
the CUDA library through fla.py.

A sample is one sparse-seeded cloud state at a deposit time together with the
sources of a densely seeded cloud of the same flow at the same time (the
target).  The loss of fla_learn_grad is the mean over the source components
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
    covered: np.ndarray           # cells where the dense reference has D > 0


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


def make_samples(ctx: "fla.Context", flow_seeds, windows, scale: int = 4, seeding: int = 8,
                 nsteps: int = 1000) -> list[Sample]:
    """Runs the sparse (base seeding) and the dense (``seeding``^2 times the
    seeds) jet of each flow and keeps a sample at the end of each listed window."""
    import torch
    samples = []
    for fs in flow_seeds:
        wl_s = I.jet_vortex_2d(scale=scale, nsteps=nsteps, lpt_per_batch=0, flow_seed=fs)
        wl_d = I.jet_vortex_2d(scale=scale, nsteps=nsteps, lpt_per_batch=0, flow_seed=fs, seeding=seeding)
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
                samples.append(Sample(snapshot(sims[0].fla), sims[0].m, wl_s, target, covered))
                keep.discard(w)
            w += 1
        del sims
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


def evaluate(ctx, samples: list[Sample], net=None) -> float:
    """Mean sample error of the plain method (net None) or the learned one."""
    return float(np.mean([sample_error(deposit_fields(ctx, s, net), s.target, s.covered) for s in samples]))


def train(ctx, samples: list[Sample], iters: int = 200, cells_per_sample: int = 1700, lr: float = 2e-3,
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
        bufs.append(fla.LearnBuffers(ctx, s.cloud, s.m, cells, s.target[cells]))
    wl = samples[0].wl
    grad = torch.zeros(fla.MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    mom, var = torch.zeros_like(grad), torch.zeros_like(grad)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(1, iters + 1):
        grad.zero_()
        loss.zero_()
        for b, s in zip(bufs, samples):
            cfg = fla.deposit_cfg(wl.kernel, s.wl.h_min, s.wl.h_max, s.wl.window * s.wl.dt, s.wl.p, mlp=net)
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
