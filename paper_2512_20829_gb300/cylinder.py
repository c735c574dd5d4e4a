"""Flow past a cylinder with droplets injected upstream: the paper's test case
(Sec. 5) on the periodic two-way carrier.  Orchestration only: the carrier,
the advance and the deposits run in the CUDA library through fla.py.

One run couples one droplet representation to the carrier: the FLA seeds
with the kernel-regression sources (Eq. 16), or the PSI-CELL parcels with the
box-count sources (Eqs. 10-11), as the paper compares two simulations.  The
carrier first runs without droplets (warm_steps); then per window of 10
steps: the carrier's node values, the fused advance, the deposit, and the
carrier's 10 steps with the window's sources.  Reported: the force
coefficients C_d, C_l = F / (rho U^2 R) per window (F the force on the
penalised cylinder, rho = 1), the sources averaged over the last windows, and
their profiles across the flow at x/R = 0, 3, 6, 9, 12 from the cylinder
centre (the paper's stations)."""
from __future__ import annotations

import numpy as np

from . import fla
from . import inputs as I

STATIONS = (0, 3, 6, 9, 12)


def run(ctx, case: I.CylinderCase, method: str = "fla", dtype: int = fla.F32, coupled: bool = True,
        average_windows: int = 10) -> dict:
    import torch
    wl = case.wl
    N = wl.n_cells_axis
    ns = fla.NavierStokes(ctx, N, case.nu, case.diff, wl.dt, np.zeros((N, N)), mean_u=case.mean_u, body=case.body)
    if case.warm_steps:
        ns.step(case.warm_steps)
    U = case.mean_u[0]
    f_clean = ns.body_force()
    m = fla.mesh(2, N)
    nodes = fla.nodes_buffer(m, dtype)
    src = wl.fla if method == "fla" else wl.lpt
    cloud = fla.DeviceCloud.from_seeds(src, 2, wl.delta, wl.dt, dtype)
    ws = fla.aligned_ws(fla.workspace(m, dtype, wl.kernel, cloud.n))
    if method == "fla":
        out = fla.SourceFields(m, dtype)
        cfg = fla.deposit_cfg(wl.kernel, wl.h_min, wl.h_max, wl.window * wl.dt, wl.p)
    else:
        out = fla.PsicellFields(m, dtype)
    n_windows = wl.nsteps // wl.window
    s_mass = torch.zeros(N * N, dtype=torch.float64, device="cuda")
    s_mom = torch.zeros(2, N * N, dtype=torch.float64, device="cuda")
    forces = []
    for w in range(n_windows):
        step = w * wl.window
        ns.nodes(dtype, nodes)
        fla.advance(ctx, cloud, m, nodes, step, wl.window, wl.dt, reset_acc=True)
        if method == "fla":
            fla.deposit_sources(ctx, cloud, m, cfg, out, ws)
        else:
            fla.psicell(ctx, cloud, m, wl.window * wl.dt, out, ws)
        ns.step(wl.window, out if coupled else None)
        forces.append(ns.body_force())
        if w >= n_windows - average_windows:
            s_mass += out.s_mass.double()
            s_mom += out.s_mom.double()
    torch.cuda.synchronize()
    k = min(average_windows, n_windows)
    Sm = (s_mass / k).cpu().numpy().reshape(N, N)
    Sx, Sy = ((s_mom / k).cpu().numpy()[q].reshape(N, N) for q in range(2))
    F = np.array(forces)
    scale = U * U * case.R
    cols = [min(int((case.xc + st * case.R) * N), N - 1) for st in STATIONS]
    return {"method": method, "cd": F[:, 0] / scale, "cl": F[:, 1] / scale,
            "cd_clean": f_clean[0] / scale, "cl_clean": f_clean[1] / scale,
            "S_mass": Sm, "S_mom_x": Sx, "S_mom_y": Sy,
            "profiles": {st: {"S_mass": Sm[:, c], "S_mom_x": Sx[:, c], "S_mom_y": Sy[:, c]}
                         for st, c in zip(STATIONS, cols)},
            "fields": ns.fields()}


def compare(a: dict, b: dict, field: str = "S_mom_y") -> dict:
    """Per station: the correlation of two runs' profiles and the ratio of their
    norms (statistical agreement, not parity: the paper shows figures only)."""
    out = {}
    for st in STATIONS:
        x, y = a["profiles"][st][field], b["profiles"][st][field]
        nx, ny = np.linalg.norm(x), np.linalg.norm(y)
        corr = float(x @ y / (nx * ny)) if nx > 0 and ny > 0 else float("nan")
        out[st] = {"corr": corr, "norm_ratio": float(nx / ny) if ny > 0 else float("nan")}
    return out
