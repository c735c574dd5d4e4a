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
        order = fla.workspace_order(ws, m, cloud.n) if w > 0 else None   # cell-sorted by the last deposit
        fla.advance(ctx, cloud, m, nodes, step, wl.window, wl.dt, reset_acc=True, order=order)
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


def main(argv=None) -> int:
    """The paper's four cases (Re = 20, 100; without and with evaporation) at
    full resolution: per case the FLA-coupled and PSI-CELL-coupled runs, their
    force coefficients, profile agreement at the stations and wall times.
    Prints one JSON object."""
    import argparse
    import json
    import time

    import torch
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--scale", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warm", type=int, default=2000)
    args = ap.parse_args(argv)
    ctx = fla.Context(0)
    res = {}
    for re_, evap in ((20.0, False), (100.0, False), (20.0, True), (100.0, True)):
        case = I.cylinder_flow(re=re_, evaporating=evap, scale=args.scale, nsteps=args.steps, warm_steps=args.warm)
        runs, times = {}, {}
        for method in ("fla", "psicell"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            runs[method] = run(ctx, case, method)
            torch.cuda.synchronize()
            times[method] = time.perf_counter() - t0
        fl, ps = runs["fla"], runs["psicell"]
        tail = max(1, len(fl["cd"]) // 4)
        res[case.wl.name] = {
            "seeds_fla": case.wl.fla.n, "parcels_psicell": case.wl.lpt.n,
            "cd_clean": round(float(fl["cd_clean"]), 4),
            "cd_fla": round(float(fl["cd"][-tail:].mean()), 4), "cd_psicell": round(float(ps["cd"][-tail:].mean()), 4),
            "cl_amplitude_fla": round(float(np.ptp(fl["cl"][-tail:]) / 2), 4),
            "cl_amplitude_psicell": round(float(np.ptp(ps["cl"][-tail:]) / 2), 4),
            "S_mom_y": compare(fl, ps, "S_mom_y"), "S_mom_x": compare(fl, ps, "S_mom_x"),
            "S_mass": compare(fl, ps, "S_mass") if evap else None,
            "seconds": {k: round(v, 3) for k, v in times.items()}}
    ctx.close()
    print(json.dumps(res))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
