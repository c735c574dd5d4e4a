"""Seeded synthetic workloads for the FLA advance and the source-term deposits.

This module only *describes* inputs: meshes, carrier parameters, seed positions,
release schedules and per-release parameters, drawn from NumPy's PCG64 with
fixed seeds.  It holds none of the method's arithmetic (no carrier evaluation,
no drag, no Jacobian, no kernel), so the CPU oracle and the CUDA path can both
consume it without sharing any computation.  It imports nothing but NumPy.

The workloads mirror the paper's setting (Sec. 5: a single injection line
feeding a monodisperse evaporating cloud, St in [0.1, 0.5] per Table 1) on
synthetic carriers, because the paper's cylinder-flow data is not published
(Data Availability statement).  Sizes and parameters:

* ``taylor_green_2d``   64^2 mesh, steady Taylor-Green vortex, 4,096 FLA seeds
  on a lattice in the strip y in [0.45, 0.55], St0 = 0.5, delta = -0.2,
  200 RK4 steps of dt = 1e-3, FP64 path; PSI-CELL reference of 262,144
  uniformly seeded parcels in the same strip.
* ``jet_vortex_2d``     512^2 mesh, planar Gaussian jet (centre speed 1, width
  0.05) plus 8 Lamb-Oseen vortices advected with the jet, 256 releases of
  1,024 seeds at the inlet x = 0 over 1,000 steps, St0 ~ U[0.2, 2] per release,
  PSI-CELL reference of 2^24 parcels (65,536 per release).
* ``abc_jet_3d``        128^3 mesh, ABC flow (1, 0.7, 0.43) at wavenumber 2 pi
  plus a round jet, 2^21 seeds on a volume-preserving lattice in a cone,
  St0 = 1, 500 steps, anisotropic kernel.

Every generator takes a ``scale`` argument that shrinks the seed counts and
the mesh for fast tests while keeping the structure.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# Carrier kinds.  The numeric codes are part of the C interface of both the
# oracle and the CUDA library (each defines its own copy of the enum).
CARRIER_UNIFORM = 0
CARRIER_LINEAR = 1
CARRIER_TAYLOR_GREEN_2D = 2
CARRIER_JET_VORTEX_2D = 3
CARRIER_ABC_JET_3D = 4

KERNEL_ISO = 0
KERNEL_ANISO = 1

CLOUD_FLA = 0
CLOUD_LPT = 1

NO_DEADLINE = 2**31 - 1


@dataclass
class Carrier:
    """Parameters of an analytic carrier velocity field u(x, t) on [0,1]^dim."""
    kind: int
    dim: int
    U: np.ndarray = field(default_factory=lambda: np.zeros(3))       # uniform part
    A: np.ndarray = field(default_factory=lambda: np.zeros((3, 3)))  # linear part
    xref: np.ndarray = field(default_factory=lambda: np.zeros(3))
    # Lamb-Oseen vortices: rows (x0, yc, Gamma, rc, Uadv); centre x(t) = frac(x0 + Uadv t)
    vortices: np.ndarray = field(default_factory=lambda: np.zeros((0, 5)))
    jet_width: float = 0.05          # planar jet: u_x += exp(-((y-1/2)/w)^2)
    abc: np.ndarray = field(default_factory=lambda: np.array([1.0, 0.7, 0.43]))
    jet_amp: float = 1.0             # round jet: u_z += amp exp(-(rho/r)^2)
    jet_radius: float = 0.05
    steady: bool = True


@dataclass
class Cloud:
    """Seeds of one cloud: initial positions and the release table."""
    kind: int                  # CLOUD_FLA or CLOUD_LPT
    x0: np.ndarray             # (n, dim) float64 seed positions
    batch: np.ndarray          # (n,) int32 release index of each seed
    step_start: np.ndarray     # (n_batches,) int32 step at which the release enters
    St0: np.ndarray            # (n_batches,) float64 Stokes number at release
    n0: np.ndarray             # (n_batches,) float64 number density at release (FLA) or parcel weight (LPT)
    h0: np.ndarray             # (n_batches,) float64 initial smoothing length (FLA)

    @property
    def n(self) -> int:
        return int(self.x0.shape[0])


@dataclass
class Workload:
    name: str
    dim: int
    n_cells_axis: int
    dt: float
    nsteps: int
    window: int                # steps per deposit window (also the carrier frozen period)
    delta: float               # d^2-law rate (rate of change of surface area), r0 = 1
    carrier: Carrier
    fla: Cloud
    lpt: Cloud | None
    kernel: int
    h_min: float
    h_max: float
    p: float = 1.0             # exponent of |det J| in h = h0 |det J|^p

    @property
    def n_cells(self) -> int:
        return self.n_cells_axis ** self.dim

    @property
    def dx(self) -> float:
        return 1.0 / self.n_cells_axis


def _lattice_strip(nx: int, ny: int, y_lo: float, y_hi: float) -> np.ndarray:
    """Cell-centred nx-by-ny lattice on [0,1] x [y_lo, y_hi], x fastest."""
    xs = (np.arange(nx) + 0.5) / nx
    ys = y_lo + (np.arange(ny) + 0.5) * (y_hi - y_lo) / ny
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def taylor_green_2d(scale: int = 1) -> Workload:
    """64^2 cells, steady Taylor-Green vortex, lattice seeding of a strip.

    ``scale`` > 1 divides the mesh and the seed counts per axis by ``scale``.
    """
    N = 64 // scale
    n_side = 64 // scale
    x0 = _lattice_strip(n_side, n_side, 0.45, 0.55)
    nf = x0.shape[0]
    car = Carrier(kind=CARRIER_TAYLOR_GREEN_2D, dim=2)
    fla = Cloud(kind=CLOUD_FLA, x0=x0, batch=np.zeros(nf, np.int32),
                step_start=np.zeros(1, np.int32), St0=np.array([0.5]),
                n0=np.array([1.0]), h0=np.array([1.0 / n_side]))
    rng = np.random.default_rng(1)
    m = 262_144 // (scale * scale * scale)
    xl = np.stack([rng.uniform(0.0, 1.0, m), rng.uniform(0.45, 0.55, m)], axis=1)
    lpt = Cloud(kind=CLOUD_LPT, x0=xl, batch=np.zeros(m, np.int32),
                step_start=np.zeros(1, np.int32), St0=np.array([0.5]),
                n0=np.array([0.1 / m]),   # parcel weight: strip area x n0 / parcels
                h0=np.zeros(1))
    dx = 1.0 / N
    return Workload(name=f"taylor_green_2d_{N}x{N}_{nf}fla", dim=2, n_cells_axis=N, dt=1e-3,
                    nsteps=200, window=10, delta=-0.2, carrier=car, fla=fla, lpt=lpt,
                    kernel=KERNEL_ISO, h_min=0.5 * dx, h_max=4.0 * dx)


@dataclass
class TwoWayCase:
    """A two-way coupled workload: the droplet workload on a periodic carrier
    (Eqs. 1-2) with its initial nodal vorticity and mean flow."""
    wl: Workload
    nu: float                  # 1/Re
    diff: float                # vapour diffusivity
    omega0: np.ndarray         # (N, N) nodal vorticity, x fastest
    mean_u: tuple


def two_way_taylor_green(scale: int = 1, nsteps: int = 200, n0: float = 1.0) -> TwoWayCase:
    """128^2 periodic cells, Re = 1000, vapour diffusivity 1e-3; the carrier
    starts as the Taylor-Green vortex of unit speed and period 1, stream
    function sin(2 pi x) sin(2 pi y)/(2 pi), nodal vorticity
    4 pi sin(2 pi x) sin(2 pi y).  A strip of FLA seeds (a 128 x 128 lattice in
    y in [0.45, 0.55]) with St0 = 0.5 and delta = -0.2, number density n0,
    spherical kernel, deposit every 10 steps; the carrier takes those 10 steps
    with the window's sources.  ``scale`` divides the mesh and the lattice."""
    N = 128 // scale
    n_side = 128 // scale
    x0 = _lattice_strip(n_side, n_side, 0.45, 0.55)
    nf = x0.shape[0]
    fla = Cloud(kind=CLOUD_FLA, x0=x0, batch=np.zeros(nf, np.int32),
                step_start=np.zeros(1, np.int32), St0=np.array([0.5]),
                n0=np.array([n0]), h0=np.array([1.0 / n_side]))
    dx = 1.0 / N
    wl = Workload(name=f"two_way_taylor_green_{N}x{N}_{nf}fla", dim=2, n_cells_axis=N, dt=1e-3,
                  nsteps=nsteps, window=10, delta=-0.2, carrier=Carrier(kind=CARRIER_UNIFORM, dim=2),
                  fla=fla, lpt=None, kernel=KERNEL_ISO, h_min=0.5 * dx, h_max=4.0 * dx)
    g = np.arange(N) / N
    omega0 = 4.0 * np.pi * np.sin(2 * np.pi * g)[None, :] * np.sin(2 * np.pi * g)[:, None]
    return TwoWayCase(wl=wl, nu=1e-3, diff=1e-3, omega0=omega0, mean_u=(0.0, 0.0))


@dataclass
class CylinderCase:
    """Flow past a cylinder with droplets injected upstream (the paper's test
    case, Sec. 5) on the periodic two-way carrier: the droplet workload (FLA
    seeds and PSI-CELL parcels), the carrier's viscosity and vapour
    diffusivity, the cylinder (volume penalisation) and fringe, the inflow and
    the carrier steps run before the first release."""
    wl: Workload
    nu: float
    diff: float
    body: dict
    mean_u: tuple
    warm_steps: int
    R: float
    xc: float


def cylinder_flow(re: float = 20.0, evaporating: bool = False, scale: int = 1, nsteps: int = 2000,
                  warm_steps: int = 1000, lpt: bool = True) -> CylinderCase:
    """Cylinder of radius R = 0.05 at (0.3, 0.5) in a periodic unit square of
    256^2 cells (R = 12.8 cells), inflow U = (1, 0) held fixed, Re = 2 U R / nu
    (20: steady wake; 100: shedding), vapour diffusivity nu/2 (Schmidt number 2,
    within the explicit diffusion's limit at 256^2),
    a fringe strip 0.92 <= x <= 1 absorbing the wake.  Droplets enter at
    x/R = -5 (x = 0.05) across 0.3 <= y <= 0.7: FLA releases of 100 seeds every
    5 steps, PSI-CELL releases of 2,000 parcels every step (100 times the droplets
    per unit time, as in the paper), n0 = 1, St = tau U / 2R of 0.1 (0.5 for the
    evaporating Re = 100 case, as Table 1), delta = -0.2 when evaporating.
    The carrier runs warm_steps steps before the first release.  ``scale``
    divides the mesh (the droplet counts stay)."""
    N = 256 // scale
    R, xc, yc, U = 0.05, 0.3, 0.5, 1.0
    dt = 1e-3
    nu = 2.0 * U * R / re
    st = 0.5 if (evaporating and re >= 100) else 0.1
    St0 = st * 2.0 * R / U
    delta = -0.2 if evaporating else 0.0
    y_lo, y_hi, x_inj = 0.3, 0.7, xc - 5.0 * R
    # FLA: 100 seeds per release every 5 steps
    every, per = 5, 100
    n_rel = nsteps // every
    ys = y_lo + (np.arange(per) + 0.5) * (y_hi - y_lo) / per
    x0 = np.stack([np.full(n_rel * per, x_inj), np.tile(ys, n_rel)], axis=1)
    batch = np.repeat(np.arange(n_rel, dtype=np.int32), per)
    step_start = (np.arange(n_rel) * every).astype(np.int32)
    tau = every * dt
    h0 = max((y_hi - y_lo) / per, U * tau)
    fla = Cloud(kind=CLOUD_FLA, x0=x0, batch=batch, step_start=step_start, St0=np.full(n_rel, St0),
                n0=np.ones(n_rel), h0=np.full(n_rel, h0))
    lp = None
    if lpt:
        m_b = 2000
        rng = np.random.default_rng(5)
        xl = np.stack([np.full(nsteps * m_b, x_inj), rng.uniform(y_lo, y_hi, nsteps * m_b)], axis=1)
        V_inj = (y_hi - y_lo) * U * dt          # swept by the inlet per release
        lp = Cloud(kind=CLOUD_LPT, x0=xl, batch=np.repeat(np.arange(nsteps, dtype=np.int32), m_b),
                   step_start=np.arange(nsteps, dtype=np.int32), St0=np.full(nsteps, St0),
                   n0=np.full(nsteps, V_inj / m_b), h0=np.zeros(nsteps))
    dx = 1.0 / N
    wl = Workload(name=f"cylinder_re{int(re)}{'_evap' if evaporating else ''}_{N}x{N}", dim=2, n_cells_axis=N, dt=dt,
                  nsteps=nsteps, window=10, delta=delta, carrier=Carrier(kind=CARRIER_UNIFORM, dim=2),
                  fla=fla, lpt=lp, kernel=KERNEL_ISO, h_min=0.5 * dx, h_max=4.0 * dx)
    body = dict(xc=xc, yc=yc + 0.25 * dx, r=R, eta=2.0 * dt, fringe_x0=0.92, fringe_x1=1.0, fringe_sigma=200.0,
                hold_mean_flow=True)   # off the node lattice's symmetry line by a quarter cell: shedding can start
    return CylinderCase(wl=wl, nu=nu, diff=0.5 * nu, body=body, mean_u=(U, 0.0), warm_steps=warm_steps, R=R, xc=xc)


def _jet_vortices(rng: np.random.Generator, n_vort: int, width: float) -> np.ndarray:
    x0 = rng.uniform(0.0, 1.0, n_vort)
    yc = rng.uniform(0.3, 0.7, n_vort)
    gam = rng.uniform(-0.5, 0.5, n_vort)
    rc = np.full(n_vort, 0.02)
    # each vortex is carried at the jet speed found at its own centre line
    uadv = np.exp(-((yc - 0.5) / width) ** 2)
    return np.stack([x0, yc, gam, rc, uadv], axis=1)


def jet_vortex_2d(scale: int = 1, nsteps: int = 1000, lpt_per_batch: int = 65_536, flow_seed: int = 2,
                  seeding: int = 1) -> Workload:
    """512^2 cells, planar jet + 8 Lamb-Oseen vortices, inlet releases.

    ``scale`` divides the mesh by ``scale`` and the release count and release
    size by ``scale``; the number of steps is kept unless ``nsteps`` is given.
    ``flow_seed`` draws the vortices and the releases' Stokes numbers.
    ``seeding`` multiplies both the release count and the seeds per release
    (``seeding**2`` times the seeds of the same droplet population: each
    release of the base seeding is split into ``seeding`` releases with its
    Stokes number); the PSI-CELL parcels are built for ``seeding == 1`` only.
    """
    N = 512 // scale
    base_batches = 256 // scale
    n_batches = base_batches * seeding
    per_batch = (1024 // scale) * seeding
    width = 0.05
    rng = np.random.default_rng(flow_seed)
    car = Carrier(kind=CARRIER_JET_VORTEX_2D, dim=2, vortices=_jet_vortices(rng, 8, width),
                  jet_width=width, steady=False)
    St0 = np.repeat(rng.uniform(0.2, 2.0, base_batches), seeding)
    step_start = np.floor(nsteps * np.arange(n_batches) / n_batches).astype(np.int32)
    ys = 0.45 + (np.arange(per_batch) + 0.5) * (0.1 / per_batch)
    x0 = np.zeros((n_batches * per_batch, 2))
    x0[:, 1] = np.tile(ys, n_batches)
    batch = np.repeat(np.arange(n_batches, dtype=np.int32), per_batch)
    dt = 1e-3
    tau_inj = nsteps * dt / n_batches
    # Appendix A: each seed stands for V_inj / N_FLA with V_inj = A_inj v_inj tau_inj;
    # v_inj is the mean jet speed over the inlet, the largest seed spacing sets h0.
    v_inj = width * math.sqrt(math.pi) * math.erf(0.05 / width) / 0.1
    h0 = max(tau_inj * 1.0, 0.1 / per_batch)
    fla = Cloud(kind=CLOUD_FLA, x0=x0, batch=batch, step_start=step_start, St0=St0,
                n0=np.ones(n_batches), h0=np.full(n_batches, h0))
    lpt = None
    if lpt_per_batch and seeding == 1:
        m_b = lpt_per_batch // (scale * scale) if scale > 1 else lpt_per_batch
        rng3 = np.random.default_rng(3)
        xl = np.zeros((n_batches * m_b, 2))
        xl[:, 1] = rng3.uniform(0.45, 0.55, n_batches * m_b)
        V_inj = 0.1 * v_inj * tau_inj
        lpt = Cloud(kind=CLOUD_LPT, x0=xl, batch=np.repeat(np.arange(n_batches, dtype=np.int32), m_b),
                    step_start=step_start.copy(), St0=St0.copy(),
                    n0=np.full(n_batches, V_inj / m_b), h0=np.zeros(n_batches))
    dx = 1.0 / N
    return Workload(name=f"jet_vortex_2d_{N}x{N}_{x0.shape[0]}fla_flow{flow_seed}", dim=2, n_cells_axis=N, dt=dt,
                    nsteps=nsteps, window=10, delta=-0.2, carrier=car, fla=fla, lpt=lpt,
                    kernel=KERNEL_ISO, h_min=0.5 * dx, h_max=4.0 * dx)


def _square_to_disc(a: np.ndarray, b: np.ndarray):
    """Shirley-Chiu concentric map of [0,1)^2 onto the unit disc (area preserving)."""
    sa = 2.0 * a - 1.0
    sb = 2.0 * b - 1.0
    r = np.where(np.abs(sa) > np.abs(sb), sa, sb)
    with np.errstate(divide="ignore", invalid="ignore"):
        phi = np.where(np.abs(sa) > np.abs(sb),
                       (math.pi / 4.0) * (sb / sa),
                       (math.pi / 2.0) - (math.pi / 4.0) * (sa / sb))
    phi = np.nan_to_num(phi)
    return r * np.cos(phi), r * np.sin(phi)


def abc_jet_3d(scale: int = 1, nsteps: int = 500, seeds_side: int | None = None, flow_seed: int | None = None,
               kernel: int = KERNEL_ANISO) -> Workload:
    """128^3 cells, ABC flow + round jet, 2^21 seeds in a cone, anisotropic kernel.

    ``scale`` divides the mesh and the seed lattice per axis; ``seeds_side``
    sets the seed lattice (n_side^3 seeds) independently of the mesh.
    ``flow_seed`` (None: the canonical flow) draws the ABC amplitudes and the
    jet radius within +-10 % of (1, 0.7, 0.43) and 0.05, for families of
    flows of the same kind.  ``kernel`` selects the deposit kernel."""
    N = 128 // scale
    n_side = seeds_side if seeds_side is not None else 128 // scale
    g = (np.arange(n_side) + 0.5) / n_side
    X1, X2, X3 = np.meshgrid(g, g, g, indexing="ij")
    xi1, xi2, xi3 = X1.ravel(), X2.ravel(), X3.ravel()
    order = np.lexsort((xi1, xi2, xi3))          # x fastest
    xi1, xi2, xi3 = xi1[order], xi2[order], xi3[order]
    apex, length, half_angle = 0.1, 0.6, math.radians(30.0)
    z = apex + length * np.cbrt(xi3)             # volume-preserving axial coordinate
    radius = (z - apex) * math.tan(half_angle)
    dxd, dyd = _square_to_disc(xi1, xi2)
    x0 = np.stack([0.5 + radius * dxd, 0.5 + radius * dyd, z], axis=1)
    n = x0.shape[0]
    v_cone = math.pi * (length * math.tan(half_angle)) ** 2 * length / 3.0
    h0 = (v_cone / n) ** (1.0 / 3.0)
    abc, radius = np.array([1.0, 0.7, 0.43]), 0.05
    if flow_seed is not None:
        rng = np.random.default_rng(flow_seed)
        abc = abc * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, 3))
        radius = radius * (1.0 + 0.1 * rng.uniform(-1.0, 1.0))
    car = Carrier(kind=CARRIER_ABC_JET_3D, dim=3, abc=abc, jet_amp=1.0, jet_radius=radius)
    fla = Cloud(kind=CLOUD_FLA, x0=x0, batch=np.zeros(n, np.int32), step_start=np.zeros(1, np.int32),
                St0=np.array([1.0]), n0=np.array([1.0]), h0=np.array([h0]))
    dx = 1.0 / N
    tag = "" if flow_seed is None else f"_flow{flow_seed}"
    return Workload(name=f"abc_jet_3d_{N}^3_{n}fla{tag}", dim=3, n_cells_axis=N, dt=1e-3, nsteps=nsteps,
                    window=10, delta=-0.2, carrier=car, fla=fla, lpt=None,
                    kernel=kernel, h_min=0.5 * dx, h_max=2.0 * dx)


# ---------------------------------------------------------------------------
# Synthetic cloud states for deposit-only tests: positions, Jacobians and
# window accumulators drawn directly (no integration), shaped like a cloud
# after some deformation: compressed and stretched regions, inactive seeds,
# droplets on cell faces and on the upper domain edge.
# ---------------------------------------------------------------------------

@dataclass
class CloudState:
    dim: int
    x: np.ndarray          # (n, dim) float32 positions
    v: np.ndarray          # (n, dim) float32 velocities
    J: np.ndarray          # (n, dim, dim) float32 Jacobian dx/dx0
    W: np.ndarray          # (n, dim, dim) float32 its rate
    acc: np.ndarray        # (n, 1+dim) float32 window sums of mdot and F + mdot v
    status: np.ndarray     # (n,) int32: 0 pending, 1 active, 2 dead
    batch: np.ndarray      # (n,) int32
    n0: np.ndarray         # (n_batches,) float64
    h0: np.ndarray         # (n_batches,) float64


def synthetic_state(dim: int, n: int, n_cells_axis: int, seed: int, *, band=(0.3, 0.7),
                    n_batches: int = 4, h0_cells: float = 2.0, inactive_frac: float = 0.05,
                    jac_spread: float = 0.5, edge_cases: bool = True) -> CloudState:
    rng = np.random.default_rng(seed)
    N = n_cells_axis
    x = rng.uniform(0.0, 1.0, (n, dim))
    x[:, -1] = rng.uniform(band[0], band[1], n)          # a band across the last axis
    if edge_cases and n >= 16:
        k = max(1, n // 64)
        idx = rng.choice(n, 4 * k, replace=False)
        f = rng.integers(0, N + 1, (k, dim)) / N            # exactly on cell faces
        x[idx[:k]] = f
        x[idx[k:2 * k], 0] = 1.0                            # upper domain edge
        x[idx[2 * k:3 * k], :] = x[idx[2 * k], :]              # one crowded spot
    # Jacobian: random rotation-ish matrix times log-normal stretches
    M = np.eye(dim)[None] + jac_spread * rng.standard_normal((n, dim, dim)) / math.sqrt(dim)
    scale = np.exp(rng.uniform(-1.5, 1.0, (n, 1, 1)))
    J = M * scale
    W = rng.standard_normal((n, dim, dim))
    v = rng.standard_normal((n, dim))
    acc = np.empty((n, 1 + dim))
    acc[:, 0] = -1e-3 * (1.0 + 0.5 * rng.standard_normal(n))
    acc[:, 1:] = 1e-2 * rng.standard_normal((n, dim)) + 1e-2 * np.sin(2 * math.pi * x)
    status = np.where(rng.uniform(size=n) < inactive_frac, 2, 1).astype(np.int32)
    batch = rng.integers(0, n_batches, n).astype(np.int32)
    n0 = rng.uniform(0.5, 2.0, n_batches)
    h0 = np.full(n_batches, h0_cells / N) * rng.uniform(0.7, 1.3, n_batches)
    return CloudState(dim=dim, x=x.astype(np.float32), v=v.astype(np.float32), J=J.astype(np.float32),
                      W=W.astype(np.float32), acc=acc.astype(np.float32), status=status, batch=batch,
                      n0=n0, h0=h0)


def batch_clouds(seed: int = 4, n_clouds: int = 64, nsteps: int = 100, n_min: float = 1e3, n_max: float = 5e5,
                 meshes2=(32, 64, 128, 256), meshes3=(32, 64)) -> list[Workload]:
    """Many clouds of uneven size and resolution for the batched path: sizes
    log-uniform in [n_min, n_max], half 2D (meshes ``meshes2``, Taylor-Green or
    jet + vortices, spherical kernel, h_max = 4 dx) and half 3D (meshes
    ``meshes3``, ABC + round jet, J-scaled kernel, h_max = 2 dx).  Each cloud
    is one release at step 0 of seeds uniform in a random box, Stokes number
    U[0.2, 2], delta = -0.2, h0 = (box volume / seeds)^(1/dim), dt = 1e-3,
    windows of 10 steps."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_clouds):
        dim = 2 if k % 2 == 0 else 3
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        N = int(rng.choice(meshes2 if dim == 2 else meshes3))
        lo = rng.uniform(0.1, 0.5, dim)
        size = np.minimum(rng.uniform(0.2, 0.4, dim), 0.9 - lo)
        x0 = lo + size * rng.uniform(0.0, 1.0, (n, dim))
        if dim == 2:
            if rng.uniform() < 0.5:
                car = Carrier(kind=CARRIER_TAYLOR_GREEN_2D, dim=2)
            else:
                car = Carrier(kind=CARRIER_JET_VORTEX_2D, dim=2, vortices=_jet_vortices(rng, 8, 0.05),
                              jet_width=0.05, steady=False)
            kernel, hmax = KERNEL_ISO, 4.0
        else:
            car = Carrier(kind=CARRIER_ABC_JET_3D, dim=3)
            kernel, hmax = KERNEL_ANISO, 2.0
        St0 = rng.uniform(0.2, 2.0, 1)
        h0 = float(np.prod(size) / n) ** (1.0 / dim)
        cl = Cloud(kind=CLOUD_FLA, x0=x0, batch=np.zeros(n, np.int32), step_start=np.zeros(1, np.int32), St0=St0,
                   n0=np.ones(1), h0=np.array([h0]))
        dx = 1.0 / N
        out.append(Workload(name=f"batch{seed}_{k}_{dim}d_{N}_{n}", dim=dim, n_cells_axis=N, dt=1e-3, nsteps=nsteps,
                            window=10, delta=-0.2, carrier=car, fla=cl, lpt=None, kernel=kernel, h_min=0.5 * dx,
                            h_max=hmax * dx))
    return out
