"""FP64 oracle of the two-way carrier: the incompressible Navier-Stokes carrier
(Eq. 1) with the droplets' momentum source, and the vapour transport (Eq. 2)
with their mass source, on a periodic unit square.  Test infrastructure: only
the tests, the smoke check and the bench's CPU baseline use it; it shares no
code with the CUDA path.  NumPy only (np.fft as the library FFT).

Discretisation (plain, second order in space, first order in time):

* Nodes (i h, j h) and cells ((i + 1/2) h, (j + 1/2) h), h = 1/N, periodic;
  arrays are indexed [j, i] (x fastest, as the mesh's cell keys).
* Vorticity-streamfunction form of Eq. 1: omega at the nodes is the
  prognostic field, psi solves Lap_h psi = -omega with the 5-point Laplacian
  (exactly, in Fourier space), and the velocity at the nodes is
  u = U_x + D_y psi, v = U_y - D_x psi (central differences), U the mean
  velocity, which a periodic streamfunction cannot carry.
* One step of dt: R = -(u D_x omega + v D_y omega) + curl S_mom at the nodes
  (S_mom at the cells, the curl from the four cells around a node), then
  omega <- (omega + dt R) / (1 - dt nu lambda) in Fourier space (advection and
  source explicit, viscosity 1/Re implicit; lambda the 5-point Laplacian's
  eigenvalue), the mean vorticity kept zero, and U <- U + dt mean(S_mom).
* Vapour rho at the cells, Eq. 2 read with the physical sign of diffusion
  (the printed equation puts D grad^2 on the left, which would be
  anti-diffusion): rho <- rho + dt (-div_h F + D Lap_h rho + S_mass), F the
  first-order upwind fluxes with face velocities from psi at the face's two
  corner nodes (exactly divergence-free cell by cell).
* An immersed cylinder (optional, Body): the momentum equation gains the
  volume-penalisation force -chi u / eta (its curl in the vorticity equation,
  by central differences of the nodal products), a fringe strip relaxes the
  vorticity to zero, and the mean flow is either held (constant inflow) or
  decelerated by the mean penalisation force.  The force on the body is the
  sum of chi u / eta h^2 over the nodes.
* For the droplets: u, v and grad u at the (N+1)^2 mesh nodes (the periodic
  node N repeats node 0), grad u by central differences of the nodal
  velocity (trace-free exactly), in the node layout of the analytic carriers
  (u[2], grad u[4], 2 pad).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Body:
    """An immersed cylinder by volume penalisation (Brinkman): the momentum
    equation gains -chi u / eta, chi = (1 - tanh((r - R)/h))/2 at the nodes,
    r the distance to the centre; and a fringe strip x0 <= x <= x1 where the
    vorticity relaxes to zero at the rate sigma_max sin^2(pi (x - x0)/(x1 - x0)),
    so the periodic wake does not re-enter.  hold_mean_flow keeps U fixed (a
    mean pressure gradient balances the mean forcing: a constant inflow)."""
    xc: float
    yc: float
    R: float
    eta: float
    x0: float = 0.0
    x1: float = 0.0
    sigma_max: float = 0.0
    hold_mean_flow: bool = True


@dataclass
class NSState:
    N: int
    nu: float             # 1/Re
    D: float              # vapour diffusivity
    omega_hat: np.ndarray  # (N, N) complex: Fourier coefficients of the nodal vorticity
    U: np.ndarray          # (2,) mean velocity
    rho: np.ndarray        # (N, N) vapour at the cells
    t: float = 0.0
    body: Body | None = None


def laplacian_eigenvalues(N: int) -> np.ndarray:
    """lambda[ky, kx] of the periodic 5-point Laplacian with h = 1/N."""
    k = np.arange(N)
    s = np.sin(np.pi * k / N) ** 2
    return -4.0 * N * N * (s[:, None] + s[None, :])


def _dx(f, h):
    return (np.roll(f, -1, axis=1) - np.roll(f, 1, axis=1)) / (2.0 * h)


def _dy(f, h):
    return (np.roll(f, -1, axis=0) - np.roll(f, 1, axis=0)) / (2.0 * h)


def lap5(f, h):
    """5-point Laplacian, periodic."""
    return (np.roll(f, 1, 0) + np.roll(f, -1, 0) + np.roll(f, 1, 1) + np.roll(f, -1, 1) - 4.0 * f) / (h * h)


def init(N: int, nu: float, D: float, omega: np.ndarray, U=(0.0, 0.0), rho=None, body: Body | None = None) -> NSState:
    """State from a nodal vorticity field (its mean is removed)."""
    oh = np.fft.fft2(np.asarray(omega, np.float64))
    oh[0, 0] = 0.0
    r = np.zeros((N, N)) if rho is None else np.array(rho, np.float64)
    return NSState(N=N, nu=float(nu), D=float(D), omega_hat=oh, U=np.array(U, np.float64), rho=r, body=body)


def body_mask(N: int, b: Body) -> np.ndarray:
    """chi at the nodes (i h, j h), [j, i]."""
    x = np.arange(N) / N
    r = np.hypot(x[None, :] - b.xc, x[:, None] - b.yc)
    return 0.5 * (1.0 - np.tanh((r - b.R) * N))


def fringe(N: int, b: Body) -> np.ndarray:
    """sigma(x) at the nodes, [j, i]."""
    x = np.arange(N) / N
    s = np.zeros(N)
    if b.x1 > b.x0 and b.sigma_max > 0:
        inside = (x >= b.x0) & (x <= b.x1)
        s[inside] = b.sigma_max * np.sin(np.pi * (x[inside] - b.x0) / (b.x1 - b.x0)) ** 2
    return np.broadcast_to(s[None, :], (N, N)).copy()


def body_force(st: NSState) -> np.ndarray:
    """Force of the fluid on the body: sum over the nodes of chi u / eta h^2."""
    b = st.body
    u, v = velocity(st)
    chi = body_mask(st.N, b) / b.eta
    return np.array([(chi * u).sum(), (chi * v).sum()]) / (st.N * st.N)


def streamfunction(st: NSState) -> np.ndarray:
    lam = laplacian_eigenvalues(st.N)
    lam[0, 0] = 1.0
    ph = -st.omega_hat / lam
    ph[0, 0] = 0.0
    return np.real(np.fft.ifft2(ph))


def omega(st: NSState) -> np.ndarray:
    return np.real(np.fft.ifft2(st.omega_hat))


def velocity(st: NSState, psi=None):
    """(u, v) at the nodes."""
    h = 1.0 / st.N
    psi = streamfunction(st) if psi is None else psi
    return st.U[0] + _dy(psi, h), st.U[1] - _dx(psi, h)


def curl_cells(Sx: np.ndarray, Sy: np.ndarray, h: float) -> np.ndarray:
    """curl of a cell-centred vector at the nodes: node (i, j) from cells
    (i-1, j-1), (i, j-1), (i-1, j), (i, j)."""
    sy_r = Sy + np.roll(Sy, 1, axis=0)                  # cells (i, j) + (i, j-1)
    dSy_dx = (sy_r - np.roll(sy_r, 1, axis=1)) / (2.0 * h)
    sx_t = Sx + np.roll(Sx, 1, axis=1)                  # cells (i, j) + (i-1, j)
    dSx_dy = (sx_t - np.roll(sx_t, 1, axis=0)) / (2.0 * h)
    return dSy_dx - dSx_dy


def face_velocities(st: NSState, psi: np.ndarray):
    """Normal velocity on the x-faces (x = i h, between cells i-1 and i) and
    the y-faces (y = j h), from psi at each face's two corner nodes."""
    N = st.N
    ux = st.U[0] + (np.roll(psi, -1, axis=0) - psi) * N   # corners (i, j), (i, j+1)
    vy = st.U[1] - (np.roll(psi, -1, axis=1) - psi) * N   # corners (i, j), (i+1, j)
    return ux, vy


def step(st: NSState, dt: float, S_mass=None, Sx=None, Sy=None, nsub: int = 1) -> NSState:
    """nsub steps of dt with the droplet sources (cell arrays, per unit volume;
    None for zero) held fixed."""
    N = st.N
    h = 1.0 / N
    lam = laplacian_eigenvalues(N)
    z = np.zeros((N, N))
    Sm = z if S_mass is None else np.asarray(S_mass, np.float64).reshape(N, N)
    Sx = z if Sx is None else np.asarray(Sx, np.float64).reshape(N, N)
    Sy = z if Sy is None else np.asarray(Sy, np.float64).reshape(N, N)
    curl = curl_cells(Sx, Sy, h)
    mean_S = np.array([Sx.mean(), Sy.mean()])
    b = st.body
    if b is not None:
        chi = body_mask(N, b) / b.eta
        sig = fringe(N, b)
        if b.hold_mean_flow:
            mean_S = np.zeros(2)
    for _ in range(nsub):
        psi = streamfunction(st)
        u, v = velocity(st, psi)
        w = omega(st)
        R = -(u * _dx(w, h) + v * _dy(w, h)) + curl
        if b is not None:   # curl of -chi u / eta, and the fringe's relaxation
            R += -(_dx(chi * v, h) - _dy(chi * u, h)) - sig * w
        # vapour: upwind fluxes on the faces, diffusion, source
        ux, vy = face_velocities(st, psi)
        rho = st.rho
        Fx = np.where(ux > 0, ux * np.roll(rho, 1, axis=1), ux * rho)   # face i: cells i-1 | i
        Fy = np.where(vy > 0, vy * np.roll(rho, 1, axis=0), vy * rho)
        div = (np.roll(Fx, -1, axis=1) - Fx + np.roll(Fy, -1, axis=0) - Fy) / h
        st.rho = rho + dt * (-div + st.D * lap5(rho, h) + Sm)
        oh = (st.omega_hat + dt * np.fft.fft2(R)) / (1.0 - dt * st.nu * lam)
        oh[0, 0] = 0.0
        st.omega_hat = oh
        if b is not None and not b.hold_mean_flow:   # the mean of the penalisation force
            st.U = st.U + dt * (mean_S - np.array([(chi * u).mean(), (chi * v).mean()]))
        else:
            st.U = st.U + dt * mean_S
        st.t += dt
    return st


def carrier_nodes(st: NSState) -> np.ndarray:
    """u, v, grad u at the (N+1)^2 mesh nodes: ((N+1)^2, 8) in the layout of
    the analytic carriers' node arrays (u, v, du/dx, du/dy, dv/dx, dv/dy, 0, 0)."""
    N = st.N
    h = 1.0 / N
    u, v = velocity(st)
    vals = [u, v, _dx(u, h), _dy(u, h), _dx(v, h), _dy(v, h)]
    out = np.zeros(((N + 1) * (N + 1), 8))
    jj, ii = np.meshgrid(np.arange(N + 1) % N, np.arange(N + 1) % N, indexing="ij")
    for q, f in enumerate(vals):
        out[:, q] = f[jj, ii].ravel()
    return out


def taylor_green_omega(N: int, amp: float = 1.0) -> np.ndarray:
    """Nodal vorticity of psi = amp sin(2 pi x) sin(2 pi y) / (2 pi) under the
    discrete operator: omega = -Lap_h psi (a discrete eigenfunction)."""
    x = np.arange(N) / N
    psi = amp * np.sin(2 * np.pi * x)[None, :] * np.sin(2 * np.pi * x)[:, None] / (2 * np.pi)
    return -lap5(psi, 1.0 / N)
