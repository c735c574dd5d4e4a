"""Pins of the two-way carrier oracle (oracle/carrier_ns.py): Eq. 1 in
vorticity-streamfunction form with the droplets' momentum source and Eq. 2
with their mass source, checked against what the discretisation and the
mathematics fix -- discrete eigenfunctions, exact invariants, closed forms and
convergence orders -- not against itself."""
import numpy as np
import pytest

from oracle import carrier_ns as NS


def _random_state(N, seed, nu=1e-3, D=1e-3):
    rng = np.random.default_rng(seed)
    k = np.fft.fftfreq(N, 1.0 / N)
    spec = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) * np.exp(
        -(k[:, None] ** 2 + k[None, :] ** 2) / 8.0)
    w = np.real(np.fft.ifft2(spec)) * N
    rho = 1.0 + 0.5 * rng.standard_normal((N, N))
    return NS.init(N, nu, D, w, U=(0.3, -0.2), rho=rho)


def test_poisson_solve_inverts_the_five_point_laplacian():
    """-Lap_h psi = omega, the stencil applied in physical space."""
    st = _random_state(32, 1)
    psi = NS.streamfunction(st)
    w = NS.omega(st)
    assert np.abs(-NS.lap5(psi, 1.0 / 32) - w).max() <= 1e-10 * np.abs(w).max()
    assert abs(psi.mean()) < 1e-14


def test_laplacian_eigenvalues_are_the_stencil_symbols():
    N = 16
    lam = NS.laplacian_eigenvalues(N)
    x = np.arange(N) / N
    for kx, ky in ((1, 0), (3, 5), (8, 8), (2, 13)):
        f = np.cos(2 * np.pi * (kx * x[None, :] + ky * x[:, None]))
        assert np.allclose(NS.lap5(f, 1.0 / N), lam[ky, kx] * f, atol=1e-9 * abs(lam[ky, kx]))


def test_face_velocities_are_divergence_free_and_node_gradient_trace_free():
    st = _random_state(24, 2)
    psi = NS.streamfunction(st)
    ux, vy = NS.face_velocities(st, psi)
    div = (np.roll(ux, -1, axis=1) - ux + np.roll(vy, -1, axis=0) - vy) * 24
    assert np.abs(div).max() <= 1e-11 * np.abs(ux).max() * 24
    nodes = NS.carrier_nodes(st)
    assert np.abs(nodes[:, 2] + nodes[:, 5]).max() <= 1e-10 * np.abs(nodes[:, 2:6]).max()
    # the periodic node N repeats node 0
    g = nodes.reshape(25, 25, 8)
    assert np.array_equal(g[24], g[0]) and np.array_equal(g[:, 24], g[:, 0])


def test_discrete_taylor_green_decays_at_the_discrete_rate():
    """psi = sin(2 pi x) sin(2 pi y) / (2 pi) is an eigenfunction of Lap_h, the
    advection term vanishes identically, and the implicit step divides omega by
    (1 - dt nu lambda) exactly."""
    N, nu, dt, n = 32, 0.01, 2e-3, 25
    w0 = NS.taylor_green_omega(N)
    st = NS.init(N, nu, 0.0, w0)
    NS.step(st, dt, nsub=n)
    lam = NS.laplacian_eigenvalues(N)[1, 1]
    expect = w0 / (1.0 - dt * nu * lam) ** n
    assert np.abs(NS.omega(st) - expect).max() <= 1e-11 * np.abs(w0).max()


def test_taylor_green_rate_converges_to_the_continuum_at_second_order():
    """-lambda_(1,1) -> 8 pi^2 with an error ratio of 4 per mesh doubling."""
    err = [abs(-NS.laplacian_eigenvalues(N)[1, 1] - 8 * np.pi ** 2) for N in (16, 32, 64)]
    assert err[0] / err[1] == pytest.approx(4.0, rel=0.05)
    assert err[1] / err[2] == pytest.approx(4.0, rel=0.05)


def test_uniform_momentum_source_accelerates_the_mean_flow_only():
    """A uniform source has no curl: it moves U by n dt S exactly, and with
    U = 0 and a vorticity-free start (omega = 0) the flow stays uniform."""
    N, dt, n = 16, 1e-3, 30
    st = _random_state(N, 3)
    U0 = st.U.copy()
    Sx = np.full((N, N), 0.7)
    Sy = np.full((N, N), -0.4)
    assert np.abs(NS.curl_cells(Sx, Sy, 1.0 / N)).max() < 1e-10
    NS.step(st, dt, Sx=Sx, Sy=Sy, nsub=n)
    assert np.allclose(st.U, U0 + n * dt * np.array([0.7, -0.4]), rtol=0, atol=1e-14)
    calm = NS.init(N, 1e-3, 0.0, np.zeros((N, N)))
    NS.step(calm, dt, Sx=Sx, Sy=Sy, nsub=n)
    nodes = NS.carrier_nodes(calm)
    assert np.allclose(nodes[:, 0], n * dt * 0.7, atol=1e-14) and np.allclose(nodes[:, 1], -n * dt * 0.4, atol=1e-14)
    assert np.abs(nodes[:, 2:6]).max() == 0.0


def test_curl_of_cell_source_converges_at_second_order():
    """S = (-sin 2 pi y, sin 2 pi x) at the cell centres: curl = 2 pi (cos 2 pi x
    + cos 2 pi y) at the nodes."""
    errs = []
    for N in (16, 32, 64):
        c = (np.arange(N) + 0.5) / N
        n_ = np.arange(N) / N
        Sx = -np.sin(2 * np.pi * c)[:, None] * np.ones((1, N))
        Sy = np.sin(2 * np.pi * c)[None, :] * np.ones((N, 1))
        curl = NS.curl_cells(Sx, Sy, 1.0 / N)
        exact = 2 * np.pi * (np.cos(2 * np.pi * n_)[None, :] + np.cos(2 * np.pi * n_)[:, None])
        errs.append(np.abs(curl - exact).max())
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.1)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.1)


def test_vapour_mass_changes_exactly_by_the_source():
    N, dt, n = 24, 1e-3, 40
    st = _random_state(N, 4, D=2e-3)
    rng = np.random.default_rng(5)
    Sm = rng.uniform(0.0, 2.0, (N, N))
    m0 = st.rho.sum()
    NS.step(st, dt, S_mass=Sm, nsub=n)
    assert st.rho.sum() == pytest.approx(m0 + n * dt * Sm.sum(), rel=1e-13, abs=1e-10)


def test_uniform_vapour_stays_uniform_in_any_flow():
    N = 20
    st = _random_state(N, 6, D=1e-3)
    st.rho = np.full((N, N), 2.5)
    NS.step(st, 1e-3, nsub=30)
    assert np.abs(st.rho - 2.5).max() <= 1e-12


def test_upwind_advection_keeps_vapour_bounded():
    """Monotone transport: with no source and dt |u| / h < 1, 4 D dt / h^2 < 1,
    the vapour stays within its initial range."""
    N = 32
    st = _random_state(N, 7, D=5e-4)
    st.rho = np.clip(st.rho, 0.0, None)
    lo, hi = st.rho.min(), st.rho.max()
    u, v = NS.velocity(st)
    dt = 0.2 / (N * (np.abs(u).max() + np.abs(v).max()))
    NS.step(st, dt, nsub=20)
    assert st.rho.min() >= lo - 1e-12 and st.rho.max() <= hi + 1e-12


def test_velocity_is_the_curl_of_the_streamfunction():
    """u = d psi/dy, v = -d psi/dx: the Taylor-Green field's velocity at (1/4, 0)
    is (+1, 0) up to the central difference's sin(2 pi h)/(2 pi h), and the
    curl of the nodal velocity approaches omega at second order."""
    errs = []
    for N in (16, 32, 64):
        st = NS.init(N, 1e-3, 0.0, NS.taylor_green_omega(N))
        nodes = NS.carrier_nodes(st).reshape(N + 1, N + 1, 8)
        h = 1.0 / N
        assert nodes[0, N // 4, 0] == pytest.approx(np.sin(2 * np.pi * h) / (2 * np.pi * h), rel=1e-12)
        assert abs(nodes[0, N // 4, 1]) < 1e-12
        curl = (nodes[:N, :N, 4] - nodes[:N, :N, 3])         # dv/dx - du/dy
        w = NS.omega(st)
        errs.append(np.abs(curl - w).max() / np.abs(w).max())
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.1)


def test_vapour_diffuses_at_the_discrete_rate_in_still_fluid():
    """omega = 0, U = 0: a Fourier mode of rho is multiplied by (1 + dt D lambda)
    each step (explicit diffusion), lambda the 5-point Laplacian's eigenvalue."""
    N, D, dt, n = 16, 2e-3, 1e-3, 12
    c = (np.arange(N) + 0.5) / N
    rho0 = 3.0 + np.cos(2 * np.pi * (2 * c[None, :] + 1 * c[:, None]))
    st = NS.init(N, 1e-3, D, np.zeros((N, N)), rho=rho0)
    NS.step(st, dt, nsub=n)
    lam = NS.laplacian_eigenvalues(N)[1, 2]
    expect = 3.0 + (rho0 - 3.0) * (1.0 + dt * D * lam) ** n
    assert np.abs(st.rho - expect).max() <= 1e-12


def test_vorticity_is_carried_by_the_mean_flow():
    """omega = cos(2 pi k x) (no self-advection: its velocity is along y) in a
    mean flow U along x, nu = 0: each explicit step multiplies the mode by
    1 - i dt U sin(2 pi k h)/h (the central difference's symbol)."""
    N, k, U, dt, n = 32, 3, 0.8, 1e-3, 15
    x = np.arange(N) / N
    w0 = np.cos(2 * np.pi * k * x)[None, :] * np.ones((N, 1))
    st = NS.init(N, 0.0, 0.0, w0, U=(U, 0.0))
    NS.step(st, dt, nsub=n)
    g = (1.0 - 1j * dt * U * np.sin(2 * np.pi * k / N) * N) ** n
    expect = np.real(g * np.exp(2j * np.pi * k * x))[None, :] * np.ones((N, 1))
    assert np.abs(NS.omega(st) - expect).max() <= 1e-12


def test_advance_with_given_nodes_equals_the_sampled_carrier():
    """The oracle advance fed node values (as the two-way carrier feeds it)
    equals the advance that samples the same analytic carrier itself."""
    from oracle import oracle as O
    from paper_2512_20829_gb300 import inputs as I
    wl = I.taylor_green_2d(scale=4)
    nodes = O.carrier_nodes(wl.carrier, 0.0, wl.n_cells_axis)
    a = O.initial_state(wl.fla, 2)
    b = O.initial_state(wl.fla, 2)
    adv = O.Advancer(wl, wl.fla)
    adv.advance(a, 0, 30, reset_acc=True)
    adv.advance(b, 0, 30, reset_acc=True, nodes=nodes)
    assert np.array_equal(a.y, b.y) and np.array_equal(a.acc, b.acc) and np.array_equal(a.status, b.status)


# ----------------------------------------------------------------- immersed cylinder

def test_cylinder_mask_area_converges_at_second_order():
    b = NS.Body(xc=0.41, yc=0.47, R=0.13, eta=1e-3)
    errs = [abs(NS.body_mask(N, b).sum() / N ** 2 - np.pi * b.R ** 2) for N in (64, 128, 256)]
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.25)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.25)


def test_uniform_penalisation_damps_each_mode_in_closed_form():
    """chi = 1 everywhere: a single Fourier mode (no self-advection) is multiplied
    each step by (1 - dt g / eta)/(1 - dt nu lambda), g = (sin^2 2 pi k_x h +
    sin^2 2 pi k_y h) / (4 (sin^2 pi k_x h + sin^2 pi k_y h)) -- the wide-stencil
    curl of the velocity over the compact Laplacian -- and the force on the body
    is U / eta with the mean flow decelerating at the same rate."""
    N, kx, ky, nu, dt, eta, n = 32, 2, 3, 1e-3, 1e-3, 5e-3, 10
    x = np.arange(N) / N
    w0 = np.cos(2 * np.pi * (kx * x[None, :] + ky * x[:, None]))
    b = NS.Body(xc=0.5, yc=0.5, R=10.0, eta=eta, hold_mean_flow=False)
    assert np.all(NS.body_mask(N, b) == 1.0)
    st = NS.init(N, nu, 0.0, w0, U=(0.3, 0.0), body=b)
    F0 = NS.body_force(st)
    assert np.allclose(F0, [0.3 / eta, 0.0], rtol=1e-12, atol=1e-9)
    NS.step(st, dt, nsub=n)
    h = 1.0 / N
    g = (np.sin(2 * np.pi * kx * h) ** 2 + np.sin(2 * np.pi * ky * h) ** 2) / (
        4 * (np.sin(np.pi * kx * h) ** 2 + np.sin(np.pi * ky * h) ** 2))
    lam = NS.laplacian_eigenvalues(N)[ky, kx]
    # the mean-flow advection of a single mode rotates its phase; compare amplitudes
    amp = np.abs(np.fft.fft2(NS.omega(st))[ky, kx]) / (N * N / 2)
    assert amp == pytest.approx(((1 - dt * g / eta) / (1 - dt * nu * lam)) ** n, rel=1e-3)
    assert st.U[0] == pytest.approx(0.3 * (1 - dt / eta) ** n, rel=1e-12)


def test_fringe_relaxes_vorticity_in_its_strip_only():
    """omega = cos(2 pi k x) (velocity along y: no self-advection), nu = 0, U = 0:
    each step multiplies omega by 1 - dt sigma(x) at each node, then removes the
    mean; outside the strip only the mean removal acts."""
    N, k, dt, n = 32, 2, 1e-3, 8
    x = np.arange(N) / N
    w = np.cos(2 * np.pi * k * x)[None, :] * np.ones((N, 1))
    b = NS.Body(xc=-5.0, yc=-5.0, R=0.01, eta=1.0, x0=0.6, x1=0.9, sigma_max=40.0)
    assert NS.body_mask(N, b).max() < 1e-300
    sig = NS.fringe(N, b)
    assert sig[:, x < 0.6].max() == 0.0 and sig[:, x > 0.9].max() == 0.0
    assert sig.max() == pytest.approx(40.0 * np.sin(np.pi * (np.round(0.75 * N) / N - 0.6) / 0.3) ** 2)
    st = NS.init(N, 0.0, 0.0, w, body=b)
    for _ in range(n):
        w = w * (1 - dt * sig)
        w = w - w.mean()
    NS.step(st, dt, nsub=n)
    assert np.abs(NS.omega(st) - w).max() <= 1e-12
