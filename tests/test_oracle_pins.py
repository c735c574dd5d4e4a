"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Nothing here re-types an oracle formula: each check compares the oracle with a
closed-form solution, an integral identity, a symmetry, a library routine or a
brute-force alternative, chosen so that a dropped term, a wrong sign, a wrong
index or a transposed operand in the oracle fails at least one of them.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2512_20829_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _wl(dim=2, N=32, dt=1e-3, delta=-0.2, carrier=None, kernel=I.KERNEL_ISO, window=10):
    car = carrier or I.Carrier(kind=I.CARRIER_UNIFORM, dim=dim)
    dx = 1.0 / N
    return I.Workload(name="t", dim=dim, n_cells_axis=N, dt=dt, nsteps=0, window=window, delta=delta,
                      carrier=car, fla=None, lpt=None, kernel=kernel, h_min=0.5 * dx, h_max=4 * dx)


def _cloud(x0, St0, step_start=0, kind=I.CLOUD_FLA):
    x0 = np.atleast_2d(np.asarray(x0, float))
    n = x0.shape[0]
    return I.Cloud(kind=kind, x0=x0, batch=np.zeros(n, np.int32), step_start=np.array([step_start], np.int32),
                   St0=np.array([St0]), n0=np.array([1.0]), h0=np.array([0.05]))


# ---------------------------------------------------------------------------
# Carrier fields
# ---------------------------------------------------------------------------

def _carriers():
    rng = np.random.default_rng(7)
    jet = I.jet_vortex_2d(scale=8, lpt_per_batch=0).carrier
    jet.vortices[:, 3] = 0.05  # wider cores so central differences resolve them
    return [I.Carrier(kind=I.CARRIER_TAYLOR_GREEN_2D, dim=2), jet,
            I.Carrier(kind=I.CARRIER_ABC_JET_3D, dim=3)], rng


def test_carrier_gradient_is_jacobian_of_velocity():
    """G_ij = du_i/dx_j against central differences of u (Eq. 8 needs grad u)."""
    cars, rng = _carriers()
    eps = 1e-6
    for car in cars:
        d = car.dim
        for _ in range(40):
            x = rng.uniform(0.05, 0.95, d)
            t = rng.uniform(0, 0.3)
            _, G = O.carrier_eval(car, t, x)
            Gfd = np.zeros((d, d))
            for j in range(d):
                e = np.zeros(d); e[j] = eps
                up, _ = O.carrier_eval(car, t, x + e)
                um, _ = O.carrier_eval(car, t, x - e)
                Gfd[:, j] = (up - um) / (2 * eps)
            scale = max(1.0, np.abs(G).max())
            assert np.abs(G - Gfd).max() < 2e-6 * scale, (car.kind, x, G, Gfd)


def test_carriers_are_divergence_free():
    """The carrier of Eq. 1 is incompressible: tr(grad u) = 0."""
    cars, rng = _carriers()
    for car in cars:
        for _ in range(50):
            x = rng.uniform(0, 1, car.dim)
            _, G = O.carrier_eval(car, 0.1, x)
            assert abs(np.trace(G)) < 1e-12 * max(1.0, np.abs(G).max())


def test_lamb_oseen_circulation():
    """Stokes: the circulation of one Lamb-Oseen vortex inside radius R is
    Gamma (1 - exp(-R^2/rc^2)); integrate the oracle velocity round a circle."""
    for gam, rc, R in [(0.4, 0.02, 0.01), (-0.3, 0.02, 0.03), (0.5, 0.05, 0.08)]:
        car = I.Carrier(kind=I.CARRIER_JET_VORTEX_2D, dim=2, vortices=np.array([[0.5, 0.5, gam, rc, 0.0]]),
                        jet_width=1e-9)  # jet switched off (zero width: exp(-inf) = 0 away from y = 0.5)
        m = 2000
        th = (np.arange(m) + 0.5) * 2 * math.pi / m
        circ = 0.0
        for a in th:
            x = np.array([0.5 + R * math.cos(a), 0.5 + R * math.sin(a) + 0.0])
            u, _ = O.carrier_eval(car, 0.0, x)
            circ += (u[0] * -math.sin(a) + u[1] * math.cos(a)) * R * (2 * math.pi / m)
        # the two far images at x +- 1 add a small circulation-free field: subtract none, bound it
        assert circ == pytest.approx(gam * (1 - math.exp(-R * R / (rc * rc))), rel=1e-6, abs=1e-9)


def test_interpolation_exact_for_linear_and_second_order_for_smooth():
    """Bilinear/trilinear interpolation reproduces linear fields and converges as dx^2."""
    rng = np.random.default_rng(3)
    for d in (2, 3):
        A = rng.standard_normal((d, d)); A -= np.eye(d) * np.trace(A) / d
        car = I.Carrier(kind=I.CARRIER_LINEAR, dim=d, U=np.r_[rng.standard_normal(d), np.zeros(3 - d)],
                        A=A, xref=np.r_[rng.uniform(size=d), np.zeros(3 - d)])
        N = 8
        nodes = O.carrier_nodes(car, 0.0, N)
        for _ in range(20):
            x = rng.uniform(-0.01, 1.01, d)  # includes slight extrapolation past the edge
            u, G = O.interp(nodes, d, N, x)
            ua, Ga = O.carrier_eval(car, 0.0, x)
            assert np.allclose(u, ua, atol=1e-13) and np.allclose(G, Ga, atol=1e-13)
    car = I.Carrier(kind=I.CARRIER_TAYLOR_GREEN_2D, dim=2)
    xs = rng.uniform(0, 1, (200, 2))
    errs = []
    for N in (16, 32, 64):
        nodes = O.carrier_nodes(car, 0.0, N)
        errs.append(max(np.abs(O.interp(nodes, 2, N, x)[0] - O.carrier_eval(car, 0, x)[0]).max() for x in xs))
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


# ---------------------------------------------------------------------------
# Advance: closed forms (Eqs. 3, 4, 5, 8)
# ---------------------------------------------------------------------------

def _active_state(wl, x0, v0):
    cl = _cloud(x0, 1.0)
    st = O.initial_state(cl, wl.dim)
    d = wl.dim
    st.y[:, d:2 * d] = v0
    st.y[:, 2 * d:2 * d + d * d] = np.eye(d).ravel()
    st.status[:] = O.ACTIVE
    return st


@pytest.mark.parametrize("delta", [0.0, -0.2])
def test_uniform_flow_drag_relaxation_closed_form(delta):
    """P1: in a uniform stream, w = v - U obeys w' = -w/(St0 (1 + delta t)), so
    w = w0 (1 + delta t)^(-1/(St0 delta))  (-> e^{-t/St0} as delta -> 0), and x is its integral.
    J stays I and W stays 0 because grad u = 0."""
    U = np.array([0.3, -0.1])
    car = I.Carrier(kind=I.CARRIER_UNIFORM, dim=2, U=np.r_[U, 0.0])
    wl = _wl(carrier=car, delta=delta)
    St0 = 0.3
    x0 = np.array([0.2, 0.6]); v0 = np.array([-0.2, 0.4])
    st = _active_state(wl, x0, v0)
    st.St0 = None
    cl = _cloud(x0, St0)
    adv = O.Advancer(wl, cl, use_mesh=True)
    nsteps = 400
    adv.advance(st, 0, nsteps, reset_acc=True)
    T = nsteps * wl.dt
    w0 = v0 - U
    if delta == 0.0:
        w = w0 * math.exp(-T / St0)
        xint = w0 * St0 * (1 - math.exp(-T / St0))
    else:
        al = 1.0 / (St0 * delta)
        w = w0 * (1 + delta * T) ** (-al)
        xint = w0 * ((1 + delta * T) ** (1 - al) - 1) / (delta * (1 - al))
    assert np.allclose(st.v[0], U + w, rtol=0, atol=1e-11)
    assert np.allclose(st.x[0], x0 + U * T + xint, rtol=0, atol=1e-11)
    assert np.array_equal(st.J[0], np.eye(2)) and np.array_equal(st.W[0], np.zeros((2, 2)))


def test_window_sums_match_mass_and_momentum_change():
    """P11: mdot = dm/dt and F + mdot v = d(m v)/dt (Eq. 9 with F = m x''), so the
    window sums approach m(T) - m(0) and m(T)v(T) - m(0)v(0).  The left-rectangle
    rule of the substep sum leaves exactly the Euler-Maclaurin term -dt/2 [f]_0^T + O(dt^2)."""
    U = np.array([0.2, 0.1])
    car = I.Carrier(kind=I.CARRIER_UNIFORM, dim=2, U=np.r_[U, 0.0])
    delta = -0.2
    wl = _wl(carrier=car, delta=delta)
    St0 = 0.25
    x0 = np.array([0.3, 0.3]); v0 = np.array([0.5, -0.3])
    st = _active_state(wl, x0, v0)
    adv = O.Advancer(wl, _cloud(x0, St0), use_mesh=False)
    nsteps, dt = 300, wl.dt
    v_hist = [st.v[0].copy()]
    for _ in range(nsteps):   # record v at every step start to evaluate the boundary terms
        adv.advance(st, _, 1, reset_acc=False)
        v_hist.append(st.v[0].copy())
    T = nsteps * dt
    r = lambda t: math.sqrt(1 + delta * t)
    m = lambda t: r(t) ** 3
    mdot = lambda t: 1.5 * delta * r(t)
    dm = m(T) - m(0)
    assert st.acc[0, 0] - dm == pytest.approx(-dt / 2 * (mdot(T) - mdot(0)), rel=2e-2, abs=1e-12)
    dmv = m(T) * v_hist[-1] - m(0) * v_hist[0]
    f = lambda t, v: m(t) * (U - v) / (St0 * r(t) ** 2) + mdot(t) * v
    em = -dt / 2 * (f(T, v_hist[-1]) - f(0, v_hist[0]))
    assert np.allclose(st.acc[0, 1:] - dmv, em, rtol=2e-2, atol=1e-9)
    assert abs(st.acc[0, 0] - dm) < 1e-3 * abs(dm)


@pytest.mark.parametrize("use_mesh", [True, False])
def test_linear_shear_exact(use_mesh):
    """P2: u = (gamma (y - y_r), 0) with v0 = u(x0): the droplet moves with the
    flow, J = I + G t and det J = 1; RK4 is exact for this polynomial motion."""
    g = 1.7
    A = np.zeros((3, 3)); A[0, 1] = g
    car = I.Carrier(kind=I.CARRIER_LINEAR, dim=2, A=A, xref=np.array([0.0, 0.5, 0.0]))
    wl = _wl(carrier=car, delta=-0.2, N=16)
    x0 = np.array([[0.1, 0.55], [0.2, 0.45], [0.3, 0.5]])
    cl = _cloud(x0, 0.4)
    st = O.initial_state(cl, 2)
    adv = O.Advancer(wl, cl, use_mesh=use_mesh)
    adv.advance(st, 0, 250)
    T = 250 * wl.dt
    G = np.array([[0, g], [0, 0.0]])
    for i in range(3):
        assert np.allclose(st.x[i], [x0[i, 0] + g * (x0[i, 1] - 0.5) * T, x0[i, 1]], atol=1e-13)
        assert np.allclose(st.J[i], np.eye(2) + G * T, atol=1e-12)
        assert np.allclose(st.W[i], G, atol=1e-12)
        assert abs(np.linalg.det(st.J[i]) - 1) < 1e-12


@pytest.mark.parametrize("use_mesh", [True, False])
def test_linear_strain_through_fold_caustic(use_mesh):
    """P3: u = (a (x - 1/2), -a (y - 1/2)), delta = 0.  Each diagonal entry of J solves
    St q'' + q' -+ a q = 0 with q(0) = 1, q'(0) = +-a, and x - 1/2 = (x0 - 1/2) J_xx.
    With 4 a St > 1 the compressive entry oscillates, so det J crosses zero (a fold)."""
    a, St = 10.0, 1.0
    A = np.zeros((3, 3)); A[0, 0] = a; A[1, 1] = -a
    car = I.Carrier(kind=I.CARRIER_LINEAR, dim=2, A=A, xref=np.array([0.5, 0.5, 0.0]))
    wl = _wl(carrier=car, delta=0.0, N=16)
    x0 = np.array([[0.52, 0.6], [0.47, 0.35]])
    cl = _cloud(x0, St)
    st = O.initial_state(cl, 2)
    adv = O.Advancer(wl, cl, use_mesh=use_mesh)
    l1 = (-1 + math.sqrt(1 + 4 * a * St)) / (2 * St)
    l2 = (-1 - math.sqrt(1 + 4 * a * St)) / (2 * St)
    B = (a - l1) / (l2 - l1); Aq = 1 - B
    sig = 1 / (2 * St); om = math.sqrt(4 * a * St - 1) / (2 * St); C2 = (sig - a) / om
    dets = []
    for k in range(60):
        adv.advance(st, 10 * k, 10)
        t = 10 * (k + 1) * wl.dt
        q = Aq * math.exp(l1 * t) + B * math.exp(l2 * t)
        p = math.exp(-sig * t) * (math.cos(om * t) + C2 * math.sin(om * t))
        for i in range(2):
            assert np.allclose(st.J[i], np.diag([q, p]), atol=2e-10 * max(1, abs(q)))
            assert np.allclose(st.x[i] - 0.5, (x0[i] - 0.5) * np.array([q, p]), atol=1e-10)
        dets.append(np.linalg.det(st.J[0]))
    dets = np.array(dets)
    assert dets.max() > 0 and dets.min() < 0   # crossed the fold


def test_tracer_limit_keeps_det_near_one():
    """P4: as St -> 0 the droplets follow the divergence-free carrier, and Liouville
    gives det J -> 1; for small St, d ln det J/dt = div v = -St tr(G^2) + O(St^2),
    |tr G^2| <= 2 pi^2 in the Taylor-Green vortex."""
    car = I.Carrier(kind=I.CARRIER_TAYLOR_GREEN_2D, dim=2)
    res = []
    for St in (1e-2, 1e-3):
        wl = _wl(carrier=car, delta=0.0, dt=min(1e-3, St / 10))
        rng = np.random.default_rng(5)
        x0 = rng.uniform(0.2, 0.8, (8, 2))
        cl = _cloud(x0, St)
        st = O.initial_state(cl, 2)
        T = 0.1
        O.Advancer(wl, cl, use_mesh=False).advance(st, 0, int(round(T / wl.dt)))
        dev = np.abs(np.linalg.det(st.J) - 1).max()
        assert dev <= 2 * math.pi ** 2 * St * T * 1.05
        res.append(dev)
    assert res[1] < res[0] / 5


def _fd_check(car, St0, delta, x0, nsteps, window, dt=1e-3, eps=1e-6):
    d = car.dim
    wl = _wl(dim=d, carrier=car, delta=delta, dt=dt, window=window)
    def run(xs):
        cl = _cloud(xs, St0)
        st = O.initial_state(cl, d)
        adv = O.Advancer(wl, cl, use_mesh=False)
        s = 0
        while s < nsteps:
            k = min(window, nsteps - s)
            adv.advance(st, s, k)
            s += k
        return st
    base = run(x0)
    fd = np.zeros((x0.shape[0], d, d))
    for k in range(d):
        e = np.zeros(d); e[k] = eps
        fd[:, :, k] = (run(x0 + e).x - run(x0 - e).x) / (2 * eps)
    return base.J, fd


def test_jacobian_matches_finite_differences_of_trajectories():
    """P14: J = dx/dx0 (Eq. 7) against central differences of whole trajectories in x0,
    with the release rule v0 = u(x0) perturbed consistently (W(t0) = dv0/dx0).
    Covers the steady Taylor-Green vortex, the unsteady jet + vortices (carrier frozen
    per window) and the 3D ABC flow with a round jet."""
    rng = np.random.default_rng(11)
    jet = I.jet_vortex_2d(scale=8, lpt_per_batch=0).carrier
    cases = [(I.Carrier(kind=I.CARRIER_TAYLOR_GREEN_2D, dim=2), 0.5, -0.2, rng.uniform(0.3, 0.7, (4, 2)), 200),
             (jet, 0.8, -0.2, np.c_[rng.uniform(0.1, 0.3, 4), rng.uniform(0.45, 0.55, 4)], 200),
             (I.Carrier(kind=I.CARRIER_ABC_JET_3D, dim=3), 1.0, -0.2, rng.uniform(0.35, 0.65, (3, 3)), 100)]
    for car, St0, delta, x0, nsteps in cases:
        J, fd = _fd_check(car, St0, delta, x0, nsteps, window=10)
        scale = np.abs(J).max()
        assert np.abs(J - fd).max() < 1e-6 * max(1.0, scale), (car.kind, np.abs(J - fd).max())


def test_rk4_is_fourth_order():
    """P10: classical RK4 error falls 16x per halving of dt (Richardson ratio)."""
    car = I.Carrier(kind=I.CARRIER_TAYLOR_GREEN_2D, dim=2)
    x0 = np.array([[0.3, 0.4], [0.6, 0.55]])
    T = 0.4
    sols = []
    for dt in (0.02, 0.01, 0.005):
        wl = _wl(carrier=car, delta=-0.2, dt=dt)
        cl = _cloud(x0, 0.3)
        st = O.initial_state(cl, 2)
        O.Advancer(wl, cl, use_mesh=False).advance(st, 0, int(round(T / dt)))
        sols.append(st.y.copy())
    r = np.abs(sols[0] - sols[1]).max() / np.abs(sols[1] - sols[2]).max()
    assert 16 * 0.8 < r < 16 * 1.2, r


def test_release_schedule_and_domain_exit():
    """Seeds enter at their release step (earlier they stay pending and untouched) and
    a droplet that leaves [0,1]^d stops (outflow)."""
    car = I.Carrier(kind=I.CARRIER_UNIFORM, dim=2, U=np.array([1.0, 0.0, 0.0]))
    wl = _wl(carrier=car, delta=-0.2)
    cl = I.Cloud(kind=I.CLOUD_FLA, x0=np.array([[0.95, 0.5], [0.5, 0.5]]), batch=np.array([0, 1], np.int32),
                 step_start=np.array([0, 30], np.int32), St0=np.array([0.5, 0.5]), n0=np.ones(2), h0=np.ones(2))
    st = O.initial_state(cl, 2)
    adv = O.Advancer(wl, cl)
    adv.advance(st, 0, 29)
    assert st.status[1] == O.PENDING and np.array_equal(st.y[1, :2], [0.5, 0.5])
    adv.advance(st, 29, 40)
    assert st.status[1] == O.ACTIVE and st.x[1, 0] == pytest.approx(0.5 + 39 * wl.dt, abs=1e-12)
    assert st.status[0] == O.DEAD          # crossed x = 1 after ~50 steps


def test_evaporation_deadline_is_first_step_below_threshold():
    """The release stops at the first step s with 1 + delta (s - s0) dt < max(0.01, 4 dt/St0),
    checked in exact rational arithmetic (cases chosen away from exact ties, where the
    host's double-precision decision may legitimately fall on either side)."""
    for St0, delta, dt, s0 in [(0.5, -0.27, 1e-3, 0), (0.02, -2.3, 1e-3, 17), (2.0, -50.0, 1e-3, 5)]:
        s = O.step_dead(St0, delta, dt, s0)
        thr = max(Fraction(1, 100), 4 * Fraction(dt) / Fraction(St0))
        lhs = lambda k: 1 + Fraction(delta) * (k - s0) * Fraction(dt)
        assert lhs(s) < thr and not lhs(s - 1) < thr
    assert O.step_dead(0.5, 0.0, 1e-3, 0) == I.NO_DEADLINE


def test_taylor_green_point_symmetry_of_full_path():
    """P5: the Taylor-Green vortex is odd under (x, y) -> (1 - x, 1 - y) and the 64^2
    strip lattice is invariant, so the end-to-end sources satisfy
    S_mass(c') = S_mass(c) and S_mom(c') = -S_mom(c)."""
    wl = I.taylor_green_2d(scale=2)
    st = O.run(wl)
    D = O.dep_struct(wl)
    Sm, Sv, Ds = O.nw_deposit_celllist(D, st.x, st.J, st.acc, st.status, st.batch, wl.fla.n0, wl.fla.h0)
    N = wl.n_cells_axis
    Sm2, Sv2 = Sm.reshape(N, N), Sv.reshape(N, N, 2)
    assert np.abs(Sm2).max() > 0
    assert np.allclose(Sm2, Sm2[::-1, ::-1], rtol=1e-9, atol=1e-12 * np.abs(Sm2).max())
    assert np.allclose(Sv2, -Sv2[::-1, ::-1], rtol=1e-9, atol=1e-12 * np.abs(Sv2).max())


# ---------------------------------------------------------------------------
# Deposit: kernel regression (Eqs. 13-16) and PSI-CELL (Eqs. 10-11)
# ---------------------------------------------------------------------------

def test_nw_reproduces_constant_field_and_single_droplet():
    """P6: the NW estimator is a weighted mean, so a cloud with n a = const gives
    S = -const on every covered cell and 0 on uncovered cells, and one droplet gives
    S = -n a on its whole support (Eq. 13, signs of Eq. 9)."""
    s = I.synthetic_state(2, 300, 64, seed=1, edge_cases=False)
    D = O.dep_struct(dim=2, N=64, kernel=I.KERNEL_ISO, h_min=0.5 / 64, h_max=2 / 64, p=1.0, window_dt=0.01)
    detJ = np.abs(np.linalg.det(s.J.astype(np.float64)))
    K = np.array([2.0, -1.0, 0.5])
    acc = K[None, :] * detJ[:, None] / s.n0[s.batch][:, None] * 0.01
    Sm, Sv, Ds = O.nw_deposit(D, s.x, s.J, acc, s.status, s.batch, s.n0, s.h0)
    cov = Ds > 0
    assert cov.sum() > 100 and (~cov).sum() > 0
    assert np.allclose(Sm[cov], -K[0], rtol=1e-12) and np.allclose(Sv[cov], -K[1:], rtol=1e-12)
    assert np.all(Sm[~cov] == 0) and np.all(Sv[~cov] == 0)
    one = np.zeros_like(s.status); one[5] = 1
    Sm1, _, Ds1 = O.nw_deposit(D, s.x, s.J, acc * 3.0, one, s.batch, s.n0, s.h0)
    assert np.allclose(Sm1[Ds1 > 0], -3 * K[0], rtol=1e-12)


@pytest.mark.parametrize("d,N,kernel", [(2, 64, I.KERNEL_ISO), (3, 32, I.KERNEL_ISO), (2, 64, I.KERNEL_ANISO),
                                        (3, 32, I.KERNEL_ANISO)])
def test_kernel_normalisation_and_second_moment(d, N, kernel):
    """P7: sum_c V_c Khat(x_c - x_i) equals the Gaussian mass inside q <= 9,
    P(chi2_d <= 9) (1 - e^{-4.5} in 2D), and the second moment
    sum_c V_c Khat (x_c - x_i)(x_c - x_i)^T equals Sigma P(chi2_{d+2} <= 9),
    with Sigma = h^2 I (spherical, Eqs. 14-15) or h0^2 J J^T + h_min^2 I (J-scaled);
    a non-normal J tells J J^T from J^T J.  The paper's weight (prefactor 1/h)
    integrates to (2 pi)^{d/2} h^{d-1} times that mass."""
    dx = 1.0 / N
    D = O.dep_struct(dim=d, N=N, kernel=kernel, h_min=0.5 * dx, h_max=(12 if d == 2 else 5) * dx,
                     p=1.0, window_dt=1.0)
    x = np.full(d, 0.5) + 0.3 * dx
    if kernel == I.KERNEL_ISO:
        J = np.eye(d) * (1.0 if d == 2 else 1.0)
        h0 = (3.0 if d == 2 else 1.6) * dx
        Sigma = h0 ** 2 * np.eye(d)
    else:
        J = np.eye(d); J[0, 1] = 1.2; J[1, 0] = -0.3; J[d - 1, d - 1] = 1.3
        h0 = (2.5 if d == 2 else 1.0) * dx
        Sigma = h0 ** 2 * J @ J.T + (0.5 * dx) ** 2 * np.eye(d)
    w = O.kernel_on_cells(D, x, J, 1.0, h0, normalised=True)
    V = dx ** d
    idx = np.indices((N,) * d).reshape(d, -1)[::-1].T   # x fastest
    xc = (idx + 0.5) * dx
    dv = xc - x
    mass = V * w.sum()
    mom2 = V * np.einsum("c,ci,cj->ij", w, dv, dv)
    assert mass == pytest.approx(stats.chi2.cdf(9, d), abs=2.5e-3)
    assert np.allclose(mom2, Sigma * stats.chi2.cdf(9, d + 2), rtol=0, atol=1e-2 * np.abs(Sigma).max())
    raw = O.kernel_on_cells(D, x, J, 1.0, h0, normalised=False)
    if kernel == I.KERNEL_ISO:
        assert V * raw.sum() == pytest.approx((2 * math.pi) ** (d / 2) * h0 ** (d - 1) * stats.chi2.cdf(9, d),
                                              rel=2.5e-3)


def test_anisotropic_support_respects_trace_cap():
    """A strongly stretched J is scaled so that trace(Sigma) <= h_max^2, so no weight
    reaches past 3 h_max from the droplet, while the h_min^2 I floor keeps the thin
    directions wide enough to reach the nearest cell centres."""
    N = 32; dx = 1.0 / N
    D = O.dep_struct(dim=3, N=N, kernel=I.KERNEL_ANISO, h_min=0.5 * dx, h_max=2 * dx, p=1.0, window_dt=1.0)
    x = np.array([0.5, 0.5, 0.5])
    J = np.diag([30.0, 0.2, 1.0]); J[0, 2] = 5.0
    w = O.kernel_on_cells(D, x, J, 1.0, 2 * dx, normalised=False)
    idx = np.indices((N,) * 3).reshape(3, -1)[::-1].T
    dist = np.linalg.norm((idx + 0.5) * dx - x, axis=1)
    assert w.max() > 0 and dist[w > 0].max() <= 3 * 2 * dx + 1e-12


@pytest.mark.parametrize("d,kernel,fp32", [(2, I.KERNEL_ISO, False), (2, I.KERNEL_ISO, True),
                                           (3, I.KERNEL_ANISO, False), (3, I.KERNEL_ANISO, True),
                                           (2, I.KERNEL_ANISO, True), (3, I.KERNEL_ISO, True)])
def test_cell_list_equals_brute_force_bitwise(d, kernel, fp32):
    """P9: the cell-list deposit visits exactly the droplets the brute force would
    include and sums them in the same ascending order, so both agree bit for bit."""
    N = 16
    s = I.synthetic_state(d, 64 if d == 2 else 96, N, seed=4 + d, h0_cells=1.5)
    D = O.dep_struct(dim=d, N=N, kernel=kernel, h_min=0.5 / N, h_max=3.0 / N, p=1.0, window_dt=0.01,
                     fp32_decision=fp32)
    a = O.nw_deposit(D, s.x, s.J, s.acc, s.status, s.batch, s.n0, s.h0)
    b = O.nw_deposit_celllist(D, s.x, s.J, s.acc, s.status, s.batch, s.n0, s.h0)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    assert (a[2] > 0).sum() > 20


def test_records_number_density_invariant():
    """P12: n |det J| = n0 for every seed (Eq. 6), the n floor only at |det J| < 1e-12,
    and h = h0 |det J| clamped to [h_min, h_max] (Eq. 15)."""
    s = I.synthetic_state(2, 200, 32, seed=9)
    D = O.dep_struct(dim=2, N=32, kernel=I.KERNEL_ISO, h_min=0.5 / 32, h_max=4 / 32, p=1.0, window_dt=0.01)
    J = s.J.astype(np.float64)
    J[0] = [[1.0, 2.0], [0.5, 1.0]]            # singular: det = 0
    r = O.records(D, s.x, J, s.acc, s.batch, s.n0, s.h0)
    det = np.linalg.det(J)
    ok = np.abs(det) > 1e-9
    assert np.allclose(r[ok, 0] * np.abs(det[ok]), s.n0[s.batch][ok], rtol=1e-12)
    assert r[0, 0] == pytest.approx(s.n0[s.batch[0]] / 1e-12)
    h = np.clip(s.h0[s.batch] * np.abs(det), 0.5 / 32, 4 / 32)
    assert np.allclose(r[:, 2], h, rtol=1e-12)


def test_cell_keys_sort_and_bins_against_library():
    """Cell keys: floor(x N) clamped to N - 1, x fastest, inactive or outside the
    domain -> 0xFFFFFFFF; the cell list is NumPy's stable argsort and searchsorted."""
    for d, N in ((2, 64), (3, 16)):
        s = I.synthetic_state(d, 5000, N, seed=21)
        x = s.x.astype(np.float64)
        x[:3] = -1e-3   # outside
        keys = O.cell_keys(d, N, x, s.status, fp32=True)
        c = np.minimum(np.floor(s.x.astype(np.float32) * np.float32(N)).astype(np.int64), N - 1)
        lin = sum(c[:, a] * N ** a for a in range(d))
        inside = np.all((x >= 0) & (x <= 1), axis=1) & (s.status == 1)
        ref = np.where(inside, lin, 0xFFFFFFFF).astype(np.uint32)
        assert np.array_equal(keys, ref)
        sk, perm, bins = O.sort_and_bins(keys, N ** d)
        assert np.all(np.diff(sk.astype(np.int64)) >= 0)
        for cc in np.random.default_rng(0).integers(0, N ** d, 50):
            members = np.nonzero(keys == cc)[0]
            assert np.array_equal(perm[bins[cc]:bins[cc + 1]], members)


def test_psicell_conserves_totals():
    """P8: box counting puts every parcel in exactly one cell, so
    sum_c S_c V_c = -sum_i w_i a_i and sum_c count_c = #active parcels in the domain."""
    for d, N in ((2, 32), (3, 16)):
        s = I.synthetic_state(d, 4000, N, seed=8)
        D = O.dep_struct(dim=d, N=N, kernel=0, h_min=0, h_max=1, p=1.0, window_dt=0.01)
        w = np.array([1e-4, 2e-4, 3e-4, 4e-4])
        counts, Sm, Sv = O.psicell(D, s.x, s.acc, s.status, s.batch, w, fp32_keys=True)
        act = s.status == 1
        V = (1.0 / N) ** d
        wi = w[s.batch]
        assert counts.sum() == act.sum()
        assert np.array_equal(counts, np.bincount(O.cell_keys(d, N, s.x, s.status, True)[act], minlength=N ** d))
        a = s.acc.astype(np.float64) / 0.01
        assert (Sm * V).sum() == pytest.approx(-(wi * a[:, 0])[act].sum(), rel=1e-12)
        assert np.allclose((Sv * V).sum(0), -(wi[:, None] * a[:, 1:])[act].sum(0), rtol=1e-12)


def test_oracle_threads_do_not_change_results():
    """The oracle's OpenMP loops (droplets of a step, cells of a deposit) compute
    each droplet and cell with the same sequential code: one thread and all
    threads give identical bits."""
    wl = I.jet_vortex_2d(scale=16, nsteps=120, lpt_per_batch=0)
    out = []
    nthreads = O.threads()
    try:
        for t in (1, max(nthreads, 2)):
            O.set_threads(t)
            st = O.run(wl)
            D = O.dep_struct(wl)
            src = O.nw_deposit_celllist(D, st.x, st.J, st.acc, st.status, st.batch, wl.fla.n0, wl.fla.h0)
            brute = O.nw_deposit(D, st.x, st.J, st.acc, st.status, st.batch, wl.fla.n0, wl.fla.h0)
            out.append((st.y.copy(), st.acc.copy(), src, brute))
    finally:
        O.set_threads(nthreads)
    (y1, a1, s1, b1), (y2, a2, s2, b2) = out
    assert np.array_equal(y1, y2) and np.array_equal(a1, a2)
    for u, v in zip(s1 + b1, s2 + b2):
        assert np.array_equal(u, v)
    for u, v in zip(s1, b1):   # pin P9 at this size too: cell list == brute force
        assert np.array_equal(u, v)


# ---------------------------------------------------------------------------
# The single-precision truncation decision (fp32_decision) against q <= 9 in
# double.  The GPU's single-precision kernels decide whether a pair is inside
# the 3-sigma support on single-precision operands, and the parity tests give
# the oracle the same decision.  These pins tie that mode to the decision in
# double: every pair on which the two differ must lie within a rounding bound
# of q = 9 derived from the unit roundoff u = 2^-24 and the operand sizes, and
# the sources may differ only by the weights of those pairs.
#
# Bounds (first order in u).  Positions and cell centres in [0, 1] round with
# absolute error <= u/2 each and their difference adds u |dx|: eps = u (1 + |dx|)
# per coordinate.
#   spherical: q = r^2/h^2 against r2max = 9 h^2.  r^2 from the rounded
#     differences (d multiply-adds) is off by <= 2 sqrt(d) |r| eps + d u r^2;
#     r2max (h rounded, 9 h^2 rounded) by <= 9 h^2 (3u + 2 rho), rho the relative
#     error of |det J| in the decision: 0 in 2D (double from the given J), and in
#     3D <= 5u H / |det J| <= 500 u where the single-precision cofactor expansion
#     is used (only while |det J| >= 1e-2 H, H the product of the rows' L1 norms).
#     At r = 3 h:  |q - 9| <= 6 sqrt(d) eps / h + 9 d u + 27 u + 18 rho.
#   J-scaled: q = d^T P d with P the single-precision inverse of Sigma, whose
#     condition number is at most tr(Sigma) / h_min^2 <= h_max^2 / h_min^2 = kappa:
#     |P_f - P| <= 20 kappa u |P|; the position term is 2 |P d| eps sqrt(d) with
#     |P d| <= 3 / h_min at q = 9; the products and sums add 2 d u q:
#     |q - 9| <= 9 (20 kappa + 2 d) u + 6 sqrt(d) eps / h_min.
U32 = 2.0 ** -24


def _double_state(dim, n, N, seed, h0_cells, fold_frac):
    """A synthetic state with double-precision positions and Jacobians (so that
    the single-precision operands really are rounded), a fraction of them close
    to a fold: J = R diag(s1, s2[, s3]) R' with the smallest singular value
    1e-4..1e-2 of the largest."""
    s = I.synthetic_state(dim, n, N, seed=seed, band=(0.4, 0.6), h0_cells=h0_cells, jac_spread=0.3)
    rng = np.random.default_rng(seed + 100)
    x = s.x.astype(np.float64) + rng.uniform(-0.5, 0.5, s.x.shape) * 2.0 ** -26
    J = s.J.astype(np.float64) * (1.0 + 1e-7 * rng.standard_normal(s.J.shape))
    k = rng.uniform(size=n) < fold_frac
    m = int(k.sum())
    Q1 = np.linalg.qr(rng.standard_normal((m, dim, dim)))[0]
    Q2 = np.linalg.qr(rng.standard_normal((m, dim, dim)))[0]
    sv = np.exp(rng.uniform(-0.3, 0.3, (m, dim)))
    sv[:, -1] = sv[:, 0] * 10.0 ** rng.uniform(-4, -2, m)
    J[k] = np.einsum("nij,nj,nkj->nik", Q1, sv, Q2)
    return x, J, s


def _audit(dim, kernel, N, n, hmax_cells, h0_cells, ncells, seed):
    x, J, s = _double_state(dim, n, N, seed, h0_cells, fold_frac=0.2)
    h_min, h_max = 0.5 / N, hmax_cells / N
    kw = dict(dim=dim, N=N, kernel=kernel, h_min=h_min, h_max=h_max, p=1.0, window_dt=0.01)
    D32 = O.dep_struct(fp32_decision=True, **kw)
    D64 = O.dep_struct(fp32_decision=False, **kw)
    rng = np.random.default_rng(seed)
    band = np.arange(int(0.42 * N), int(0.58 * N))
    cells = rng.integers(0, N, (ncells, dim))
    cells[:, -1] = rng.choice(band, ncells)
    lin = cells[:, 0] + N * cells[:, 1] + (N * N * cells[:, 2] if dim == 3 else 0)
    lin = np.unique(lin)
    oc, od, oq, found, inside = O.decision_audit(D32, x, J, s.acc, s.status, s.batch, s.n0, s.h0, lin)
    eps = U32 * (1.0 + 3.0 * h_max * np.sqrt(dim))
    if kernel == I.KERNEL_ISO:
        rho = 0.0 if dim == 2 else 500.0 * U32
        rec = O.records(D64, x, J, s.acc, s.batch, s.n0, s.h0)     # n, det J, h, pref per droplet
        h = rec[od, 2]
        bound = 6 * np.sqrt(dim) * eps / h + 9 * dim * U32 + 27 * U32 + 18 * rho
    else:
        kappa = h_max ** 2 / h_min ** 2
        bound = np.full(len(oq), 9 * (20 * kappa + 2 * dim) * U32 + 6 * np.sqrt(dim) * eps / h_min)
    return dict(x=x, J=J, s=s, D32=D32, D64=D64, cells=lin, oc=oc, od=od, oq=oq, found=found, inside=inside,
                bound=bound)


def _check_sources(a):
    """Per cell: the two decisions' sources differ by at most the flipped pairs'
    weights (w = pref exp(-q/2) at q near 9) times |a_i| + |S_c|, over D_c."""
    s, x, J, lin = a["s"], a["x"], a["J"], a["cells"]
    m32, v32, d32 = O.nw_deposit_celllist(a["D32"], x, J, s.acc, s.status, s.batch, s.n0, s.h0, cells=lin)
    m64, v64, d64 = O.nw_deposit_celllist(a["D64"], x, J, s.acc, s.status, s.batch, s.n0, s.h0, cells=lin)
    rec = O.records(a["D64"], x, J, s.acc, s.batch, s.n0, s.h0)
    n_i, pref = rec[:, 0], rec[:, 3]
    am = np.abs(n_i * s.acc[:, 0] / 0.01)
    av = np.abs(n_i[:, None] * s.acc[:, 1:] / 0.01).max(axis=1)
    w = pref[a["od"]] * np.exp(-0.5 * a["oq"])
    jm = np.zeros(len(lin))
    jv = np.zeros(len(lin))
    jd = np.zeros(len(lin))
    np.add.at(jd, a["oc"], w)
    np.add.at(jm, a["oc"], w * (am[a["od"]] + np.abs(m64[a["oc"]])))
    np.add.at(jv, a["oc"], w * (av[a["od"]] + np.abs(v64[a["oc"]]).max(axis=1)))
    dmin = np.maximum(np.minimum(d32, d64), 1e-300)
    tol = 1e-12 * (np.abs(m64) + 1.0)
    assert np.all(np.abs(d32 - d64) <= jd * (1 + 1e-9) + 1e-12 * d64)
    assert np.all(np.abs(m32 - m64) <= jm / dmin * (1 + 1e-6) + tol)
    assert np.all(np.abs(v32 - v64).max(axis=1) <= jv / dmin * (1 + 1e-6) + tol)
    return int((a["oc"] >= 0).sum())


@pytest.mark.parametrize("dim,kernel,N,n,hmax,h0,ncells", [
    (2, I.KERNEL_ISO, 512, 262_144, 4.0, 2.0, 20_000),
    (3, I.KERNEL_ISO, 64, 262_144, 2.0, 1.2, 4_000),
    (3, I.KERNEL_ANISO, 128, 2_097_152, 2.0, 0.45, 2_000),
])
def test_single_precision_decision_within_rounding_of_q9(dim, kernel, N, n, hmax, h0, ncells):
    a = _audit(dim, kernel, N, n, hmax, h0, ncells, seed=41 + 3 * dim + kernel)
    print(f"\n{dim}D kernel {kernel}: {a['found']} of {a['inside']} pairs decided differently; "
          f"max |q - 9| {np.abs(a['oq'] - 9).max() if a['found'] else 0:.2e}, bound "
          f"{a['bound'].min() if a['found'] else 0:.2e}..{a['bound'].max() if a['found'] else 0:.2e}")
    assert a["inside"] > 100 * len(a["cells"])
    assert a["found"] == len(a["oq"])                       # all recorded
    assert np.all(np.abs(a["oq"] - 9.0) <= a["bound"]), np.abs(a["oq"] - 9.0).max()
    assert a["found"] <= 1e-3 * a["inside"]
    _check_sources(a)


def test_decision_audit_detects_a_single_precision_det_near_folds():
    """The audit separates a right decision from a wrong one.  Droplets with large,
    ill-conditioned J (singular values 40, 40, 1/1600: |det J| = 1, so h is not
    clamped, while the rows' L1 norms multiply to ~3e5) have a single-precision
    cofactor det J off by up to ~10 %.  The mixed mode switches to double there
    (|det J| < 1e-2 H) and stays within the bound; deciding with the
    single-precision det J -- what a wrong threshold would do, and what the plain
    mode does by design -- moves pairs far outside it."""
    N, n = 32, 32_768
    x, J, s = _double_state(3, n, N, seed=13, h0_cells=1.2, fold_frac=0.0)
    rng = np.random.default_rng(14)
    k = rng.uniform(size=n) < 0.3
    m = int(k.sum())
    Q1 = np.linalg.qr(rng.standard_normal((m, 3, 3)))[0]
    Q2 = np.linalg.qr(rng.standard_normal((m, 3, 3)))[0]
    J[k] = np.einsum("nij,j,nkj->nik", Q1, np.array([40.0, 40.0, 1.0 / 1600.0]), Q2)
    lin = np.unique(rng.integers(0, N ** 3, 3000))
    kw = dict(dim=3, N=N, kernel=I.KERNEL_ISO, h_min=0.5 / N, h_max=2.0 / N, p=1.0, window_dt=0.01,
              fp32_decision=True)
    rec = O.records(O.dep_struct(**{**kw, "fp32_decision": False}), x, J, s.acc, s.batch, s.n0, s.h0)
    eps = U32 * (1.0 + 3.0 * (2.0 / N) * np.sqrt(3))
    res = {}
    for name, plain in (("mixed", False), ("single-precision det", True)):
        oc, od, oq, found, inside = O.decision_audit(O.dep_struct(plain=plain, **kw), x, J, s.acc, s.status,
                                                     s.batch, s.n0, s.h0, lin)
        bound = 6 * np.sqrt(3) * eps / rec[od, 2] + 27 * U32 + 27 * U32 + 18 * 500 * U32
        res[name] = (found, int((np.abs(oq - 9.0) > bound).sum()), inside)
    print("\n", res)
    assert res["mixed"][1] == 0
    assert res["single-precision det"][1] > 10


# ---------------------------------------------------------------------------
# Cloud-In-Cell deposit (Sec. 1: the C^1 alternative to PSI-CELL): tent
# weights W = prod_a (1 - |x_a - xc_a| N)^+ to the cell centres around a parcel.

def _cic_cloud(d, N, n, seed, margin):
    rng = np.random.default_rng(seed)
    x = rng.uniform(margin, 1.0 - margin, (n, d))
    acc = rng.standard_normal((n, 1 + d))
    status = np.ones(n, np.int32)
    batch = rng.integers(0, 3, n).astype(np.int32)
    w = rng.uniform(0.5, 2.0, 3)
    return x, acc, status, batch, w


@pytest.mark.parametrize("d,N", [(2, 32), (3, 12)])
def test_cic_conserves_zeroth_and_first_moments(d, N):
    """Away from the walls (parcels at least half a cell inside) the tent weights of
    a parcel sum to 1 and reproduce linear functions: sum_c S_c V = -sum_i w_i a_i
    and sum_c x_c S_c V = -sum_i w_i a_i x_i, for every source component."""
    x, acc, status, batch, w = _cic_cloud(d, N, 400, 3 + d, margin=0.5 / N)
    D = O.dep_struct(dim=d, N=N, kernel=0, h_min=0.1, h_max=0.1, p=1.0, window_dt=0.5)
    counts, Sm, Sv = O.cic(D, x, acc, status, batch, w)
    V = (1.0 / N) ** d
    S = np.concatenate([Sm[:, None], Sv], axis=1)
    a = w[batch][:, None] * acc / 0.5
    assert np.allclose(S.sum(axis=0) * V, -a.sum(axis=0), rtol=1e-12, atol=1e-12)
    idx = np.arange(N ** d)
    xc = np.stack([((idx // N ** k) % N + 0.5) / N for k in range(d)], axis=1)
    for k in range(d):
        assert np.allclose((xc[:, k:k + 1] * S).sum(axis=0) * V, -(x[:, k:k + 1] * a).sum(axis=0),
                           rtol=1e-12, atol=1e-12)
    assert counts.sum() == 400


def test_cic_single_parcels_split_by_tent_weights():
    """A parcel at a cell centre stays in its cell; one on the face between two
    centres splits 1/2 : 1/2; one on a node of four centres splits into quarters;
    a quarter cell off a centre gives 3/4 : 1/4 along that axis."""
    N = 8
    D = O.dep_struct(dim=2, N=N, kernel=0, h_min=0.1, h_max=0.1, p=1.0, window_dt=1.0, per_cell=True)
    one = np.ones((1, 3))
    cases = [((2.5 / N, 3.5 / N), {(2, 3): 1.0}),
             ((3.0 / N, 3.5 / N), {(2, 3): 0.5, (3, 3): 0.5}),
             ((3.0 / N, 4.0 / N), {(2, 3): 0.25, (3, 3): 0.25, (2, 4): 0.25, (3, 4): 0.25}),
             ((2.75 / N, 3.5 / N), {(2, 3): 0.75, (3, 3): 0.25})]
    for pos, expect in cases:
        _, Sm, _ = O.cic(D, np.array([pos]), one, np.ones(1, np.int32), np.zeros(1, np.int32), np.ones(1))
        got = {(c % N, c // N): -v for c, v in enumerate(Sm) if v != 0.0}
        assert set(got) == set(expect) and all(abs(got[k] - expect[k]) < 1e-15 for k in expect), (pos, got)


@pytest.mark.parametrize("d,N", [(2, 16), (3, 8)])
def test_cic_cell_list_equals_brute_force(d, N):
    x, acc, status, batch, w = _cic_cloud(d, N, 300, 11 + d, margin=0.0)
    x[:5] = np.round(x[:5] * N) / N          # parcels exactly on faces and nodes
    x[5, 0] = 1.0                            # on the upper wall
    status[7:12] = 2                         # inactive parcels
    D = O.dep_struct(dim=d, N=N, kernel=0, h_min=0.1, h_max=0.1, p=1.0, window_dt=0.1)
    a = O.cic(D, x, acc, status, batch, w, brute=True)
    b = O.cic(D, x, acc, status, batch, w, brute=False)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
