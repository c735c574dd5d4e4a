"""Two-way coupling on the GPU (fla_ns_*, fla.TwoWay) against the FP64 oracle:
the periodic carrier of Eqs. 1-2 alone (random vorticity, random sources,
single- and double-precision source arrays), its node values for the
advance, the discrete Taylor-Green decay in closed form, and a coupled run of
droplets and carrier (App. B) end to end."""
import numpy as np
import pytest
import torch

from helpers import rel_l2
from oracle import carrier_ns as NS
from oracle import oracle as O
from paper_2512_20829_gb300 import fla
from paper_2512_20829_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = fla.Context(0)
    yield c
    c.close()


def _random_field(N, seed, width=6.0):
    rng = np.random.default_rng(seed)
    k = np.fft.fftfreq(N, 1.0 / N)
    spec = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) * np.exp(
        -(k[:, None] ** 2 + k[None, :] ** 2) / (2 * width ** 2))
    f = np.real(np.fft.ifft2(spec))
    return f / np.abs(f).max()


@pytest.mark.parametrize("N,src_dtype", [(64, fla.F64), (64, fla.F32), (32, None), (128, fla.F64)])
def test_carrier_matches_oracle(ctx, N, src_dtype):
    nu, D, dt, nsub = 2e-3, 1e-3, 1e-3, 40
    w0 = 20.0 * _random_field(N, 1)
    rho0 = 1.0 + 0.5 * _random_field(N, 2)
    U0 = (0.2, -0.1)
    ns = fla.NavierStokes(ctx, N, nu, D, dt, w0, mean_u=U0, rho=rho0)
    st = NS.init(N, nu, D, w0, U=U0, rho=rho0)
    src = None
    if src_dtype is not None:
        m = fla.mesh(2, N)
        src = fla.SourceFields(m, src_dtype)
        Sm = 2.0 * _random_field(N, 3)
        Sx, Sy = 5.0 * _random_field(N, 4) + 0.3, 5.0 * _random_field(N, 5)
        td = torch.float64 if src_dtype == fla.F64 else torch.float32
        src.s_mass.copy_(torch.as_tensor(Sm.ravel(), dtype=td))
        src.s_mom.copy_(torch.as_tensor(np.stack([Sx.ravel(), Sy.ravel()]), dtype=td))
        # the oracle gets the values the GPU reads
        Sm = src.s_mass.double().cpu().numpy().reshape(N, N)
        Sx, Sy = (a.reshape(N, N) for a in src.s_mom.double().cpu().numpy())
        NS.step(st, dt, S_mass=Sm, Sx=Sx, Sy=Sy, nsub=nsub)
    else:
        NS.step(st, dt, nsub=nsub)
    ns.step(nsub, src)
    g = ns.fields()
    torch.cuda.synchronize()
    psi = NS.streamfunction(st)
    assert rel_l2(g["psi"], psi) <= 1e-11
    assert rel_l2(g["omega"], -NS.lap5(psi, 1.0 / N)) <= 1e-11
    assert rel_l2(g["rho"], st.rho) <= 1e-11
    assert np.allclose(g["U"], st.U, rtol=1e-13, atol=1e-15)
    for dtype, tol in ((fla.F64, 1e-11), (fla.F32, 1e-6)):
        nodes = fla.nodes_buffer(fla.mesh(2, N), dtype)
        ns.nodes(dtype, nodes)
        torch.cuda.synchronize()
        got = nodes.double().cpu().numpy().reshape(-1, 8)
        ref = NS.carrier_nodes(st)
        scale = np.abs(ref).max(axis=0) + 1e-30
        assert np.all(np.abs(got - ref) <= tol * scale), (np.abs(got - ref).max(axis=0) / scale)


def test_discrete_taylor_green_decay_on_the_gpu(ctx):
    """The discrete eigenfunction decays by (1 - dt nu lambda)^n, advection
    vanishing identically (closed form, no oracle run)."""
    N, nu, dt, n = 64, 0.01, 2e-3, 50
    w0 = NS.taylor_green_omega(N)
    ns = fla.NavierStokes(ctx, N, nu, 0.0, dt, w0)
    ns.step(n)
    g = ns.fields()
    lam = NS.laplacian_eigenvalues(N)[1, 1]
    assert np.abs(g["omega"] - w0 / (1.0 - dt * nu * lam) ** n).max() <= 1e-11 * np.abs(w0).max()


def _oracle_two_way(case, n_windows):
    wl = case.wl
    N, k = wl.n_cells_axis, wl.window
    st = NS.init(N, case.nu, case.diff, case.omega0, U=case.mean_u)
    ost = O.initial_state(wl.fla, 2)
    adv = O.Advancer(wl, wl.fla)
    D = O.dep_struct(wl)
    for w in range(n_windows):
        adv.advance(ost, w * k, k, reset_acc=True, nodes=NS.carrier_nodes(st))
        Sm, Sv, _ = O.nw_deposit_celllist(D, ost.x, ost.J, ost.acc, ost.status, ost.batch, wl.fla.n0, wl.fla.h0)
        NS.step(st, wl.dt, S_mass=Sm.reshape(N, N), Sx=Sv[:, 0].reshape(N, N), Sy=Sv[:, 1].reshape(N, N), nsub=k)
    return st, ost


def test_two_way_coupled_run_matches_oracle(ctx):
    """Droplets and carrier in double precision, 8 windows of 10 steps on the
    32^2 reduction: carrier fields and droplet states against the oracle's
    coupled loop; the coupling changes the carrier measurably."""
    case = I.two_way_taylor_green(scale=4, nsteps=80, n0=5.0)
    wl = case.wl
    N = wl.n_cells_axis
    ns = fla.NavierStokes(ctx, N, case.nu, case.diff, wl.dt, case.omega0, mean_u=case.mean_u)
    tw = fla.TwoWay(ctx, wl, ns, dtype=fla.F64)
    tw.run(8)
    g = ns.fields()
    gh = tw.fla.to_host()
    torch.cuda.synchronize()
    st, ost = _oracle_two_way(case, 8)
    psi = NS.streamfunction(st)
    print(f"\ntwo-way 32^2: psi rel-L2 {rel_l2(g['psi'], psi):.2e}, rho {rel_l2(g['rho'], st.rho):.2e}, "
          f"U {g['U']} vs {st.U}")
    assert np.array_equal(gh["status"], ost.status)
    act = ost.status == 1
    assert act.sum() > 100
    assert np.abs(gh["x"][act] - ost.x[act]).max() <= 1e-10
    assert rel_l2(g["psi"], psi) <= 1e-9
    assert rel_l2(g["rho"], st.rho) <= 1e-9
    assert np.allclose(g["U"], st.U, rtol=1e-9, atol=1e-14)
    # without the coupling the carrier is measurably different
    ns1 = fla.NavierStokes(ctx, N, case.nu, case.diff, wl.dt, case.omega0, mean_u=case.mean_u)
    fla.TwoWay(ctx, wl, ns1, dtype=fla.F64, coupled=False).run(8)
    g1 = ns1.fields()
    assert rel_l2(g1["psi"], g["psi"]) > 1e-4
    assert np.abs(g1["rho"]).max() == 0.0 and np.abs(g["rho"]).max() > 0.0


def test_two_way_single_precision_droplets_follow_double(ctx):
    """The coupled run with single-precision droplets (mixed form) stays close to
    the double-precision one on the carrier fields (the carrier is double in
    both)."""
    case = I.two_way_taylor_green(scale=2, nsteps=100, n0=5.0)
    wl = case.wl
    N = wl.n_cells_axis
    res = []
    for dtype in (fla.F64, fla.F32):
        ns = fla.NavierStokes(ctx, N, case.nu, case.diff, wl.dt, case.omega0, mean_u=case.mean_u)
        fla.TwoWay(ctx, wl, ns, dtype=dtype).run(10)
        res.append(ns.fields())
    torch.cuda.synchronize()
    e_psi, e_rho = rel_l2(res[1]["psi"], res[0]["psi"]), rel_l2(res[1]["rho"], res[0]["rho"])
    print(f"\nsingle vs double droplets, 64^2, 100 steps: psi {e_psi:.2e}, rho {e_rho:.2e}")
    assert e_psi <= 1e-4 and e_rho <= 1e-3


@pytest.mark.parametrize("hold", [True, False])
def test_carrier_with_cylinder_matches_oracle(ctx, hold):
    """The immersed cylinder (penalisation, fringe strip, held or decelerated
    mean flow): fields, mean flow and the force on the body against the oracle."""
    N, nu, D, dt, nsub = 64, 5e-3, 1e-3, 1e-3, 30
    body = dict(xc=0.3, yc=0.52, r=0.06, eta=2e-3, fringe_x0=0.8, fringe_x1=0.98, fringe_sigma=200.0,
                hold_mean_flow=hold)
    w0 = 5.0 * _random_field(N, 7)
    ns = fla.NavierStokes(ctx, N, nu, D, dt, w0, mean_u=(1.0, 0.0), body=body)
    ob = NS.Body(xc=0.3, yc=0.52, R=0.06, eta=2e-3, x0=0.8, x1=0.98, sigma_max=200.0, hold_mean_flow=hold)
    st = NS.init(N, nu, D, w0, U=(1.0, 0.0), body=ob)
    F0 = ns.body_force()
    assert np.allclose(F0, NS.body_force(st), rtol=1e-11, atol=1e-9)
    ns.step(nsub)
    NS.step(st, dt, nsub=nsub)
    g = ns.fields()
    psi = NS.streamfunction(st)
    print(f"\nhold {hold}: psi rel-L2 {rel_l2(g['psi'], psi):.2e}, U {g['U']} vs {st.U}, "
          f"force {ns.body_force()} vs {NS.body_force(st)}")
    assert rel_l2(g["psi"], psi) <= 1e-10
    assert np.allclose(g["U"], st.U, rtol=1e-11, atol=1e-14)
    assert np.allclose(ns.body_force(), NS.body_force(st), rtol=1e-9, atol=1e-9)
    if hold:
        assert np.array_equal(g["U"], [1.0, 0.0])
