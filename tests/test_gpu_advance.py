"""Carrier sampling and the FLA / LPT advance on the GPU against the FP64 oracle,
from identical seeds.

Tolerances.  The double-precision path follows the oracle's arithmetic up to
operation order: states agree to ~1e-12.  The compensated single-precision
path (double-float, about 48 significant bits, u_df ~ 4e-15 per operation)
from double-float carrier nodes lands within ~1e-12 of it; the tests allow
1e-9 (1 + |J|)^k.  The single-precision path rounds
each of the ~10^3 operations of a step (u = 2^-24 ~ 6e-8); rounding errors of
k steps add up to about sqrt(k) * 30 u relative per step in a smooth carrier
and are carried forward by the flow map, whose amplification is bounded by
|J| itself.  For k <= 200 steps the tests allow 1e-4 (1 + |J|) on x and v and
1e-4 (1 + |J|)^2 on J and W.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2512_20829_gb300 import fla
from paper_2512_20829_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = fla.Context(0)
    yield c
    c.close()


def _carriers():
    jet = I.jet_vortex_2d(scale=8, lpt_per_batch=0).carrier
    A = np.zeros((3, 3)); A[0, 1] = 0.7; A[1, 0] = -0.3; A[0, 0] = 0.2; A[1, 1] = -0.2
    return [(I.Carrier(kind=I.CARRIER_TAYLOR_GREEN_2D, dim=2), 2, 64),
            (jet, 2, 128),
            (I.Carrier(kind=I.CARRIER_ABC_JET_3D, dim=3), 3, 32),
            (I.Carrier(kind=I.CARRIER_LINEAR, dim=2, U=np.array([0.1, 0.2, 0]), A=A,
                       xref=np.array([0.5, 0.5, 0])), 2, 16),
            (I.Carrier(kind=I.CARRIER_UNIFORM, dim=3, U=np.array([0.1, -0.2, 0.3])), 3, 8)]


@pytest.mark.parametrize("idx", range(5))
@pytest.mark.parametrize("dtype", [fla.F32, fla.F64, fla.F32X2])
def test_carrier_nodes_match_oracle(ctx, idx, dtype):
    car, dim, N = _carriers()[idx]
    m = fla.mesh(dim, N)
    nodes = fla.nodes_buffer(m, dtype)
    t = 0.137
    fla.carrier_sample(ctx, fla.carrier_desc(car), m, t, dtype, nodes)
    stride = 8 if dim == 2 else 12
    g = nodes.double().cpu().numpy()
    o = O.carrier_nodes(car, t, N)
    nv = dim + dim * dim
    if dtype == fla.F32X2:
        # the a array, then the b array, then the tail of component maxima: each a
        # is a multiple of its component's grid Q = 2^(e - 11), 2^e above the
        # component's largest magnitude, and |b| <= Q/2 + |lo| with the low part
        # |lo| <= 2^(e - 25) of the double value's float split
        total = o.shape[0] * stride
        A = g[:total].reshape(-1, stride)[:, :nv]
        B = g[total:2 * total].reshape(-1, stride)[:, :nv]
        M = np.abs(A + B).max(axis=0)
        e = np.frexp(M.astype(np.float32))[1].astype(np.float64)
        Q = np.ldexp(1.0, (e - 11).astype(int))
        assert np.array_equal(A / Q, np.rint(A / Q)) and np.all(np.abs(A / Q) <= 2048)
        assert np.all(np.abs(B) <= Q * (0.5 + 2.0 ** -13))
        g, tol = A + B, 2.0 ** -34      # a + b within 2^-24 |b| <= 2^(e - 36) of the value
    else:
        g = g.reshape(-1, stride)[:, :nv]
        tol = 2e-6 if dtype == fla.F32 else 1e-13
    scale = np.abs(o).max(axis=0) + 1e-30
    assert np.all(np.abs(g - o) <= tol * scale), np.abs(g - o).max(axis=0) / scale


def _run_both(ctx, wl, cloud, dtype, nsteps):
    m = fla.mesh(wl.dim, wl.n_cells_axis)
    desc = fla.carrier_desc(wl.carrier)
    nodes = fla.nodes_buffer(m, dtype)
    dc = fla.DeviceCloud.from_seeds(cloud, wl.dim, wl.delta, wl.dt, dtype)
    s = 0
    while s < nsteps:
        k = min(wl.window, nsteps - s)
        fla.carrier_sample(ctx, desc, m, 0.0 if wl.carrier.steady else s * wl.dt, dtype, nodes)
        fla.advance(ctx, dc, m, nodes, s, k, wl.dt, reset_acc=True)
        s += k
    torch.cuda.synchronize()
    g = dc.to_host()
    adv = O.Advancer(wl, cloud)
    st = O.initial_state(cloud, wl.dim)
    s = 0
    while s < nsteps:
        k = min(wl.window, nsteps - s)
        adv.advance(st, s, k, reset_acc=True)
        s += k
    return g, st


def _compare(g, st, tol, dim, fla_cloud=True, acc_tol=None):
    """acc_tol: tolerance of the window sums (the compensated path keeps them in
    single precision: a sum of <= 10 single-precision terms, relative ~1e-7)."""
    acc_tol = tol if acc_tol is None else acc_tol
    assert np.array_equal(g["status"], st.status)
    act = st.status == 1
    assert act.sum() > 0
    Jn = np.linalg.norm(st.J[act], axis=(1, 2)) if fla_cloud else np.zeros(act.sum())
    s1 = (1 + Jn)[:, None]
    assert np.all(np.abs(g["x"][act] - st.x[act]) <= tol * s1)
    assert np.all(np.abs(g["v"][act] - st.v[act]) <= tol * s1 * (1 + np.abs(st.v[act])))
    if fla_cloud:
        s2 = ((1 + Jn) ** 2)[:, None, None]
        assert np.all(np.abs(g["J"][act] - st.J[act]) <= tol * s2)
        Wn = 1 + np.linalg.norm(st.W[act], axis=(1, 2))[:, None, None]
        assert np.all(np.abs(g["W"][act] - st.W[act]) <= tol * s2 * Wn)
    an = 1 + np.abs(st.acc[act])
    assert np.all(np.abs(g["acc"][act] - st.acc[act]) <= acc_tol * an * (1 + Jn)[:, None])


@pytest.mark.parametrize("dtype,tol", [(fla.F64, 1e-11), (fla.F32, 1e-4), (fla.F32X2, 1e-9)])
def test_advance_taylor_green_full_window_schedule(ctx, dtype, tol):
    wl = I.taylor_green_2d(scale=2)
    g, st = _run_both(ctx, wl, wl.fla, dtype, 200)
    _compare(g, st, tol, 2, acc_tol=2e-6 if dtype == fla.F32X2 else None)


@pytest.mark.parametrize("dtype,tol", [(fla.F64, 1e-11), (fla.F32, 1e-4), (fla.F32X2, 1e-9)])
def test_advance_jet_vortex_releases(ctx, dtype, tol):
    """Releases enter at their step, the carrier is re-sampled every window."""
    wl = I.jet_vortex_2d(scale=8, nsteps=200, lpt_per_batch=0)
    g, st = _run_both(ctx, wl, wl.fla, dtype, 150)
    assert (st.status == 0).sum() > 0 and (st.status == 1).sum() > 0
    _compare(g, st, tol, 2, acc_tol=2e-6 if dtype == fla.F32X2 else None)


@pytest.mark.parametrize("dtype,tol", [(fla.F64, 1e-11), (fla.F32, 1e-4), (fla.F32X2, 1e-9)])
def test_advance_abc_jet_3d(ctx, dtype, tol):
    wl = I.abc_jet_3d(scale=16, nsteps=60)
    g, st = _run_both(ctx, wl, wl.fla, dtype, 60)
    _compare(g, st, tol, 3, acc_tol=2e-6 if dtype == fla.F32X2 else None)


@pytest.mark.parametrize("dtype,tol", [(fla.F64, 1e-11), (fla.F32X2, 1e-9)])
@pytest.mark.parametrize("dim", [2, 3])
def test_advance_lpt_parcels(ctx, dim, dtype, tol):
    wl = I.taylor_green_2d(scale=4) if dim == 2 else I.abc_jet_3d(scale=16, nsteps=30)
    cloud = wl.lpt if dim == 2 else I.Cloud(kind=I.CLOUD_LPT, x0=wl.fla.x0[:3000], batch=wl.fla.batch[:3000],
                                            step_start=wl.fla.step_start, St0=wl.fla.St0, n0=wl.fla.n0,
                                            h0=wl.fla.h0)
    g, st = _run_both(ctx, wl, cloud, dtype, 30)
    _compare(g, st, tol, dim, fla_cloud=False, acc_tol=2e-6 if dtype == fla.F32X2 else None)


def test_outflow_and_evaporation_deadline(ctx):
    """A droplet leaving the domain and a release reaching its evaporation deadline
    both stop, on the same step as in the oracle."""
    car = I.Carrier(kind=I.CARRIER_UNIFORM, dim=2, U=np.array([2.0, 0.0, 0.0]))
    cl = I.Cloud(kind=I.CLOUD_FLA, x0=np.array([[0.99, 0.5], [0.2, 0.5], [0.3, 0.3]]),
                 batch=np.array([0, 1, 1], np.int32), step_start=np.array([0, 3], np.int32),
                 St0=np.array([0.5, 0.5]), n0=np.ones(2), h0=np.ones(2) * 0.01)
    wl = I.Workload(name="t", dim=2, n_cells_axis=16, dt=1e-3, nsteps=200, window=10, delta=-40.0,
                    carrier=car, fla=cl, lpt=None, kernel=0, h_min=0.01, h_max=0.1)
    for dtype in (fla.F64, fla.F32X2):
        g, st = _run_both(ctx, wl, cl, dtype, 200)
        assert np.array_equal(g["status"], st.status) and np.all(st.status == 2)
