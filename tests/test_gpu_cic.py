"""Cloud-In-Cell deposit (cic_deposit) on the GPU against the FP64 oracle.

The tent weight of a parcel for a cell centre, prod_a (1 - |x_a - xc_a| N)^+,
is formed in the cloud's precision; per cell the GPU sums at most the parcels
of the 3^dim cells around it in a fixed order.  Counts (the box counts) are
bit-exact; the sources are compared element by element against
sum_i W_ic |w a_i| (the size of the terms each cell adds): 1e-12 of it in
double precision, 1e-5 in single precision (a few roundings of the product and
a 32-lane sum), plus, in single precision, the absolute error of each tent
factor 1 - |x - x_c| N: the rounded centre, difference, product with N and
subtraction from 1 leave at most (N + 3) u (u = 2^-24), so a weight is off by
at most d (N + 3) u whatever its size, times sum |w a| over the parcels of
the 3^dim cells around the cell.
"""
import numpy as np
import pytest
import torch

from helpers import gpu_cloud_from_state
from oracle import oracle as O
from paper_2512_20829_gb300 import fla
from paper_2512_20829_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = fla.Context(0)
    yield c
    c.close()


def _run(ctx, s, N, dtype, w, window_dt=0.01, per_cell=False):
    m = fla.mesh(s.dim, N)
    cl = gpu_cloud_from_state(s, dtype, kind=fla.CLOUD_LPT, weights=w)
    ws = fla.aligned_ws(fla.workspace(m, dtype, fla.KERNEL_ISO, max(s.x.shape[0], 1)))
    out = fla.PsicellFields(m, dtype)
    fla.cic(ctx, cl, m, window_dt, out, ws, per_cell=per_cell)
    torch.cuda.synchronize()
    return (out.counts.cpu().numpy().astype(np.uint32), out.s_mass.double().cpu().numpy(),
            out.s_mom.double().cpu().numpy().T)


def _near_abs(s, N, w, window_dt=0.01, per_cell=False):
    """Per cell, sum |w a| (the largest of the components) over the parcels binned in
    the 3^dim cells around it, in the sources' scaling."""
    d = s.dim
    D = O.dep_struct(dim=d, N=N, kernel=0, h_min=0.5 / N, h_max=0.5 / N, p=1.0, window_dt=window_dt,
                     per_cell=per_cell)
    _, pm, pv = O.psicell(D, s.x.astype(np.float64), np.abs(s.acc), s.status, s.batch, w, fp32_keys=False)
    box = np.maximum(np.abs(pm), np.abs(pv).max(axis=1)).reshape((N,) * d)   # axes (z,) y, x
    pad = np.pad(box, 1)
    near = np.zeros_like(box)
    for off in np.ndindex(*(3,) * d):
        near += pad[tuple(slice(o, o + N) for o in off)]
    return near.ravel()


def _oracle(s, N, w, window_dt=0.01, per_cell=False, fp32_keys=False):
    """fp32_keys: the box counts' keys in single precision, as a single-precision
    cloud forms them (x N floored in the cloud's precision; the tent weights do
    not depend on the key)."""
    D = O.dep_struct(dim=s.dim, N=N, kernel=0, h_min=0.5 / N, h_max=0.5 / N, p=1.0, window_dt=window_dt,
                     per_cell=per_cell)
    x = s.x.astype(np.float64)
    c, m, v = O.cic(D, x, s.acc, s.status, s.batch, w, fp32_keys=fp32_keys)
    _, am, av = O.cic(D, x, np.abs(s.acc), s.status, s.batch, w)
    return c, m, v, np.abs(am), np.abs(av)


@pytest.mark.parametrize("dim,N,n", [(2, 64, 40_000), (3, 24, 60_000)])
@pytest.mark.parametrize("dtype", [fla.F32, fla.F64])
def test_cic_matches_oracle(ctx, dim, N, n, dtype):
    s = I.synthetic_state(dim, n, N, seed=90 + dim, band=(0.1, 0.9), inactive_frac=0.05)
    w = np.random.default_rng(4).uniform(0.5, 2.0, len(s.n0))
    gc, gm, gv = _run(ctx, s, N, dtype, w)
    oc, om, ov, am, av = _oracle(s, N, w, fp32_keys=dtype == fla.F32)
    tol = 1e-12 if dtype == fla.F64 else 1e-5
    absw = 0.0 if dtype == fla.F64 else dim * (N + 3) * 2.0 ** -24 * _near_abs(s, N, w)
    assert np.array_equal(gc, oc)
    assert np.all(np.abs(gm - om) <= tol * am + absw + 1e-300)
    absv = absw[:, None] if dtype != fla.F64 else 0.0
    assert np.all(np.abs(gv - ov) <= tol * av + absv + 1e-300)


def test_cic_full_size_jet_mesh(ctx):
    """2^22 parcels on the 512^2 mesh in a band, single precision, every cell."""
    N, n = 512, 1 << 22
    s = I.synthetic_state(2, n, N, seed=97, band=(0.4, 0.6), inactive_frac=0.02)
    w = np.array([0.7, 1.1, 1.3, 0.9])
    gc, gm, gv = _run(ctx, s, N, fla.F32, w, per_cell=True)
    oc, om, ov, am, av = _oracle(s, N, w, per_cell=True, fp32_keys=True)
    absw = 2 * (N + 3) * 2.0 ** -24 * _near_abs(s, N, w, per_cell=True)
    assert np.array_equal(gc, oc)
    assert np.all(np.abs(gm - om) <= 1e-5 * am + absw + 1e-300)
    assert np.all(np.abs(gv - ov) <= 1e-5 * av + absw[:, None] + 1e-300)


def test_cic_edge_cases(ctx):
    """Parcels on cell faces, on nodes, on the upper wall x = 1 and at the lower
    wall, an inactive parcel, and an empty cloud."""
    N = 8
    pts = np.array([[3.0, 3.5], [3.0, 4.0], [8.0, 2.5], [0.0, 0.0], [2.5, 2.5], [7.99, 7.99]]) / N
    n = pts.shape[0]
    s = I.CloudState(dim=2, x=pts.astype(np.float32), v=np.zeros((n, 2), np.float32), J=np.zeros((n, 2, 2), np.float32),
                     W=np.zeros((n, 2, 2), np.float32), acc=np.ones((n, 3), np.float32),
                     status=np.array([1, 1, 1, 1, 2, 1], np.int32), batch=np.zeros(n, np.int32), n0=np.ones(1),
                     h0=np.ones(1))
    w = np.ones(1)
    for dtype in (fla.F32, fla.F64):
        gc, gm, gv = _run(ctx, s, N, dtype, w, per_cell=True)
        oc, om, ov, _, _ = _oracle(s, N, w, per_cell=True, fp32_keys=dtype == fla.F32)
        assert np.array_equal(gc, oc)
        assert np.allclose(gm, om, rtol=1e-6, atol=1e-9) and np.allclose(gv, ov, rtol=1e-6, atol=1e-9)
    empty = I.CloudState(dim=2, x=np.zeros((0, 2), np.float32), v=np.zeros((0, 2), np.float32),
                         J=np.zeros((0, 2, 2), np.float32), W=np.zeros((0, 2, 2), np.float32),
                         acc=np.zeros((0, 3), np.float32), status=np.zeros(0, np.int32), batch=np.zeros(0, np.int32),
                         n0=np.ones(1), h0=np.ones(1))
    gc, gm, gv = _run(ctx, empty, N, fla.F32, w)
    assert gc.sum() == 0 and not gm.any() and not gv.any()
