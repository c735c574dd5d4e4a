"""Kernel-regression and PSI-CELL deposits on the GPU against the FP64 oracle on
identical seeded cloud states.

Tolerances.  The double-precision path must agree to rel-L2 1e-12.  The
single-precision path takes the same truncation decisions as the oracle (both
decide on single-precision operands), so the remaining differences are
roundings: records and weights carry a relative error of a few 1e-7 each
(single-precision rounding, the ex2.approx weight), and plain sums of up to
1,024 terms (a staged chunk of the tile gather; 2,048 candidates over 32 lanes
and a 32-lane sum in the 2D gather) add at most 1,024 u ~ 6e-5 relative to
sum_i K_i |a_i|.  Element-wise
the test allows 1e-4 of that scale; the field-level bar is rel-L2 <= 1e-4.
"""
import numpy as np
import pytest

from helpers import gpu_cloud_from_state, oracle_deposit, oracle_scale, rel_l2
from oracle import oracle as O
from paper_2512_20829_gb300 import fla
from paper_2512_20829_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = fla.Context(0)
    yield c
    c.close()


def _gpu_deposit(ctx, s, N, kernel, h_min, h_max, window_dt, dtype, p=1.0, per_cell=False):
    m = fla.mesh(s.dim, N)
    cl = gpu_cloud_from_state(s, dtype)
    ws = fla.aligned_ws(fla.workspace(m, dtype, kernel, cl.n))
    out = fla.SourceFields(m, dtype)
    cfg = fla.deposit_cfg(kernel, h_min, h_max, window_dt, p, per_cell)
    fla.deposit_sources(ctx, cl, m, cfg, out, ws)
    return (out.s_mass.double().cpu().numpy(), out.s_mom.double().cpu().numpy().T,
            out.dsum.double().cpu().numpy())


CASES = [
    # dim, N, n, kernel, h_min (cells), h_max (cells), h0 (cells)
    (2, 64, 3000, I.KERNEL_ISO, 0.5, 4.0, 2.0),
    (2, 40, 1500, I.KERNEL_ISO, 0.5, 4.0, 1.0),      # ragged tiles (40 = 2 x 16 + 8)
    (2, 96, 20000, I.KERNEL_ISO, 0.5, 2.0, 1.5),     # many staged chunks per tile
    (3, 24, 4000, I.KERNEL_ISO, 0.5, 2.0, 1.0),
    (3, 20, 3000, I.KERNEL_ANISO, 0.5, 2.0, 0.8),    # ragged 3D tiles
    (2, 48, 2500, I.KERNEL_ANISO, 0.5, 3.0, 1.0),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"d{c[0]}N{c[1]}n{c[2]}k{c[3]}")
def test_nw_deposit_fp32_matches_oracle(ctx, case):
    dim, N, n, kernel, hmin, hmax, h0 = case
    s = I.synthetic_state(dim, n, N, seed=100 + n, h0_cells=h0)
    args = (N, kernel, hmin / N, hmax / N, 0.01)
    gm, gv, gd = _gpu_deposit(ctx, s, *args, fla.F32)
    om, ov, od = oracle_deposit(s, *args, fp32=True)
    sm, sv = oracle_scale(s, *args, fp32=True)
    assert np.array_equal(gd > 0, od > 0), "coverage (D > 0) differs"
    assert (od > 0).sum() > 0.2 * od.size
    assert rel_l2(gm, om) <= 1e-4 and rel_l2(gv, ov) <= 1e-4
    assert rel_l2(gd, od) <= 1e-5
    assert np.all(np.abs(gm - om) <= 1e-4 * sm + 1e-30)
    assert np.all(np.abs(gv - ov) <= 1e-4 * sv + 1e-30)


@pytest.mark.parametrize("case", CASES[:1] + CASES[3:5], ids=lambda c: f"d{c[0]}N{c[1]}k{c[3]}")
def test_nw_deposit_fp64_matches_oracle(ctx, case):
    dim, N, n, kernel, hmin, hmax, h0 = case
    s = I.synthetic_state(dim, n, N, seed=200 + n, h0_cells=h0)
    args = (N, kernel, hmin / N, hmax / N, 0.01)
    gm, gv, gd = _gpu_deposit(ctx, s, *args, fla.F64)
    om, ov, od = oracle_deposit(s, *args, fp32=False)
    assert rel_l2(gm, om) <= 1e-12 and rel_l2(gv, ov) <= 1e-12 and rel_l2(gd, od) <= 1e-12


def test_nw_deposit_edge_cases(ctx):
    N = 32
    # no active droplet: every source and denominator is zero
    s = I.synthetic_state(2, 200, N, seed=1)
    s.status[:] = 2
    gm, gv, gd = _gpu_deposit(ctx, s, N, 0, 0.5 / N, 4 / N, 0.01, fla.F32)
    assert not gm.any() and not gv.any() and not gd.any()
    # one droplet: S = -n a on its whole support, 0 elsewhere
    s = I.synthetic_state(2, 50, N, seed=2)
    s.status[:] = 2
    s.status[7] = 1
    gm, gv, gd = _gpu_deposit(ctx, s, N, 0, 0.5 / N, 4 / N, 0.01, fla.F32)
    om, ov, od = oracle_deposit(s, N, 0, 0.5 / N, 4 / N, 0.01, fp32=True)
    assert np.array_equal(gd > 0, od > 0) and rel_l2(gm, om) < 1e-6
    # h at its floor (tiny J) and at its cap (huge J); droplets on x = 1 and y = 0
    s = I.synthetic_state(2, 400, N, seed=3)
    s.J[:100] *= np.float32(1e-4)
    s.J[100:200] *= np.float32(1e3)
    s.x[200:210, 0] = 1.0
    s.x[210:220, 1] = 0.0
    gm, gv, gd = _gpu_deposit(ctx, s, N, 0, 0.5 / N, 4 / N, 0.01, fla.F32)
    om, ov, od = oracle_deposit(s, N, 0, 0.5 / N, 4 / N, 0.01, fp32=True)
    assert rel_l2(gm, om) <= 1e-4 and rel_l2(gv, ov) <= 1e-4 and np.array_equal(gd > 0, od > 0)
    # per-cell amounts are the per-volume sources times the cell volume
    gm2, _, _ = _gpu_deposit(ctx, s, N, 0, 0.5 / N, 4 / N, 0.01, fla.F32, per_cell=True)
    assert np.allclose(gm2, gm / N ** 2, rtol=1e-6, atol=0)


def test_nw_deposit_is_deterministic(ctx):
    s = I.synthetic_state(2, 30000, 128, seed=9, h0_cells=2.0)
    a = _gpu_deposit(ctx, s, 128, 0, 0.5 / 128, 4 / 128, 0.01, fla.F32)
    b = _gpu_deposit(ctx, s, 128, 0, 0.5 / 128, 4 / 128, 0.01, fla.F32)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_nonfinite_records_are_counted(ctx):
    s = I.synthetic_state(2, 300, 32, seed=5)
    s.status[:] = 1
    s.J[3] = np.nan
    ctx.sync_status(reset=True)
    _gpu_deposit(ctx, s, 32, 0, 0.5 / 32, 4 / 32, 0.01, fla.F32)
    st = ctx.sync_status(reset=True)
    assert st.nonfinite == 1 and st.deposited == 300


@pytest.mark.parametrize("dim,N,n", [(2, 64, 50000), (3, 16, 20000), (2, 37, 3000)])
@pytest.mark.parametrize("dtype", [fla.F32, fla.F64])
def test_psicell_matches_oracle(ctx, dim, N, n, dtype):
    s = I.synthetic_state(dim, n, N, seed=7 + n)
    w = np.array([1e-5, 2e-5, 3e-5, 4e-5])
    m = fla.mesh(dim, N)
    cl = gpu_cloud_from_state(s, dtype, kind=fla.CLOUD_LPT, weights=w)
    ws = fla.aligned_ws(fla.workspace(m, dtype, 0, n))
    out = fla.PsicellFields(m, dtype)
    fla.psicell(ctx, cl, m, 0.01, out, ws)
    D = O.dep_struct(dim=dim, N=N, kernel=0, h_min=1, h_max=1, p=1, window_dt=0.01)
    counts, Sm, Sv = O.psicell(D, s.x, s.acc, s.status, s.batch, w, fp32_keys=(dtype == fla.F32))
    assert np.array_equal(out.counts.cpu().numpy().astype(np.uint32), counts)
    # scale: -(1/V) sum w |a| per cell
    _, am, av = O.psicell(D, s.x, np.abs(s.acc), s.status, s.batch, w, fp32_keys=(dtype == fla.F32))
    tol = 1e-5 if dtype == fla.F32 else 1e-13
    gm = out.s_mass.double().cpu().numpy()
    gv = out.s_mom.double().cpu().numpy().T
    assert np.all(np.abs(gm - Sm) <= tol * np.abs(am) + 1e-300)
    assert np.all(np.abs(gv - Sv) <= tol * np.abs(av) + 1e-300)
