"""The tile gather's work items against the FP64 oracle.

A tile's candidates (the records of the mesh rows within the cloud's largest
support) are cut into work items of about 4,096 (64 in double precision); a
tile of several items leaves per-cell partials that a combine kernel adds in
item order.  When a cloud's candidates exceed its item budget (its tiles +
ceil(16 n / chunk) + 1 items) the chunk grows instead.  These cases are built
so that each path is taken: a dense cluster whose tile holds many times 4,096
candidates, and a wide support that makes every record a candidate of most
tiles.  Tolerances
are those of the deposit tests: rel-L2 1e-4 per field in single precision
(1e-5 for D), 1e-12 in double precision.
"""
import math

import numpy as np
import pytest

from helpers import gpu_cloud_from_state, oracle_deposit, rel_l2
from paper_2512_20829_gb300 import fla
from paper_2512_20829_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CHUNK = 4096


@pytest.fixture(scope="module")
def ctx():
    c = fla.Context(0)
    yield c
    c.close()


def _deposit(ctx, s, N, kernel, h_min, h_max, dtype):
    m = fla.mesh(s.dim, N)
    cl = gpu_cloud_from_state(s, dtype)
    ws = fla.aligned_ws(fla.workspace(m, dtype, kernel, cl.n))
    out = fla.SourceFields(m, dtype)
    fla.deposit_sources(ctx, cl, m, fla.deposit_cfg(kernel, h_min, h_max, 0.01, 1.0, False), out, ws)
    return (out.s_mass.double().cpu().numpy(), out.s_mom.double().cpu().numpy().T,
            out.dsum.double().cpu().numpy())


def _dense(dim, n, N, seed, frac=0.85, half_width_cells=1.5, h0_cells=1.0):
    """A cloud with most droplets packed into a box of a few cells at the centre."""
    s = I.synthetic_state(dim, n, N, seed=seed, h0_cells=h0_cells)
    rng = np.random.default_rng(seed + 1)
    k = int(frac * n)
    w = half_width_cells / N
    s.x[:k] = (0.5 + rng.uniform(-w, w, (k, dim))).astype(np.float32)
    s.status[:k] = 1
    return s, k


@pytest.mark.parametrize("dim,N,n,kernel,dtype", [
    (3, 16, 30000, I.KERNEL_ANISO, fla.F32),
    (2, 48, 40000, I.KERNEL_ANISO, fla.F32),
    (3, 16, 20000, I.KERNEL_ISO, fla.F64),
], ids=["3d-aniso-f32", "2d-aniso-f32", "3d-iso-f64"])
def test_dense_tile_cut_into_items_matches_oracle(ctx, dim, N, n, kernel, dtype):
    s, k = _dense(dim, n, N, seed=300 + n)
    # the tile holding the cluster has at least k candidates: several items
    assert k > 4 * CHUNK
    args = (N, kernel, 0.5 / N, 2.0 / N)
    gm, gv, gd = _deposit(ctx, s, *args, dtype)
    om, ov, od = oracle_deposit(s, *args, 0.01, fp32=dtype == fla.F32)
    assert np.array_equal(gd > 0, od > 0)
    if dtype == fla.F32:
        assert rel_l2(gm, om) <= 1e-4 and rel_l2(gv, ov) <= 1e-4 and rel_l2(gd, od) <= 1e-5
    else:
        assert rel_l2(gm, om) <= 1e-12 and rel_l2(gv, ov) <= 1e-12 and rel_l2(gd, od) <= 1e-12


def test_chunk_grows_past_the_item_budget_matches_oracle(ctx):
    """Supports of 16 cells on a 128^2 mesh: each record is a candidate of
    about 40 of the 64 tiles, far more than the 16 items per chunk of records
    that the budget allows, so the plan widens the chunk."""
    N, n, hmax_cells = 128, 6000, 16.0
    s = I.synthetic_state(2, n, N, seed=77, h0_cells=200.0, band=(0.05, 0.95))
    R = math.floor(3 * hmax_cells + 0.5) + 1
    tiles_axis = N // 16
    per_axis = [min(tiles_axis, (min(c + R, N - 1) // 16) - (max(c - R, 0) // 16) + 1) for c in range(N)]
    mean_tiles = np.mean(per_axis) ** 2
    assert mean_tiles > 16 * 1.5
    args = (N, I.KERNEL_ISO, 0.5 / N, hmax_cells / N)
    gm, gv, gd = _deposit(ctx, s, *args, fla.F64)
    om, ov, od = oracle_deposit(s, *args, 0.01, fp32=False)
    assert np.array_equal(gd > 0, od > 0)
    assert rel_l2(gm, om) <= 1e-12 and rel_l2(gv, ov) <= 1e-12 and rel_l2(gd, od) <= 1e-12


def test_items_are_deterministic_and_independent_of_order(ctx):
    """Two runs of a multi-item deposit agree bit for bit."""
    s, _ = _dense(3, 30000, 16, seed=901)
    a = _deposit(ctx, s, 16, I.KERNEL_ANISO, 0.5 / 16, 2.0 / 16, fla.F32)
    b = _deposit(ctx, s, 16, I.KERNEL_ANISO, 0.5 / 16, 2.0 / 16, fla.F32)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
