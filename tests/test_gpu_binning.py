"""Cell keys, stable sort and bin starts on the GPU are bit-identical to the
oracle's keys, NumPy's stable argsort and searchsorted."""
import numpy as np
import pytest

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


def _check(ctx, s, N, dtype):
    m = fla.mesh(s.dim, N)
    cl = gpu_cloud_from_state(s, dtype)
    ws = fla.aligned_ws(fla.workspace(m, dtype, fla.KERNEL_ANISO, cl.n))
    keys, perm, bins = fla.cell_bins(ctx, cl, m, ws)
    keys = keys.cpu().numpy().view(np.uint32)
    perm = perm.cpu().numpy().view(np.uint32)
    bins = bins.cpu().numpy().view(np.uint32)
    x = s.x.astype(np.float64) if dtype == fla.F32 else s.x.astype(np.float64)
    ok = O.cell_keys(s.dim, N, x, s.status, fp32=(dtype == fla.F32))
    nc = N ** s.dim
    ok = np.where(ok == 0xFFFFFFFF, nc, ok).astype(np.uint32)
    sk, sp, sb = O.sort_and_bins(ok, nc)
    assert np.array_equal(keys, sk)
    assert np.array_equal(perm, sp)
    assert np.array_equal(bins, sb)


@pytest.mark.parametrize("dim,N,n", [(2, 64, 4096), (2, 512, 70_000), (3, 128, 40_000), (2, 40, 333),
                                     (3, 20, 1), (2, 16, 31), (2, 16, 33), (3, 7, 5000)])
@pytest.mark.parametrize("dtype", [fla.F32, fla.F64])
def test_bins_bit_exact(ctx, dim, N, n, dtype):
    s = I.synthetic_state(dim, n, N, seed=n + N, inactive_frac=0.1)
    _check(ctx, s, N, dtype)


def test_bins_degenerate_cases(ctx):
    # everything inactive, everything in one cell, droplets on x = 1 and on cell faces
    s = I.synthetic_state(2, 5000, 32, seed=3)
    s.status[:] = 2
    _check(ctx, s, 32, fla.F32)
    s = I.synthetic_state(2, 9000, 32, seed=4, inactive_frac=0.0)
    s.x[:] = np.float32(0.51)
    _check(ctx, s, 32, fla.F32)
    s = I.synthetic_state(3, 3000, 16, seed=5)
    s.x[::3, 0] = 1.0
    s.x[1::3, 1] = np.float32(5 / 16)
    _check(ctx, s, 16, fla.F32)
    s = I.synthetic_state(2, 600, 16, seed=6)
    s.x[:5, 0] = np.float32(-1e-7)      # just outside: not binned
    s.x[5:10, 1] = np.float32(1.0000001)
    _check(ctx, s, 16, fla.F32)


def test_empty_cloud(ctx):
    s = I.synthetic_state(2, 1, 16, seed=0)
    m = fla.mesh(2, 16)
    cl = gpu_cloud_from_state(s, fla.F32)
    cl.n = 0
    ws = fla.aligned_ws(fla.workspace(m, fla.F32, 0, 1))
    _, _, bins = fla.cell_bins(ctx, cl, m, ws)
    assert np.all(bins.cpu().numpy() == 0)


def test_large_sort_three_passes(ctx):
    """2^21 keys over 128^3 cells: 22-bit keys, three radix passes, 512 tiles."""
    s = I.synthetic_state(3, 2**21, 128, seed=12, inactive_frac=0.02, edge_cases=False)
    _check(ctx, s, 128, fla.F32)
