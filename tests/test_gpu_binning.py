"""Cell keys, stable sort and bin starts on the GPU are bit-identical to the
oracle's keys, NumPy's stable argsort and searchsorted; a look-back wait that
runs out ends the call with a status flag and leaves the context usable."""
import time

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


def test_lookback_wait_runs_out_and_context_survives(ctx):
    """The test hook leaves tile 0's look-back words of the first radix pass
    unpublished, so every later tile waits for them.  The waits give up after
    about a second: the call ends, the status block carries
    FLA_STATUS_WAIT_TIMEOUT (fla_sync_status: FLA_ERR_TIMEOUT), nothing is left
    waiting (the stream synchronises), and the next binning, with the hook
    cleared, is bit-exact again."""
    s = I.synthetic_state(2, 70_000, 512, seed=7, inactive_frac=0.1)   # 35 tiles
    m = fla.mesh(2, 512)
    cl = gpu_cloud_from_state(s, fla.F32)
    ws = fla.aligned_ws(fla.workspace(m, fla.F32, fla.KERNEL_ANISO, cl.n))
    assert ctx.sync_status(reset=True).flags == 0
    ctx.test_stall(fla.STALL_BINNING)
    t0 = time.perf_counter()
    _, _, bins = fla.cell_bins(ctx, cl, m, ws)
    with pytest.raises(fla.FlaError, match="-5"):
        ctx.sync_status()
    dt = time.perf_counter() - t0
    st = ctx.sync_status(reset=True, allow_timeout=True)
    print(f"\nstalled binning ended after {dt:.2f} s with flags {st.flags:#x}")
    assert st.flags & fla.STATUS_WAIT_TIMEOUT
    assert 0.5 < dt < 30.0
    assert not bins.any()        # bin starts cleared: every cell empty
    _check(ctx, s, 512, fla.F32)
    assert ctx.sync_status(reset=True).flags == 0
