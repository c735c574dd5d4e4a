"""The allocation-free cell binning, fla_cell_bins_noalloc, against fla_cell_bins.

fla_cell_bins_noalloc serves callers that cannot allocate device memory (a
coupling layer that only passes pointers to buffers it already owns, or code
where cudaMalloc is not allowed): it takes its scratch space from a fixed
array inside the library instead of a workspace.  Its results must equal the
workspace version bit for bit, also on the second of two calls in a row, when
the shared array still holds the first call's data.  This file is named so
that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from helpers import gpu_cloud_from_state
from paper_2512_20829_gb300 import fla
from paper_2512_20829_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MAX_DROPLETS = 262144   # FLA_NOALLOC_MAX_DROPLETS in fla.h


def _noalloc(cloud, m):
    f = fla.lib().fla_cell_bins_noalloc
    f.argtypes = [C.POINTER(fla.Cloud), C.POINTER(fla.Mesh), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    n = max(cloud.n, 1)
    keys = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    bins = torch.full((m.n ** m.dim + 1,), -1, dtype=torch.int32, device="cuda")
    cs = cloud.struct()
    rc = f(C.byref(cs), C.byref(m), keys.data_ptr(), perm.data_ptr(), bins.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return rc, keys[:cloud.n].cpu().numpy(), perm[:cloud.n].cpu().numpy(), bins.cpu().numpy()


def test_noalloc_bins_equal_workspace_bins_on_two_calls_in_a_row():
    ctx = fla.Context(0)
    # the second call is smaller and on another mesh, so stale data from the first
    # call sits in the shared scratch array beyond what the second call writes
    for dim, N, n, seed, dtype in [(2, 512, MAX_DROPLETS, 1, fla.F32), (3, 32, 40_000, 2, fla.F64)]:
        s = I.synthetic_state(dim, n, N, seed=seed, inactive_frac=0.1)
        m = fla.mesh(dim, N)
        cl = gpu_cloud_from_state(s, dtype)
        ws = fla.aligned_ws(fla.workspace(m, dtype, fla.KERNEL_ISO, n))
        k_ref, p_ref, b_ref = (t.cpu().numpy() for t in fla.cell_bins(ctx, cl, m, ws))
        rc, k, p, b = _noalloc(cl, m)
        assert rc == 0, fla.lib().fla_status_string(rc)
        assert np.array_equal(k, k_ref) and np.array_equal(p, p_ref) and np.array_equal(b, b_ref)
    ctx.close()


def test_noalloc_rejects_clouds_beyond_its_fixed_size():
    s = I.synthetic_state(2, MAX_DROPLETS + 1, 64, seed=3)
    cl = gpu_cloud_from_state(s, fla.F32)
    rc, _, _, _ = _noalloc(cl, fla.mesh(2, 64))
    assert rc == -3   # FLA_ERR_WORKSPACE, nothing enqueued
