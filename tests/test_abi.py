"""The C-ABI library loads without a GPU, exports every function fla.h declares,
and its host-side logic (layouts, sizes, deadlines, argument checks) behaves as
documented.  No kernel is launched here."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_20829_gb300 import build as B
from paper_2512_20829_gb300 import fla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return fla.lib()


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "sizeof"):
                names.append(name)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert "fla_advance" in declared and "psicell_deposit" in declared and "fla_deposit_sources" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", fla.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    for n in declared:
        assert hasattr(lib, n)
    assert set(fla.EXPORTED) <= set(declared)


def test_abi_version_and_status_strings(lib):
    assert lib.fla_abi_version() == fla.ABI_VERSION
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.fla_status_string(code)
    assert lib.fla_status_string(42) == b"unknown status"


def test_state_layout_matches_header_contract(lib):
    assert fla.state_layout(fla.CLOUD_FLA, 2) == {"n_planes": 4, "x": 0, "v": 2, "J": 4, "W": 8, "acc": 12}
    assert fla.state_layout(fla.CLOUD_FLA, 3) == {"n_planes": 7, "x": 0, "v": 3, "J": 6, "W": 15, "acc": 24}
    assert fla.state_layout(fla.CLOUD_LPT, 2) == {"n_planes": 2, "x": 0, "v": 2, "J": -1, "W": -1, "acc": 4}
    assert fla.state_layout(fla.CLOUD_LPT, 3) == {"n_planes": 3, "x": 0, "v": 3, "J": -1, "W": -1, "acc": 6}
    with pytest.raises(fla.FlaError):
        fla.state_layout(7, 2)


def test_pack_unpack_roundtrip(lib):
    rng = np.random.default_rng(0)
    for kind, dim in ((0, 2), (0, 3), (1, 2), (1, 3)):
        n = 37
        x, v = rng.random((n, dim)), rng.random((n, dim))
        acc = rng.random((n, 1 + dim))
        J = rng.random((n, dim, dim)) if kind == 0 else None
        W = rng.random((n, dim, dim)) if kind == 0 else None
        p = fla.pack_state(kind, dim, n, np.float64, x=x, v=v, J=J, W=W, acc=acc)
        u = fla.unpack_state(kind, dim, p)
        assert np.array_equal(u["x"], x) and np.array_equal(u["v"], v) and np.array_equal(u["acc"], acc)
        if kind == 0:
            assert np.array_equal(u["J"], J) and np.array_equal(u["W"], W)
        st = rng.integers(0, 3, n)
        b = rng.integers(0, 1000, n)
        m = fla.meta_words(st, b)
        assert np.array_equal(fla.status_of(m), st) and np.array_equal(m & fla.META_BATCH_MASK, b)


def test_sizes(lib):
    m = fla.mesh(2, 64)
    assert lib.fla_carrier_nodes_bytes(C.byref(m), 0) == 65 * 65 * 8 * 4
    assert lib.fla_carrier_nodes_bytes(C.byref(fla.mesh(3, 16)), 1) == 17 ** 3 * 12 * 8
    a = fla.workspace_size(m, fla.F32, fla.KERNEL_ISO, 1000)
    b = fla.workspace_size(m, fla.F32, fla.KERNEL_ISO, 100000)
    assert 0 < a < b and a % 256 == 0
    assert fla.workspace_size(fla.mesh(3, 16), fla.F32, fla.KERNEL_ANISO, 100) > \
        fla.workspace_size(fla.mesh(3, 16), fla.F32, fla.KERNEL_ISO, 100)
    out = C.c_size_t()
    assert lib.fla_workspace_size(C.byref(fla.mesh(4, 16)), 0, 0, 10, C.byref(out)) == -1
    assert lib.fla_workspace_size(C.byref(m), 0, 0, -1, C.byref(out)) == -1
    # the sorted permutation sits in one of the two value buffers, after the two key buffers
    for n in (1, 1000, 100000):
        assert lib.fla_workspace_order(C.byref(m), n, C.byref(out)) == 0
        u = (4 * n + 255) // 256 * 256
        assert out.value in (2 * u, 3 * u)
        assert out.value + 4 * n <= fla.workspace_size(m, fla.F32, fla.KERNEL_ISO, n)
    assert lib.fla_workspace_order(C.byref(m), 0, C.byref(out)) == -1
    assert lib.fla_workspace_order(C.byref(fla.mesh(4, 16)), 10, C.byref(out)) == -1


def test_batch_deadline_agrees_with_oracle(lib):
    rng = np.random.default_rng(1)
    for _ in range(200):
        St0, delta, s0 = rng.uniform(0.01, 3), -rng.uniform(0.01, 60), int(rng.integers(0, 1000))
        assert fla.batch_deadline(St0, delta, 1e-3, s0) == O.step_dead(St0, delta, 1e-3, s0)
    assert fla.batch_deadline(0.5, 0.0, 1e-3, 3) == 2**31 - 1
    with pytest.raises(fla.FlaError):
        fla.batch_deadline(-1.0, -0.2, 1e-3, 0)


def test_no_gpu_means_no_context(lib):
    """Without a usable CUDA device the library refuses to create a context (no CPU path)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.fla_create(C.byref(h), 0) == -2
    with pytest.raises(fla.FlaError):
        fla.Context(0)


def test_entry_points_reject_bad_arguments_before_launching(lib):
    m = fla.mesh(2, 16)
    cl = fla.Cloud()
    cl.kind, cl.dim, cl.dtype, cl.n, cl.n_batches = 0, 2, 0, 10, 1
    null = C.c_void_p(0)
    # null context / null pointers / bad dims -> FLA_ERR_ARG, nothing enqueued
    assert lib.fla_advance(null, C.byref(cl), C.byref(m), null, 0, 1, 1e-3, 0, null) == -1
    fake_ctx = C.c_void_p(1)   # never dereferenced: validation fails first
    assert lib.fla_advance(fake_ctx, C.byref(cl), C.byref(m), null, 0, 1, 1e-3, 0, null) == -1
    # a processing order that is not 4-byte aligned
    assert lib.fla_advance_ordered(fake_ctx, C.byref(cl), C.byref(m), C.c_void_p(256), C.c_void_p(258), 0, 1, 1e-3,
                                   0, null) == -1
    cl.dim = 3
    assert lib.fla_advance(fake_ctx, C.byref(cl), C.byref(m), null, 0, 1, 1e-3, 0, null) == -1
    cfg = fla.deposit_cfg(0, 0.0, 0.1, 0.01)
    so = fla.Sources()
    assert lib.fla_deposit_sources(fake_ctx, C.byref(cl), C.byref(m), C.byref(cfg), C.byref(so), null, 0, null) == -1
    po = fla.PsicellOut()
    assert lib.psicell_deposit(fake_ctx, C.byref(cl), C.byref(m), 0.01, 0, C.byref(po), null, 0, null) == -1
    desc = fla.carrier_desc(__import__("paper_2512_20829_gb300.inputs", fromlist=["x"]).Carrier(kind=2, dim=3))
    assert lib.fla_carrier_sample(fake_ctx, C.byref(desc), C.byref(fla.mesh(3, 8)), 0.0, 0, C.c_void_p(256), null) == -1


def test_fold_array_sizes(lib):
    # J and W in planes of 4 doubles, then the hand-over list (n u32) and its counter, 16-byte aligned
    assert lib.fla_fold_bytes(2, 1000) == 2 * 1000 * 32 + 4000 + 16
    assert lib.fla_fold_bytes(3, 1000) == 5 * 1000 * 32 + 4000 + 16
    assert lib.fla_fold_bytes(3, 3) == 5 * 3 * 32 + 16 + 16
    assert lib.fla_fold_bytes(4, 10) == 0 and lib.fla_fold_bytes(2, -1) == 0


def _batch_item(dim=2, N=16, n=100, kernel=fla.KERNEL_ISO, dtype=fla.F32):
    it = fla.BatchItem()
    it.cloud.kind, it.cloud.dim, it.cloud.dtype, it.cloud.n_batches, it.cloud.n = fla.CLOUD_FLA, dim, dtype, 1, n
    # non-null, aligned stand-in addresses: the size query reads no memory
    it.cloud.state_dev = it.cloud.meta_dev = it.cloud.batches_dev = 1 << 20
    it.mesh = fla.mesh(dim, N)
    it.carrier.kind, it.carrier.dim = 2 if dim == 2 else 4, dim
    it.nodes_dev = 1 << 20
    it.cfg = fla.deposit_cfg(kernel, 0.5 / N, 2.0 / N, 0.01)
    it.out.s_mass_dev = it.out.s_mom_dev = 1 << 20
    return it


def test_batch_workspace_size_and_argument_checks(lib):
    items = (fla.BatchItem * 3)(_batch_item(2, 16, 100), _batch_item(3, 8, 50, fla.KERNEL_ANISO),
                                _batch_item(2, 32, 1000))
    nb = C.c_size_t()
    assert lib.fla_batch_workspace_size(items, 3, C.byref(nb)) == 0
    base = nb.value
    # the workspace grows with the droplets and the cells
    items[2] = _batch_item(2, 32, 5000)
    assert lib.fla_batch_workspace_size(items, 3, C.byref(nb)) == 0 and nb.value > base
    items[2] = _batch_item(2, 64, 1000)
    assert lib.fla_batch_workspace_size(items, 3, C.byref(nb)) == 0 and nb.value > base
    # rejected items
    bad = _batch_item(2, 16, 100, dtype=fla.F64)
    assert lib.fla_batch_workspace_size((fla.BatchItem * 1)(bad), 1, C.byref(nb)) == -1
    bad = _batch_item(2, 16, 100)
    bad.mesh = fla.mesh(3, 16)                      # cloud and mesh dimensions differ
    assert lib.fla_batch_workspace_size((fla.BatchItem * 1)(bad), 1, C.byref(nb)) == -1
    bad = _batch_item(2, 16, 100)
    bad.nodes_dev = None
    assert lib.fla_batch_workspace_size((fla.BatchItem * 1)(bad), 1, C.byref(nb)) == -1
    bad = _batch_item(2, 16, 100)
    bad.cfg.mlp_dev = 1 << 20                       # no learned correction in a batch
    assert lib.fla_batch_workspace_size((fla.BatchItem * 1)(bad), 1, C.byref(nb)) == -6
    bad = _batch_item(2, 16, 100)
    bad.cfg.h_max = 8.0                             # support wider than 192 cells
    assert lib.fla_batch_workspace_size((fla.BatchItem * 1)(bad), 1, C.byref(nb)) == -6
    assert lib.fla_batch_workspace_size(items, 0, C.byref(nb)) == -1
    assert lib.fla_batch_workspace_size(None, 1, C.byref(nb)) == -1


def test_noalloc_binning_rejects_the_clouds_the_workspace_version_rejects(lib):
    """fla_cell_bins_noalloc checks its arguments with the library's shared cloud
    checks (those of fla_cell_bins) before its size limit: bad dtype, bad kind, a
    fold guard on a parcel cloud, a non-finite delta, a misaligned release table,
    a missing meta array and a mesh of the wrong dimension are all FLA_ERR_ARG,
    with nothing enqueued (no GPU is touched here)."""
    f = lib.fla_cell_bins_noalloc
    f.argtypes = [C.POINTER(fla.Cloud), C.POINTER(fla.Mesh), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    state = np.zeros(64 * 4, np.float32)
    meta = np.zeros(16, np.uint32)
    batches = np.zeros(8, np.float64)
    keys = np.zeros(16, np.uint32)

    def cloud(**kw):
        c = fla.Cloud()
        c.kind, c.dim, c.dtype, c.n_batches, c.n = fla.CLOUD_FLA, 2, fla.F32, 1, 16
        c.state_dev = state.ctypes.data
        c.meta_dev = meta.ctypes.data
        c.batches_dev = batches.ctypes.data
        c.delta = 0.0
        for k, v in kw.items():
            setattr(c, k, v)
        return c
    m2, m3 = fla.mesh(2, 8), fla.mesh(3, 8)
    bad = [cloud(dtype=7), cloud(kind=5), cloud(kind=fla.CLOUD_LPT, fold_dev=state.ctypes.data, tau_fold=0.01),
           cloud(delta=float("nan")), cloud(batches_dev=batches.ctypes.data + 4), cloud(meta_dev=None)]
    for c in bad:
        assert f(C.byref(c), C.byref(m2), keys.ctypes.data, keys.ctypes.data, keys.ctypes.data, None) == -1
    assert f(C.byref(cloud()), C.byref(m3), keys.ctypes.data, keys.ctypes.data, keys.ctypes.data, None) == -1
    big = cloud(n=262_145)
    assert f(C.byref(big), C.byref(m2), keys.ctypes.data, keys.ctypes.data, keys.ctypes.data, None) == -3
