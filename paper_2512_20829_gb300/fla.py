"""Thin Python binding of libfla (``include/fla.h``).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams; NumPy packs host
arrays into the library's plane layout.  The binding refuses to work without
the compiled library: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import inputs as I

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfla.so")

ABI_VERSION = 11            # FLA_ABI_VERSION of include/fla.h that these structures mirror
F32, F64, F32X2 = 0, 1, 2  # F32X2: compensated single precision (hi planes, then lo planes)
CLOUD_FLA, CLOUD_LPT = 0, 1
KERNEL_ISO, KERNEL_ANISO = 0, 1
META_BATCH_MASK = 0x00FFFFFF
META_FOLD = 0x20000000
META_DEAD = 0x40000000
META_ACTIVE = 0x80000000
ADVANCE_RESET_ACC = 1
MAX_VORTICES = 16

EXPORTED = ["fla_abi_version", "fla_status_string", "fla_create", "fla_destroy", "fla_state_layout",
            "fla_carrier_nodes_bytes", "fla_carrier_sample", "fla_batch_deadline", "fla_advance",
            "fla_advance_ordered", "fla_workspace_size", "fla_workspace_order", "fla_cell_bins", "fla_deposit_sources", "psicell_deposit", "cic_deposit",
            "fla_sync_status",
            "fla_profile_enable", "fla_profile_read", "fla_phase_name", "fla_fold_bytes", "fla_mlp_pack",
            "fla_mlp_forward", "fla_learn_workspace_size", "fla_learn_grad", "fla_adam_step",
            "fla_batch_workspace_size", "fla_batch_create", "fla_batch_run", "fla_batch_set_step",
            "fla_batch_tuning", "fla_batch_set_tuning", "fla_batch_set_mode", "fla_batch_mode",
            "fla_batch_destroy", "fla_test_stall", "fla_ns_workspace_size", "fla_ns_init", "fla_ns_step",
            "fla_ns_nodes", "fla_ns_fields", "fla_ns_body_force"]
STALL_BINNING = 1           # fla_test_stall: one CTA of the next binning skips its first grid barrier
STALL_BATCH_WINDOW = 2      # ... of the next persistent batch window
BATCH_AUTO, BATCH_LAUNCHES, BATCH_PERSISTENT = 0, 1, 2
STATUS_MLP_TIMEOUT, STATUS_WAIT_TIMEOUT = 1, 2   # fla_device_status.flags
MLP_FEATURES, MLP_HIDDEN, MLP_PARAMS, MLP_PACKED_BYTES = 6, 64, 8833, 19472
PREC_MIXED, PREC_PLAIN = 0, 1
TAU_FOLD = 1e-2
PHASES = ["carrier", "advance", "keys", "sort", "bins", "records", "gather", "psicell"]


class FlaError(RuntimeError):
    pass


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int32)]


class CarrierDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dim", C.c_int32), ("U", C.c_double * 3), ("A", C.c_double * 9),
                ("xref", C.c_double * 3), ("n_vortex", C.c_int32), ("vortex", (C.c_double * 5) * MAX_VORTICES),
                ("jet_width", C.c_double), ("abc", C.c_double * 3), ("jet_amp", C.c_double),
                ("jet_radius", C.c_double)]


class Cloud(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dim", C.c_int32), ("dtype", C.c_int32), ("n_batches", C.c_int32),
                ("n", C.c_int64), ("state_dev", C.c_void_p), ("meta_dev", C.c_void_p),
                ("batches_dev", C.c_void_p), ("delta", C.c_double), ("fold_dev", C.c_void_p),
                ("tau_fold", C.c_double)]


class DepositCfg(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("per_cell", C.c_int32), ("h_min", C.c_double), ("h_max", C.c_double),
                ("p", C.c_double), ("window_dt", C.c_double), ("precision", C.c_int32),
                ("reserved", C.c_int32), ("mlp_dev", C.c_void_p), ("mlp_out_dev", C.c_void_p)]


class Sources(C.Structure):
    _fields_ = [("s_mass_dev", C.c_void_p), ("s_mom_dev", C.c_void_p), ("dsum_dev", C.c_void_p)]


class PsicellOut(C.Structure):
    _fields_ = [("counts_dev", C.c_void_p), ("s_mass_dev", C.c_void_p), ("s_mom_dev", C.c_void_p)]


class BatchItem(C.Structure):
    _fields_ = [("cloud", Cloud), ("mesh", Mesh), ("carrier", CarrierDesc), ("nodes_dev", C.c_void_p),
                ("cfg", DepositCfg), ("out", Sources)]


class DeviceStatus(C.Structure):
    _fields_ = [("nonfinite", C.c_uint64), ("deposited", C.c_uint64), ("droplet_steps", C.c_uint64),
                ("pairs", C.c_uint64), ("fold_steps", C.c_uint64), ("flags", C.c_uint32), ("pad", C.c_uint32)]


BATCH_DTYPE = np.dtype([("St0", "<f8"), ("n0", "<f8"), ("h0", "<f8"), ("step_start", "<i4"),
                        ("step_dead", "<i4")])
assert BATCH_DTYPE.itemsize == 32

class NSConfig(C.Structure):
    """fla_ns_cfg: the two-way carrier on a periodic square of n x n cells."""
    _fields_ = [("n", C.c_int32), ("nu", C.c_double), ("diff", C.c_double), ("dt", C.c_double),
                ("body", C.c_int32), ("hold_mean_flow", C.c_int32), ("body_xc", C.c_double),
                ("body_yc", C.c_double), ("body_r", C.c_double), ("body_eta", C.c_double),
                ("fringe_x0", C.c_double), ("fringe_x1", C.c_double), ("fringe_sigma", C.c_double)]


_lib = None


def lib() -> C.CDLL:
    """Load libfla.so; raise if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FlaError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        v, i32, i64, u32, d = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_double
        P = C.POINTER
        L.fla_abi_version.restype = C.c_int
        L.fla_status_string.restype = C.c_char_p
        L.fla_status_string.argtypes = [C.c_int]
        L.fla_create.argtypes = [P(v), C.c_int]
        L.fla_destroy.argtypes = [v]
        L.fla_destroy.restype = None
        L.fla_state_layout.argtypes = [i32, i32] + [P(i32)] * 6
        L.fla_carrier_nodes_bytes.argtypes = [P(Mesh), i32]
        L.fla_carrier_nodes_bytes.restype = C.c_size_t
        L.fla_carrier_sample.argtypes = [v, P(CarrierDesc), P(Mesh), d, i32, v, v]
        L.fla_batch_deadline.argtypes = [d, d, d, i32, P(i32)]
        L.fla_advance.argtypes = [v, P(Cloud), P(Mesh), v, i32, i32, d, u32, v]
        L.fla_advance_ordered.argtypes = [v, P(Cloud), P(Mesh), v, v, i32, i32, d, u32, v]
        L.fla_workspace_order.argtypes = [P(Mesh), i64, P(C.c_size_t)]
        L.fla_workspace_size.argtypes = [P(Mesh), i32, i32, i64, P(C.c_size_t)]
        L.fla_cell_bins.argtypes = [v, P(Cloud), P(Mesh), v, v, v, v, C.c_size_t, v]
        L.fla_deposit_sources.argtypes = [v, P(Cloud), P(Mesh), P(DepositCfg), P(Sources), v, C.c_size_t, v]
        L.psicell_deposit.argtypes = [v, P(Cloud), P(Mesh), d, i32, P(PsicellOut), v, C.c_size_t, v]
        L.cic_deposit.argtypes = [v, P(Cloud), P(Mesh), d, i32, P(PsicellOut), v, C.c_size_t, v]
        L.fla_sync_status.argtypes = [v, v, P(DeviceStatus), C.c_int]
        L.fla_test_stall.argtypes = [v, C.c_uint32]
        L.fla_profile_enable.argtypes = [v, C.c_int, C.c_int]
        L.fla_profile_read.argtypes = [v, i32, P(C.c_double), P(i64), P(i64)]
        L.fla_phase_name.argtypes = [i32]
        L.fla_phase_name.restype = C.c_char_p
        L.fla_fold_bytes.argtypes = [i32, i64]
        L.fla_fold_bytes.restype = C.c_size_t
        L.fla_mlp_pack.argtypes = [v, v, v, v]
        L.fla_mlp_forward.argtypes = [v, v, v, i64, v, v]
        L.fla_learn_workspace_size.argtypes = [v, P(Mesh), i64, P(C.c_size_t)]
        L.fla_learn_grad.argtypes = [v, P(Cloud), P(Mesh), P(DepositCfg), v, i64, v, P(Sources), v, v, v,
                                     C.c_size_t, v, C.c_size_t, v]
        L.fla_adam_step.argtypes = [v, v, v, v, v, i64, C.c_float, C.c_float, C.c_float, C.c_float, i32, v]
        L.fla_batch_workspace_size.argtypes = [P(BatchItem), i32, P(C.c_size_t)]
        L.fla_batch_create.argtypes = [v, P(BatchItem), i32, d, i32, i32, v, C.c_size_t, P(v)]
        L.fla_batch_run.argtypes = [v, v, i32, v]
        L.fla_batch_set_step.argtypes = [v, i32, v]
        L.fla_batch_tuning.argtypes = [v, P(i32), P(i32), P(i32), P(i32)]
        L.fla_batch_set_tuning.argtypes = [v, i32, i32, i32]
        L.fla_batch_set_mode.argtypes = [v, i32]
        L.fla_batch_mode.argtypes = [v, P(i32), P(C.c_float), P(C.c_float)]
        L.fla_batch_destroy.argtypes = [v]
        L.fla_batch_destroy.restype = None
        L.fla_ns_workspace_size.argtypes = [P(NSConfig)]
        L.fla_ns_workspace_size.restype = C.c_size_t
        L.fla_ns_init.argtypes = [v, P(NSConfig), v, P(d), v, v, C.c_size_t, v]
        L.fla_ns_step.argtypes = [v, P(NSConfig), v, v, i32, i32, v, C.c_size_t, v]
        L.fla_ns_nodes.argtypes = [v, P(NSConfig), i32, v, v, C.c_size_t, v]
        L.fla_ns_fields.argtypes = [v, P(NSConfig), v, v, v, P(d), v, C.c_size_t, v]
        L.fla_ns_body_force.argtypes = [v, P(NSConfig), P(d), v, C.c_size_t, v]
        if L.fla_abi_version() != ABI_VERSION:
            raise FlaError(f"{LIB_PATH} has ABI version {L.fla_abi_version()}, the binding expects "
                           f"{ABI_VERSION}: rebuild it with __graft_entry__.build()")
        _lib = L
    return _lib


def check(code: int, what: str) -> None:
    if code != 0:
        msg = lib().fla_status_string(code).decode()
        raise FlaError(f"{what} failed: {msg} ({code})")


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


class Context:
    """Owns an fla_ctx (device handle, SM count, status block)."""

    def __init__(self, device: int = 0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise FlaError("no CUDA device: the FLA library has no CPU path")
        torch.cuda.set_device(device)
        h = C.c_void_p()
        check(lib().fla_create(C.byref(h), device), "fla_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            lib().fla_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile(self, enable: bool, reset: bool = True) -> None:
        """Per-phase launch counting is always on; enable adds CUDA-event timing
        (eager launches only, not while capturing a graph)."""
        check(lib().fla_profile_enable(self.handle, 1 if enable else 0, 1 if reset else 0), "fla_profile_enable")

    def profile_read(self) -> dict:
        n = len(PHASES)
        ms = (C.c_double * n)()
        la = (C.c_int64 * n)()
        ca = (C.c_int64 * n)()
        check(lib().fla_profile_read(self.handle, n, ms, la, ca), "fla_profile_read")
        return {PHASES[i]: {"ms": ms[i], "launches": la[i], "calls": ca[i]} for i in range(n)}

    def sync_status(self, stream=None, reset: bool = False, allow_timeout: bool = False) -> DeviceStatus:
        """The device status block.  A device-side wait that ran out raises
        (FLA_ERR_TIMEOUT) unless allow_timeout, when the caller reads .flags."""
        st = DeviceStatus()
        code = lib().fla_sync_status(self.handle, _stream_ptr(stream), C.byref(st), 1 if reset else 0)
        if code not in (0, -4) and not (allow_timeout and code == -5):
            check(code, "fla_sync_status")
        return st

    def test_stall(self, what: int) -> None:
        """Test hook (fla_test_stall): one CTA of the next binning (STALL_BINNING)
        or persistent batch window (STALL_BATCH_WINDOW) skips its first grid barrier."""
        check(lib().fla_test_stall(self.handle, what), "fla_test_stall")


def mesh(dim: int, n: int) -> Mesh:
    return Mesh(dim, n)


def state_layout(kind: int, dim: int) -> dict:
    vals = [C.c_int32() for _ in range(6)]
    check(lib().fla_state_layout(kind, dim, *[C.byref(x) for x in vals]), "fla_state_layout")
    keys = ["n_planes", "x", "v", "J", "W", "acc"]
    return {k: x.value for k, x in zip(keys, vals)}


def carrier_desc(car: I.Carrier) -> CarrierDesc:
    c = CarrierDesc()
    c.kind, c.dim = int(car.kind), int(car.dim)
    U = np.zeros(3); U[:np.asarray(car.U).size] = np.asarray(car.U, float).ravel()[:3]
    xr = np.zeros(3); xr[:np.asarray(car.xref).size] = np.asarray(car.xref, float).ravel()[:3]
    A = np.zeros((3, 3)); Ai = np.asarray(car.A, float); A[:Ai.shape[0], :Ai.shape[1]] = Ai
    for k in range(3):
        c.U[k], c.xref[k], c.abc[k] = U[k], xr[k], float(car.abc[k])
    for k in range(9):
        c.A[k] = A.ravel()[k]
    vt = np.asarray(car.vortices, float).reshape(-1, 5)
    if vt.shape[0] > MAX_VORTICES:
        raise FlaError("too many vortices")
    c.n_vortex = vt.shape[0]
    for k in range(vt.shape[0]):
        for q in range(5):
            c.vortex[k][q] = vt[k, q]
    c.jet_width, c.jet_amp, c.jet_radius = float(car.jet_width), float(car.jet_amp), float(car.jet_radius)
    return c


def batch_deadline(St0: float, delta: float, dt: float, step_start: int) -> int:
    out = C.c_int32()
    check(lib().fla_batch_deadline(float(St0), float(delta), float(dt), int(step_start), C.byref(out)),
          "fla_batch_deadline")
    return out.value


def batch_table(cloud: I.Cloud, delta: float, dt: float) -> np.ndarray:
    nb = len(cloud.St0)
    t = np.zeros(nb, BATCH_DTYPE)
    t["St0"], t["n0"], t["h0"] = cloud.St0, cloud.n0, cloud.h0
    t["step_start"] = cloud.step_start
    t["step_dead"] = [batch_deadline(s, delta, dt, ss) for s, ss in zip(cloud.St0, cloud.step_start)]
    return t


def meta_words(status: np.ndarray, batch: np.ndarray) -> np.ndarray:
    m = np.asarray(batch, np.uint32) & META_BATCH_MASK
    m = np.where(np.asarray(status) == 1, m | META_ACTIVE, m)
    m = np.where(np.asarray(status) == 2, m | META_DEAD, m)
    return m.astype(np.uint32)


def status_of(meta: np.ndarray) -> np.ndarray:
    meta = np.asarray(meta, np.uint32)
    st = np.zeros(meta.shape, np.int32)
    st[(meta & META_ACTIVE) != 0] = 1
    st[(meta & META_DEAD) != 0] = 2
    return st


def pack_state(kind: int, dim: int, n: int, np_dtype, x=None, v=None, J=None, W=None, acc=None,
               split: bool = False) -> np.ndarray:
    """Host array (n_planes, n, 4) in the library's plane layout.  split: the
    compensated layout (2 n_planes, n, 4) float32, the planes of the nearest
    floats followed by the planes of the nearest floats to the remainders."""
    L = state_layout(kind, dim)
    flat = np.zeros((n, L["n_planes"] * 4), dtype=np.float64 if split else np_dtype)
    for name, arr, width in (("x", x, dim), ("v", v, dim), ("J", J, dim * dim), ("W", W, dim * dim),
                             ("acc", acc, 1 + dim)):
        if arr is not None:
            flat[:, L[name]:L[name] + width] = np.asarray(arr).reshape(n, width)
    if split:
        hi = flat.astype(np.float32)
        lo = (flat - hi.astype(np.float64)).astype(np.float32)
        flat = np.concatenate([hi.reshape(n, L["n_planes"], 4), lo.reshape(n, L["n_planes"], 4)], axis=1)
        return np.ascontiguousarray(flat.transpose(1, 0, 2))
    return np.ascontiguousarray(flat.reshape(n, L["n_planes"], 4).transpose(1, 0, 2))


def unpack_state(kind: int, dim: int, planes: np.ndarray, split: bool = False) -> dict:
    """Inverse of pack_state; split: the compensated layout, values returned as
    float64 hi + lo."""
    L = state_layout(kind, dim)
    if split:
        npl = planes.shape[0] // 2
        planes = planes[:npl].astype(np.float64) + planes[npl:].astype(np.float64)
    n = planes.shape[1]
    flat = planes.transpose(1, 0, 2).reshape(n, -1)
    out = {"x": flat[:, 0:dim], "v": flat[:, dim:2 * dim], "acc": flat[:, L["acc"]:L["acc"] + 1 + dim]}
    if kind == CLOUD_FLA:
        out["J"] = flat[:, L["J"]:L["J"] + dim * dim].reshape(n, dim, dim)
        out["W"] = flat[:, L["W"]:L["W"] + dim * dim].reshape(n, dim, dim)
    return out


class DeviceCloud:
    """A cloud resident on the GPU: state planes, meta words and release table."""

    def __init__(self, kind: int, dim: int, dtype: int, planes: np.ndarray, meta: np.ndarray,
                 batches: np.ndarray, delta: float, device="cuda"):
        torch = _torch()
        self.kind, self.dim, self.dtype, self.delta = kind, dim, dtype, float(delta)
        self.n = int(planes.shape[1])
        self.state = torch.from_numpy(np.ascontiguousarray(planes)).to(device)
        self.meta = torch.from_numpy(np.ascontiguousarray(meta).view(np.int32)).to(device)
        self.batches = torch.from_numpy(np.ascontiguousarray(batches).view(np.uint8)).to(device)
        self.n_batches = int(len(batches))
        self.fold = None
        self.tau_fold = 0.0

    def enable_fold(self, tau: float = TAU_FOLD):
        """Attach the fold guard of single-precision FLA clouds: double-precision J, W
        for droplets with |det J| < tau (see fla_cloud.fold_dev)."""
        torch = _torch()
        nb = lib().fla_fold_bytes(self.dim, self.n)
        self.fold = torch.zeros(max(nb // 8, 4), dtype=torch.float64, device=self.state.device)
        self.tau_fold = float(tau)
        return self

    @classmethod
    def from_seeds(cls, cloud: I.Cloud, dim: int, delta: float, dt: float, dtype: int = F32, device="cuda"):
        npd = np.float32 if dtype == F32 else np.float64
        planes = pack_state(cloud.kind, dim, cloud.n, npd, x=cloud.x0, split=dtype == F32X2)
        meta = meta_words(np.zeros(cloud.n, np.int32), cloud.batch)
        return cls(cloud.kind, dim, dtype, planes, meta, batch_table(cloud, delta, dt), delta, device)

    @classmethod
    def from_state(cls, kind: int, dim: int, dtype: int, *, x, status, batch, batches: np.ndarray, delta=0.0,
                   v=None, J=None, W=None, acc=None, fold=None, fold_J=None, fold_W=None, tau_fold=TAU_FOLD,
                   device="cuda"):
        """Upload a given state.  fold (bool per droplet) with fold_J, fold_W (double
        precision) attaches the fold guard with those droplets inside it."""
        npd = np.float32 if dtype == F32 else np.float64
        n = np.asarray(x).shape[0]
        planes = pack_state(kind, dim, n, npd, x=x, v=v, J=J, W=W, acc=acc, split=dtype == F32X2)
        meta = meta_words(status, batch)
        if fold is not None:
            meta = np.where(np.asarray(fold, bool), meta | META_FOLD, meta).astype(np.uint32)
        c = cls(kind, dim, dtype, planes, meta, batches, delta, device)
        if fold is not None:
            torch = _torch()
            c.enable_fold(tau_fold)
            q = dim * dim
            npl = (2 * q + 3) // 4
            flat = np.zeros((n, npl * 4))
            if fold_J is not None:
                flat[:, :q] = np.asarray(fold_J, np.float64).reshape(n, q)
            if fold_W is not None:
                flat[:, q:2 * q] = np.asarray(fold_W, np.float64).reshape(n, q)
            planes_f = np.ascontiguousarray(flat.reshape(n, npl, 4).transpose(1, 0, 2))
            c.fold[: planes_f.size].copy_(torch.from_numpy(planes_f.ravel()))
        return c

    def snapshot(self) -> dict:
        """Copies of the device buffers a run changes (state planes, meta words,
        fold planes): the cloud's part of a checkpoint at a window boundary."""
        snap = {"state": self.state.clone(), "meta": self.meta.clone()}
        if self.fold is not None:
            snap["fold"] = self.fold.clone()
        return snap

    def restore(self, snap: dict):
        """Back to a snapshot of this cloud (or of one with the same seeds)."""
        if snap["state"].shape != self.state.shape or ("fold" in snap) != (self.fold is not None):
            raise FlaError("checkpoint does not match this cloud")
        self.state.copy_(snap["state"])
        self.meta.copy_(snap["meta"])
        if self.fold is not None:
            self.fold.copy_(snap["fold"])

    def struct(self) -> Cloud:
        c = Cloud()
        c.kind, c.dim, c.dtype, c.n_batches = self.kind, self.dim, self.dtype, self.n_batches
        c.n = self.n
        c.state_dev = self.state.data_ptr()
        c.meta_dev = self.meta.data_ptr()
        c.batches_dev = self.batches.data_ptr()
        c.delta = self.delta
        c.fold_dev = self.fold.data_ptr() if self.fold is not None else None
        c.tau_fold = self.tau_fold
        return c

    def to_host(self) -> dict:
        d = unpack_state(self.kind, self.dim, self.state.cpu().numpy(), split=self.dtype == F32X2)
        meta = self.meta.cpu().numpy().view(np.uint32)
        d["status"] = status_of(meta)
        d["batch"] = (meta & META_BATCH_MASK).astype(np.int32)
        d["fold"] = ((meta & META_FOLD) != 0) & (d["status"] == 1)
        if self.fold is not None:
            q = self.dim * self.dim
            planes = self.fold.cpu().numpy()[: (2 * q + 3) // 4 * self.n * 4].reshape(-1, self.n, 4)
            flat = planes.transpose(1, 0, 2).reshape(self.n, -1)
            d["fold_J"] = flat[:, :q].reshape(self.n, self.dim, self.dim)
            d["fold_W"] = flat[:, q:2 * q].reshape(self.n, self.dim, self.dim)
        return d


def torch_dtype(dtype: int):
    """Element type of a cloud's outputs (compensated clouds deposit in single precision)."""
    torch = _torch()
    return torch.float64 if dtype == F64 else torch.float32


def nodes_buffer(m: Mesh, dtype: int, device="cuda"):
    torch = _torch()
    nbytes = lib().fla_carrier_nodes_bytes(C.byref(m), dtype)
    return torch.empty(nbytes // (8 if dtype == F64 else 4), dtype=torch_dtype(dtype), device=device)


def carrier_sample(ctx: Context, desc: CarrierDesc, m: Mesh, t: float, dtype: int, nodes, stream=None):
    check(lib().fla_carrier_sample(ctx.handle, C.byref(desc), C.byref(m), float(t), dtype, _ptr(nodes),
                                   _stream_ptr(stream)), "fla_carrier_sample")


def advance(ctx: Context, cloud: DeviceCloud, m: Mesh, nodes, step0: int, nsteps: int, dt: float,
            reset_acc: bool = False, stream=None, order=None):
    """fla_advance; with order (n int32 words on the device, a permutation of
    the droplets, e.g. workspace_order) fla_advance_ordered: same results, the
    droplets processed in that order."""
    cs = cloud.struct()
    flags = ADVANCE_RESET_ACC if reset_acc else 0
    if order is None:
        check(lib().fla_advance(ctx.handle, C.byref(cs), C.byref(m), _ptr(nodes), int(step0), int(nsteps),
                                float(dt), flags, _stream_ptr(stream)), "fla_advance")
    else:
        check(lib().fla_advance_ordered(ctx.handle, C.byref(cs), C.byref(m), _ptr(nodes), _ptr(order), int(step0),
                                        int(nsteps), float(dt), flags, _stream_ptr(stream)), "fla_advance_ordered")


def workspace_order(ws, m: Mesh, n: int):
    """The cell-sorted permutation that the last binning of a cloud of n
    droplets left in the (aligned) workspace ws, as an int32 view."""
    torch = _torch()
    off = C.c_size_t()
    check(lib().fla_workspace_order(C.byref(m), int(n), C.byref(off)), "fla_workspace_order")
    return ws[off.value:off.value + 4 * int(n)].view(torch.int32)


def save_checkpoint(path, ck: dict) -> None:
    """Write a checkpoint (Simulation / TwoWay / Batch .checkpoint()) to a file."""
    _torch().save(ck, path)


def load_checkpoint(path, device="cuda") -> dict:
    return _torch().load(path, map_location=device)


def workspace_size(m: Mesh, dtype: int, kernel: int, n: int) -> int:
    out = C.c_size_t()
    check(lib().fla_workspace_size(C.byref(m), dtype, kernel, int(n), C.byref(out)), "fla_workspace_size")
    return out.value


def workspace(m: Mesh, dtype: int, kernel: int, n: int, device="cuda"):
    torch = _torch()
    nb = workspace_size(m, dtype, kernel, n)
    return torch.empty(nb + 256, dtype=torch.uint8, device=device)   # caching allocator blocks are 512-aligned


def n_cells(m: Mesh) -> int:
    return m.n ** m.dim


def cell_bins(ctx: Context, cloud: DeviceCloud, m: Mesh, ws, stream=None):
    torch = _torch()
    nc = n_cells(m)
    keys = torch.empty(max(cloud.n, 1), dtype=torch.int32, device=cloud.state.device)
    perm = torch.empty(max(cloud.n, 1), dtype=torch.int32, device=cloud.state.device)
    bins = torch.empty(nc + 1, dtype=torch.int32, device=cloud.state.device)
    cs = cloud.struct()
    check(lib().fla_cell_bins(ctx.handle, C.byref(cs), C.byref(m), _ptr(keys), _ptr(perm), _ptr(bins), _ptr(ws),
                              ws.numel(), _stream_ptr(stream)), "fla_cell_bins")
    return keys[:cloud.n], perm[:cloud.n], bins


def deposit_cfg(kernel: int, h_min: float, h_max: float, window_dt: float, p: float = 1.0,
                per_cell: bool = False, precision: int = PREC_MIXED, mlp=None, mlp_out=None) -> DepositCfg:
    """mlp: a LearnedCorrection (its packed image), or None for the plain method;
    mlp_out: optional float32 tensor receiving g(f) per droplet."""
    return DepositCfg(int(kernel), 1 if per_cell else 0, float(h_min), float(h_max), float(p), float(window_dt),
                      int(precision), 0, mlp.packed.data_ptr() if mlp is not None else None,
                      mlp_out.data_ptr() if mlp_out is not None else None)


class LearnedCorrection:
    """FP32 master parameters of the bandwidth network and their packed BF16 image."""

    def __init__(self, ctx: "Context", params=None, device="cuda", seed: int = 0, scale: float = 1.0):
        torch = _torch()
        self.ctx = ctx
        if params is None:
            params = init_mlp_params(seed, scale)
        self.params = torch.as_tensor(np.asarray(params, np.float32)).to(device).contiguous()
        assert self.params.numel() == MLP_PARAMS
        self.packed = torch.empty(MLP_PACKED_BYTES, dtype=torch.uint8, device=device)
        self.pack()

    def pack(self, stream=None):
        check(lib().fla_mlp_pack(self.ctx.handle, _ptr(self.params), _ptr(self.packed), _stream_ptr(stream)),
              "fla_mlp_pack")

    def forward(self, features, stream=None):
        """g(f) for a (n, 6) float32 device tensor of features."""
        torch = _torch()
        features = features.contiguous()
        n = features.shape[0]
        out = torch.empty(max(n, 1), dtype=torch.float32, device=features.device)
        check(lib().fla_mlp_forward(self.ctx.handle, _ptr(self.packed), _ptr(features), int(n), _ptr(out),
                                    _stream_ptr(stream)), "fla_mlp_forward")
        return out[:n]


class LearnBuffers:
    """Device buffers of one training sample: the cloud state (fixed), its
    workspaces, the training cells and their targets."""

    def __init__(self, ctx: "Context", cloud: "DeviceCloud", m: "Mesh", cells, targets, kernel: int = KERNEL_ISO):
        torch = _torch()
        dev = cloud.state.device
        self.ctx, self.cloud, self.m = ctx, cloud, m
        self.ws = aligned_ws(workspace(m, F32, kernel, cloud.n, dev))
        nb = C.c_size_t()
        check(lib().fla_learn_workspace_size(ctx.handle, C.byref(m), int(cloud.n), C.byref(nb)),
              "fla_learn_workspace_size")
        self.lws = aligned_ws(torch.empty(nb.value + 256, dtype=torch.uint8, device=dev))
        self.cells = torch.as_tensor(np.asarray(cells, np.int64).astype(np.int32)).to(dev)
        self.targets = torch.as_tensor(np.ascontiguousarray(targets, np.float32)).to(dev)
        self.out = SourceFields(m, F32, dev)


def learn_grad(ctx: "Context", b: LearnBuffers, cfg: DepositCfg, grad, loss, stream=None):
    """Adds this sample's loss to loss[0] and its parameter gradient to grad."""
    cs = b.cloud.struct()
    so = b.out.struct()
    check(lib().fla_learn_grad(ctx.handle, C.byref(cs), C.byref(b.m), C.byref(cfg), _ptr(b.cells),
                               int(b.cells.numel()), _ptr(b.targets), C.byref(so), _ptr(grad), _ptr(loss),
                               _ptr(b.ws), b.ws.numel(), _ptr(b.lws), b.lws.numel(), _stream_ptr(stream)),
          "fla_learn_grad")


def adam_step(ctx: "Context", params, grad, m, v, step: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
              stream=None):
    check(lib().fla_adam_step(ctx.handle, _ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(params.numel()),
                              float(lr), float(beta1), float(beta2), float(eps), int(step), _stream_ptr(stream)),
          "fla_adam_step")


def init_mlp_params(seed: int = 0, scale: float = 1.0, zero_last: bool = False) -> np.ndarray:
    """Seeded initial parameters: uniform +-scale/sqrt(fan_in) weights, zero biases."""
    rng = np.random.default_rng(seed)
    H, F = MLP_HIDDEN, MLP_FEATURES
    parts = []
    for fan_out, fan_in in ((H, F), (H, H), (H, H)):
        parts.append(rng.uniform(-1, 1, fan_out * fan_in) * scale / np.sqrt(fan_in))
        parts.append(np.zeros(fan_out))
    parts.append(np.zeros(H) if zero_last else rng.uniform(-1, 1, H) * scale / np.sqrt(H))
    parts.append(np.zeros(1))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == MLP_PARAMS
    return p


class SourceFields:
    def __init__(self, m: Mesh, dtype: int, device="cuda", with_dsum: bool = True):
        torch = _torch()
        nc = n_cells(m)
        td = torch_dtype(dtype)
        self.s_mass = torch.empty(nc, dtype=td, device=device)
        self.s_mom = torch.empty(m.dim, nc, dtype=td, device=device)
        self.dsum = torch.empty(nc, dtype=td, device=device) if with_dsum else None

    def struct(self) -> Sources:
        return Sources(self.s_mass.data_ptr(), self.s_mom.data_ptr(), self.dsum.data_ptr() if self.dsum is not None else None)


def deposit_sources(ctx: Context, cloud: DeviceCloud, m: Mesh, cfg: DepositCfg, out: SourceFields, ws, stream=None):
    cs = cloud.struct()
    so = out.struct()
    check(lib().fla_deposit_sources(ctx.handle, C.byref(cs), C.byref(m), C.byref(cfg), C.byref(so), _ptr(ws),
                                    ws.numel(), _stream_ptr(stream)), "fla_deposit_sources")


class PsicellFields:
    def __init__(self, m: Mesh, dtype: int, device="cuda"):
        torch = _torch()
        nc = n_cells(m)
        td = torch_dtype(dtype)
        self.counts = torch.empty(nc, dtype=torch.int32, device=device)
        self.s_mass = torch.empty(nc, dtype=td, device=device)
        self.s_mom = torch.empty(m.dim, nc, dtype=td, device=device)

    def struct(self) -> PsicellOut:
        return PsicellOut(self.counts.data_ptr(), self.s_mass.data_ptr(), self.s_mom.data_ptr())


def psicell(ctx: Context, cloud: DeviceCloud, m: Mesh, window_dt: float, out: PsicellFields, ws,
            per_cell: bool = False, stream=None):
    cs = cloud.struct()
    po = out.struct()
    check(lib().psicell_deposit(ctx.handle, C.byref(cs), C.byref(m), float(window_dt), 1 if per_cell else 0,
                                C.byref(po), _ptr(ws), ws.numel(), _stream_ptr(stream)), "psicell_deposit")


def cic(ctx: Context, cloud: DeviceCloud, m: Mesh, window_dt: float, out: PsicellFields, ws, per_cell: bool = False,
        stream=None):
    """Cloud-In-Cell sources of a parcel cloud into out (counts are the box counts)."""
    cs = cloud.struct()
    po = out.struct()
    check(lib().cic_deposit(ctx.handle, C.byref(cs), C.byref(m), float(window_dt), 1 if per_cell else 0,
                            C.byref(po), _ptr(ws), ws.numel(), _stream_ptr(stream)), "cic_deposit")


def aligned_ws(ws):
    """View of a workspace tensor starting on a 256-byte boundary."""
    off = (-ws.data_ptr()) % 256
    return ws[off:]


@dataclass
class RunConfig:
    dtype: int = F32
    deposit: bool = True
    psicell: bool = False


class Simulation:
    """Runs a workload's FLA cloud (and optionally its PSI-CELL parcels) window by
    window on one GPU: carrier sample -> advance (fused window) -> deposit."""

    def __init__(self, ctx: Context, wl: I.Workload, dtype: int = F32, with_psicell: bool = False,
                 device="cuda", precision: int = PREC_MIXED, fold_guard: bool = False,
                 tau_fold: float = TAU_FOLD):
        """precision (single-precision clouds): PREC_MIXED forms det J and n in double
        where det J cancels; PREC_PLAIN keeps them single.  fold_guard (mixed only)
        attaches the advance's fold guard: double-precision J, W while |det J| < tau_fold."""
        self.ctx, self.wl, self.dtype = ctx, wl, dtype
        self.precision, self.fold_guard, self.tau_fold = precision, fold_guard, tau_fold
        self.m = mesh(wl.dim, wl.n_cells_axis)
        self.desc = carrier_desc(wl.carrier)
        self.nodes = nodes_buffer(self.m, dtype, device)
        self.fla = self._fla_cloud(device)
        self.cfg = deposit_cfg(wl.kernel, wl.h_min, wl.h_max, wl.window * wl.dt, wl.p, precision=precision)
        self.out = SourceFields(self.m, dtype, device)
        n_ws = self.fla.n
        self.lpt = None
        if with_psicell and wl.lpt is not None:
            self.lpt = DeviceCloud.from_seeds(wl.lpt, wl.dim, wl.delta, wl.dt, dtype, device)
            self.psi = PsicellFields(self.m, dtype, device)
            n_ws = max(n_ws, self.lpt.n)
        self.ws = aligned_ws(workspace(self.m, dtype, wl.kernel, n_ws, device))
        self.step = 0
        self._sampled_t = None
        self._binned = None   # the cloud whose cell-sorted order self.ws holds

    def _order(self, c):
        return workspace_order(self.ws, self.m, c.n) if self._binned is c else None

    def reset(self):
        """Back to the seeds (device-side copies only re-upload the initial planes)."""
        wl = self.wl
        self.fla = self._fla_cloud(self.fla.state.device)
        if self.lpt is not None:
            self.lpt = DeviceCloud.from_seeds(wl.lpt, wl.dim, wl.delta, wl.dt, self.dtype, self.lpt.state.device)
        self.step = 0
        self._sampled_t = None
        self._binned = None

    def checkpoint(self) -> dict:
        """The run at a window boundary: its step and copies of its clouds' device
        buffers (torch.save-able).  restore() on a Simulation of the same workload
        and form continues it with results bit for bit those of the uninterrupted
        run: the advance and the deposit read nothing else that carries over."""
        ck = {"step": self.step, "fla": self.fla.snapshot()}
        if self.lpt is not None:
            ck["lpt"] = self.lpt.snapshot()
        return ck

    def restore(self, ck: dict):
        self.fla.restore(ck["fla"])
        if self.lpt is not None:
            self.lpt.restore(ck["lpt"])
        self.step = int(ck["step"])
        self._sampled_t = None
        self._binned = None   # the workspace's order belongs to no restored cloud

    def _fla_cloud(self, device):
        wl = self.wl
        c = DeviceCloud.from_seeds(wl.fla, wl.dim, wl.delta, wl.dt, self.dtype, device)
        if self.dtype == F32 and self.precision == PREC_MIXED and self.fold_guard:
            c.enable_fold(self.tau_fold)
        return c

    def window(self, deposit: bool = True, with_psicell: bool = True, stream=None):
        wl = self.wl
        k = min(wl.window, wl.nsteps - self.step) if wl.nsteps > self.step else wl.window
        t_c = self.step * wl.dt if not wl.carrier.steady else 0.0
        if self._sampled_t != t_c:
            carrier_sample(self.ctx, self.desc, self.m, t_c, self.dtype, self.nodes, stream)
            self._sampled_t = t_c
        advance(self.ctx, self.fla, self.m, self.nodes, self.step, k, wl.dt, reset_acc=True, stream=stream,
                order=self._order(self.fla))
        if self.lpt is not None:
            advance(self.ctx, self.lpt, self.m, self.nodes, self.step, k, wl.dt, reset_acc=True, stream=stream,
                    order=self._order(self.lpt))
        self.step += k
        if deposit:
            deposit_sources(self.ctx, self.fla, self.m, self.cfg, self.out, self.ws, stream)
            self._binned = self.fla
        if with_psicell and self.lpt is not None:
            psicell(self.ctx, self.lpt, self.m, wl.window * wl.dt, self.psi, self.ws, stream=stream)
            self._binned = self.lpt

    def run(self, nsteps: int | None = None, deposit_every: bool = True, stream=None):
        total = self.wl.nsteps if nsteps is None else nsteps
        while self.step < total:
            last = self.step + self.wl.window >= total
            self.window(deposit=deposit_every or last, with_psicell=deposit_every or last, stream=stream)


class Batch:
    """Many single-precision FLA clouds (one Workload each, same dt and window)
    advanced and deposited together by the batched launches of fla_batch_run."""

    def __init__(self, ctx: "Context", workloads, device="cuda", step0: int = 0):
        torch = _torch()
        self.ctx, self.workloads = ctx, list(workloads)
        wl0 = self.workloads[0]
        self.dt, self.window = wl0.dt, wl0.window
        self.clouds, self.meshes, self.nodes, self.outs, self.cfgs = [], [], [], [], []
        items = (BatchItem * len(self.workloads))()
        for k, wl in enumerate(self.workloads):
            assert wl.dt == self.dt and wl.window == self.window
            m = mesh(wl.dim, wl.n_cells_axis)
            c = DeviceCloud.from_seeds(wl.fla, wl.dim, wl.delta, wl.dt, F32, device)
            nodes = nodes_buffer(m, F32, device)
            out = SourceFields(m, F32, device)
            cfg = deposit_cfg(wl.kernel, wl.h_min, wl.h_max, wl.window * wl.dt, wl.p)
            items[k].cloud = c.struct()
            items[k].mesh = m
            items[k].carrier = carrier_desc(wl.carrier)
            items[k].nodes_dev = nodes.data_ptr()
            items[k].cfg = cfg
            items[k].out = out.struct()
            self.clouds.append(c)
            self.meshes.append(m)
            self.nodes.append(nodes)
            self.outs.append(out)
            self.cfgs.append(cfg)
        self._items = items
        nb = C.c_size_t()
        check(lib().fla_batch_workspace_size(items, len(self.workloads), C.byref(nb)), "fla_batch_workspace_size")
        self.ws = aligned_ws(torch.empty(nb.value + 256, dtype=torch.uint8, device=device))
        self.pristine = [(c.state.clone(), c.meta.clone()) for c in self.clouds]
        torch.cuda.synchronize()
        h = C.c_void_p()
        check(lib().fla_batch_create(ctx.handle, items, len(self.workloads), float(self.dt), int(self.window),
                                     int(step0), _ptr(self.ws), self.ws.numel(), C.byref(h)), "fla_batch_create")
        self.handle = h
        self.step = int(step0)
        self.n_droplets = sum(c.n for c in self.clouds)
        self.n_cells = sum(m.n ** m.dim for m in self.meshes)

    def run(self, n_windows: int, stream=None):
        check(lib().fla_batch_run(self.ctx.handle, self.handle, int(n_windows), _stream_ptr(stream)), "fla_batch_run")
        self.step += int(n_windows) * self.window

    def set_step(self, step: int, stream=None):
        check(lib().fla_batch_set_step(self.handle, int(step), _stream_ptr(stream)), "fla_batch_set_step")
        self.step = int(step)

    def reset(self, stream=None):
        """Seeds back in place and the device step at 0."""
        for c, (st, me) in zip(self.clouds, self.pristine):
            c.state.copy_(st)
            c.meta.copy_(me)
        self.set_step(0, stream)

    def checkpoint(self) -> dict:
        """Every cloud's device buffers and the step of the next window (the
        run's host-side count of the windows issued through run())."""
        return {"step": self.step, "clouds": [c.snapshot() for c in self.clouds]}

    def restore(self, ck: dict, stream=None):
        if len(ck["clouds"]) != len(self.clouds):
            raise FlaError("checkpoint does not match this batch")
        for c, snap in zip(self.clouds, ck["clouds"]):
            c.restore(snap)
        self.set_step(int(ck["step"]), stream)

    def tuning(self) -> dict:
        a, g, o, n = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        rc = lib().fla_batch_tuning(self.handle, C.byref(a), C.byref(g), C.byref(o), C.byref(n))
        return {"tuned": rc == 0, "advance_threads": a.value, "gather_ctas_per_sm": g.value,
                "tile_order": ["natural", "interleaved"][o.value], "launches_per_window": n.value}

    def set_tuning(self, advance_threads: int, gather_ctas_per_sm: int, tile_order: int):
        check(lib().fla_batch_set_tuning(self.handle, int(advance_threads), int(gather_ctas_per_sm), int(tile_order)),
              "fla_batch_set_tuning")

    def set_mode(self, mode: int):
        check(lib().fla_batch_set_mode(self.handle, int(mode)), "fla_batch_set_mode")

    def mode(self) -> dict:
        m, tp, tl = C.c_int32(), C.c_float(), C.c_float()
        check(lib().fla_batch_mode(self.handle, C.byref(m), C.byref(tp), C.byref(tl)), "fla_batch_mode")
        return {"mode": ["auto", "launches", "persistent"][m.value], "persistent_ms": tp.value,
                "launches_ms": tl.value}

    def close(self):
        if getattr(self, "handle", None):
            lib().fla_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class NavierStokes:
    """The two-way carrier (fla_ns_*): its state in a device workspace."""

    def __init__(self, ctx: "Context", n: int, nu: float, diff: float, dt: float, omega, mean_u=(0.0, 0.0),
                 rho=None, device="cuda", stream=None, body=None):
        """body: None, or a mapping with xc, yc, r, eta and optionally fringe_x0,
        fringe_x1, fringe_sigma, hold_mean_flow (default True): an immersed
        cylinder by volume penalisation (fla_ns_cfg)."""
        torch = _torch()
        self.ctx = ctx
        self.cfg = NSConfig(int(n), float(nu), float(diff), float(dt))
        if body is not None:
            self.cfg.body = 1
            self.cfg.hold_mean_flow = 1 if body.get("hold_mean_flow", True) else 0
            self.cfg.body_xc, self.cfg.body_yc = float(body["xc"]), float(body["yc"])
            self.cfg.body_r, self.cfg.body_eta = float(body["r"]), float(body["eta"])
            self.cfg.fringe_x0 = float(body.get("fringe_x0", 0.0))
            self.cfg.fringe_x1 = float(body.get("fringe_x1", 0.0))
            self.cfg.fringe_sigma = float(body.get("fringe_sigma", 0.0))
        nb = lib().fla_ns_workspace_size(C.byref(self.cfg))
        if nb == 0:
            raise FlaError("invalid two-way carrier configuration")
        self.ws = aligned_ws(torch.empty(nb + 256, dtype=torch.uint8, device=device))
        w = torch.as_tensor(np.ascontiguousarray(omega, np.float64).reshape(-1)).to(device)
        r = None if rho is None else torch.as_tensor(np.ascontiguousarray(rho, np.float64).reshape(-1)).to(device)
        U = (C.c_double * 2)(*[float(x) for x in mean_u])
        self._keep = (w, r, U)
        self.reset(stream)

    def snapshot(self) -> dict:
        """A copy of the carrier's workspace (its fields and mean flow, stored at
        offsets, so any workspace of the same configuration can take it back)."""
        return {"ws": self.ws.clone()}

    def restore(self, snap: dict):
        if snap["ws"].numel() != self.ws.numel():
            raise FlaError("checkpoint does not match this carrier")
        self.ws.copy_(snap["ws"])

    def reset(self, stream=None):
        """Back to the initial state."""
        w, r, U = self._keep
        check(lib().fla_ns_init(self.ctx.handle, C.byref(self.cfg), _ptr(w), U, _ptr(r) if r is not None else None,
                                _ptr(self.ws), self.ws.numel(), _stream_ptr(stream)), "fla_ns_init")

    def step(self, nsub: int, sources: "SourceFields | None" = None, stream=None):
        sm = sv = None
        dt = F32
        if sources is not None:
            sm, sv = _ptr(sources.s_mass), _ptr(sources.s_mom)
            dt = F64 if sources.s_mass.dtype == _torch().float64 else F32
        check(lib().fla_ns_step(self.ctx.handle, C.byref(self.cfg), sm, sv, dt, int(nsub), _ptr(self.ws),
                                self.ws.numel(), _stream_ptr(stream)), "fla_ns_step")

    def nodes(self, dtype: int, out, stream=None):
        check(lib().fla_ns_nodes(self.ctx.handle, C.byref(self.cfg), dtype, _ptr(out), _ptr(self.ws),
                                 self.ws.numel(), _stream_ptr(stream)), "fla_ns_nodes")

    def body_force(self, stream=None) -> np.ndarray:
        """Force of the fluid on the cylinder (2 values)."""
        F = (C.c_double * 2)()
        check(lib().fla_ns_body_force(self.ctx.handle, C.byref(self.cfg), F, _ptr(self.ws), self.ws.numel(),
                                      _stream_ptr(stream)), "fla_ns_body_force")
        return np.array([F[0], F[1]])

    def fields(self, stream=None) -> dict:
        torch = _torch()
        n = self.cfg.n
        dev = self.ws.device
        w, p, r = (torch.empty(n * n, dtype=torch.float64, device=dev) for _ in range(3))
        U = (C.c_double * 2)()
        check(lib().fla_ns_fields(self.ctx.handle, C.byref(self.cfg), _ptr(w), _ptr(p), _ptr(r), U, _ptr(self.ws),
                                  self.ws.numel(), _stream_ptr(stream)), "fla_ns_fields")
        return {"omega": w.cpu().numpy().reshape(n, n), "psi": p.cpu().numpy().reshape(n, n),
                "rho": r.cpu().numpy().reshape(n, n), "U": np.array([U[0], U[1]])}


class TwoWay:
    """Two-way coupled run of a 2D workload on the periodic carrier (App. B):
    per window the carrier's node values feed the droplet advance (frozen over
    the window), the kernel-regression deposit gives S_Mass and S_Mom, and the
    carrier takes the window's steps with those sources."""

    def __init__(self, ctx: "Context", wl: I.Workload, ns: NavierStokes, dtype: int = F32, device="cuda",
                 coupled: bool = True):
        assert wl.dim == 2 and wl.n_cells_axis == ns.cfg.n
        self.ctx, self.wl, self.ns, self.dtype, self.coupled = ctx, wl, ns, dtype, coupled
        self.m = mesh(2, wl.n_cells_axis)
        self.nodes = nodes_buffer(self.m, dtype, device)
        self.fla = DeviceCloud.from_seeds(wl.fla, 2, wl.delta, wl.dt, dtype, device)
        self.cfg = deposit_cfg(wl.kernel, wl.h_min, wl.h_max, wl.window * wl.dt, wl.p)
        self.out = SourceFields(self.m, dtype, device)
        self.ws = aligned_ws(workspace(self.m, dtype, wl.kernel, self.fla.n, device))
        self.step = 0
        self._restored = False
        self._seeds = (self.fla.state.clone(), self.fla.meta.clone())

    def reset(self, stream=None):
        """Droplets back to their seeds and the carrier to its initial state."""
        self.fla.state.copy_(self._seeds[0])
        self.fla.meta.copy_(self._seeds[1])
        self.ns.reset(stream)
        self.step = 0

    def checkpoint(self) -> dict:
        """Droplets, carrier and step at a window boundary (torch.save-able)."""
        return {"step": self.step, "fla": self.fla.snapshot(), "ns": self.ns.snapshot(),
                "sources": (self.out.s_mass.clone(), self.out.s_mom.clone())}

    def restore(self, ck: dict):
        self.fla.restore(ck["fla"])
        self.ns.restore(ck["ns"])
        self.out.s_mass.copy_(ck["sources"][0])
        self.out.s_mom.copy_(ck["sources"][1])
        # the next window's order comes from a deposit into this object's
        # workspace, which a restored run has not made yet
        self.step = int(ck["step"])
        self._restored = True

    def window(self, stream=None):
        wl = self.wl
        k = wl.window
        self.ns.nodes(self.dtype, self.nodes, stream)
        # after the first window the workspace holds the droplets' cell-sorted order
        order = workspace_order(self.ws, self.m, self.fla.n) if self.step > 0 and not self._restored else None
        self._restored = False
        advance(self.ctx, self.fla, self.m, self.nodes, self.step, k, wl.dt, reset_acc=True, stream=stream,
                order=order)
        deposit_sources(self.ctx, self.fla, self.m, self.cfg, self.out, self.ws, stream)
        self.ns.step(k, self.out if self.coupled else None, stream)
        self.step += k

    def run(self, n_windows: int, stream=None):
        for _ in range(n_windows):
            self.window(stream)
