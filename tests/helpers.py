"""Shared helpers of the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np

from oracle import oracle as O
from paper_2512_20829_gb300 import fla
from paper_2512_20829_gb300 import inputs as I


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))


def gpu_cloud_from_state(s: I.CloudState, dtype: int, kind: int = fla.CLOUD_FLA, weights=None):
    """Upload a synthetic cloud state; weights (LPT) go to the release table's n0."""
    nb = len(s.n0)
    t = np.zeros(nb, fla.BATCH_DTYPE)
    t["St0"] = 1.0
    t["n0"] = s.n0 if weights is None else weights
    t["h0"] = s.h0
    t["step_dead"] = 2**31 - 1
    kw = dict(x=s.x, v=s.v, acc=s.acc)
    if kind == fla.CLOUD_FLA:
        kw.update(J=s.J, W=s.W)
    return fla.DeviceCloud.from_state(kind, s.dim, dtype, status=s.status, batch=s.batch, batches=t, **kw)


def oracle_deposit(s: I.CloudState, N: int, kernel: int, h_min: float, h_max: float, window_dt: float,
                   fp32: bool, p: float = 1.0, cells=None):
    D = O.dep_struct(dim=s.dim, N=N, kernel=kernel, h_min=h_min, h_max=h_max, p=p, window_dt=window_dt,
                     fp32_decision=fp32)
    return O.nw_deposit(D, s.x, s.J, s.acc, s.status, s.batch, s.n0, s.h0, cells=cells)


def oracle_scale(s: I.CloudState, N: int, kernel: int, h_min, h_max, window_dt, fp32, cells=None):
    """sum_i K_i |a_i| / D_c per cell and component: the size of the terms each
    source value averages, used to scale element-wise tolerances."""
    absd = I.CloudState(**{**s.__dict__, "acc": np.abs(s.acc)})
    m, v, _ = oracle_deposit(absd, N, kernel, h_min, h_max, window_dt, fp32, cells=cells)
    return np.abs(m), np.abs(v)
