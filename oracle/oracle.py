"""Python front end of the FP64 CPU oracle (``fla_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It never imports the CUDA package;
its only shared input is the seeded workload description in
``paper_2512_20829_gb300.inputs`` (data, not arithmetic).

The C library computes everything; this module marshals NumPy arrays and
supplies two library primitives the oracle is allowed to lean on: NumPy's
stable argsort (the cell-key sort) and ``searchsorted`` (bin starts).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fla_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

PENDING, ACTIVE, DEAD = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no contraction),
    with OpenMP when the compiler has it (the results do not depend on it)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int) -> None:
    """Host threads of the oracle's independent loops (droplets of a step, cells)."""
    lib().ora_set_threads(int(n))


def threads() -> int:
    return int(lib().ora_threads())


class _Carrier(C.Structure):
    _fields_ = [("kind", C.c_int), ("dim", C.c_int), ("U", C.c_double * 3), ("A", C.c_double * 9),
                ("xref", C.c_double * 3), ("n_vort", C.c_int), ("vort", C.c_double * 80),
                ("jet_width", C.c_double), ("abc", C.c_double * 3), ("jet_amp", C.c_double),
                ("jet_radius", C.c_double)]


class _Setup(C.Structure):
    _fields_ = [("dim", C.c_int), ("N", C.c_int), ("cloud", C.c_int), ("dt", C.c_double),
                ("delta", C.c_double), ("car", C.POINTER(_Carrier)), ("use_mesh", C.c_int),
                ("carrier_period", C.c_int), ("n_batches", C.c_int),
                ("step_start", C.POINTER(C.c_int)), ("step_dead", C.POINTER(C.c_int)),
                ("St0", C.POINTER(C.c_double)), ("given_nodes", C.POINTER(C.c_double))]


class _Dep(C.Structure):
    _fields_ = [("dim", C.c_int), ("N", C.c_int), ("kernel", C.c_int), ("h_min", C.c_double),
                ("h_max", C.c_double), ("p", C.c_double), ("window_dt", C.c_double),
                ("per_cell", C.c_int), ("fp32_decision", C.c_int), ("plain", C.c_int),
                ("fold", C.c_void_p), ("mlp", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, v = C.c_double, C.c_int, C.c_void_p
        _lib.ora_carrier_eval.argtypes = [C.POINTER(_Carrier), d, v, v, v]
        _lib.ora_carrier_nodes.argtypes = [C.POINTER(_Carrier), d, i, v]
        _lib.ora_interp.argtypes = [v, i, i, v, v, v]
        _lib.ora_step_dead.argtypes = [d, d, d, i]
        _lib.ora_step_dead.restype = i
        _lib.ora_advance.argtypes = [C.POINTER(_Setup), i, i, i, v, v, v, v, i]
        _lib.ora_cell_keys.argtypes = [i, i, i, v, v, i, v]
        _lib.ora_nw_deposit.argtypes = [C.POINTER(_Dep), i, v, v, v, v, v, v, v, C.c_long, v, v, v, v]
        _lib.ora_nw_deposit_celllist.argtypes = [C.POINTER(_Dep), i, v, v, v, v, v, v, v, v, v, v]
        _lib.ora_nw_deposit_celllist_cells.argtypes = [C.POINTER(_Dep), i, v, v, v, v, v, v, v, C.c_long, v,
                                                       v, v, v]
        _lib.ora_kernel_on_cells.argtypes = [C.POINTER(_Dep), v, v, d, d, i, v]
        _lib.ora_records.argtypes = [C.POINTER(_Dep), i, v, v, v, v, v, v, v]
        _lib.ora_psicell.argtypes = [C.POINTER(_Dep), i, v, v, v, v, v, i, v, v, v]
        _lib.ora_mlp_nparam.restype = i
        _lib.ora_mlp_set_exact.argtypes = [i]
        _lib.ora_mlp_features.argtypes = [i, v, d, d, d, v]
        _lib.ora_mlp_forward_batch.argtypes = [v, i, v, v, v, v]
        _lib.ora_mlp_backward.argtypes = [v, v, d, v]
        _lib.ora_learn_loss_grad.argtypes = [C.POINTER(_Dep), i, v, v, v, v, v, v, v, C.c_long, v, v, v, v]
        _lib.ora_learn_records.argtypes = [C.POINTER(_Dep), i, v, v, v, v, v, v, v, v, v]
        _lib.ora_set_threads.argtypes = [i]
        _lib.ora_cic.argtypes = [C.POINTER(_Dep), i, v, v, v, v, v, i, v, v, v]
        _lib.ora_cic_celllist.argtypes = [C.POINTER(_Dep), i, v, v, v, v, v, i, v, v, v]
        _lib.ora_decision_audit.argtypes = [C.POINTER(_Dep), i, v, v, v, v, v, v, v, C.c_long, v, C.c_long, v, v,
                                            v, v]
        _lib.ora_decision_audit.restype = C.c_long
        _lib.ora_threads.restype = i
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def carrier_struct(car) -> _Carrier:
    c = _Carrier()
    c.kind, c.dim = int(car.kind), int(car.dim)
    for k in range(3):
        c.U[k] = float(np.asarray(car.U).ravel()[k]) if np.asarray(car.U).size > k else 0.0
        c.xref[k] = float(np.asarray(car.xref).ravel()[k]) if np.asarray(car.xref).size > k else 0.0
        c.abc[k] = float(car.abc[k])
    A = np.zeros((3, 3))
    Ai = np.asarray(car.A, dtype=np.float64)
    A[:Ai.shape[0], :Ai.shape[1]] = Ai
    for k in range(9):
        c.A[k] = A.ravel()[k]
    vt = np.asarray(car.vortices, dtype=np.float64).reshape(-1, 5)
    assert vt.shape[0] <= 16
    c.n_vort = vt.shape[0]
    for k, val in enumerate(vt.ravel()):
        c.vort[k] = val
    c.jet_width, c.jet_amp, c.jet_radius = float(car.jet_width), float(car.jet_amp), float(car.jet_radius)
    return c


def carrier_eval(car, t: float, x) -> tuple[np.ndarray, np.ndarray]:
    c = carrier_struct(car)
    d = car.dim
    x = _f64(x)
    u = np.zeros(d)
    G = np.zeros(d * d)
    lib().ora_carrier_eval(C.byref(c), t, _p(x), _p(u), _p(G))
    return u, G.reshape(d, d)


def carrier_nodes(car, t: float, N: int) -> np.ndarray:
    c = carrier_struct(car)
    d = car.dim
    out = np.zeros(((N + 1) ** d, d + d * d))
    lib().ora_carrier_nodes(C.byref(c), t, N, _p(out))
    return out


def interp(nodes: np.ndarray, d: int, N: int, x) -> tuple[np.ndarray, np.ndarray]:
    x = _f64(x)
    u = np.zeros(d)
    G = np.zeros(d * d)
    lib().ora_interp(_p(_f64(nodes)), d, N, _p(x), _p(u), _p(G))
    return u, G.reshape(d, d)


def step_dead(St0: float, delta: float, dt: float, step_start: int) -> int:
    return int(lib().ora_step_dead(St0, delta, dt, int(step_start)))


@dataclass
class State:
    """Oracle state of a cloud: y = (x, v[, J, W]) per droplet, window sums, status."""
    dim: int
    cloud: int
    y: np.ndarray        # (n, ny)
    acc: np.ndarray      # (n, 1+dim)
    status: np.ndarray   # (n,) int32
    batch: np.ndarray    # (n,) int32

    @property
    def x(self):
        return self.y[:, :self.dim]

    @property
    def v(self):
        return self.y[:, self.dim:2 * self.dim]

    @property
    def J(self):
        d = self.dim
        return self.y[:, 2 * d:2 * d + d * d].reshape(-1, d, d)

    @property
    def W(self):
        d = self.dim
        return self.y[:, 2 * d + d * d:2 * d + 2 * d * d].reshape(-1, d, d)


def initial_state(cloud, dim: int) -> State:
    n = cloud.n
    ny = 2 * dim + 2 * dim * dim if cloud.kind == 0 else 2 * dim
    y = np.zeros((n, ny))
    y[:, :dim] = cloud.x0
    return State(dim=dim, cloud=cloud.kind, y=y, acc=np.zeros((n, 1 + dim)),
                 status=np.zeros(n, np.int32), batch=_i32(cloud.batch))


class Advancer:
    """Holds the ctypes setup for one cloud and carrier."""

    def __init__(self, wl, cloud, *, use_mesh: bool = True, carrier=None, dt=None, delta=None):
        car = carrier if carrier is not None else wl.carrier
        self.car = carrier_struct(car)
        self.dim = wl.dim
        self.step_start = _i32(cloud.step_start)
        self.St0 = _f64(cloud.St0)
        dt = wl.dt if dt is None else dt
        delta = wl.delta if delta is None else delta
        self.step_dead = _i32([step_dead(float(s), delta, dt, int(ss))
                               for s, ss in zip(self.St0, self.step_start)])
        S = _Setup()
        S.dim, S.N, S.cloud = wl.dim, wl.n_cells_axis, int(cloud.kind)
        S.dt, S.delta = dt, delta
        S.car = C.pointer(self.car)
        S.use_mesh = 1 if use_mesh else 0
        S.carrier_period = 0 if car.steady else wl.window
        S.n_batches = len(self.St0)
        S.step_start = self.step_start.ctypes.data_as(C.POINTER(C.c_int))
        S.step_dead = self.step_dead.ctypes.data_as(C.POINTER(C.c_int))
        S.St0 = self.St0.ctypes.data_as(C.POINTER(C.c_double))
        self.S = S

    def advance(self, st: State, step0: int, nsteps: int, reset_acc: bool = False, nodes=None) -> State:
        """nodes: carrier node values ((N+1)^d, d + d*d) to use instead of the
        analytic carrier, e.g. the two-way carrier's (carrier_ns.carrier_nodes)."""
        assert st.y.flags.c_contiguous and st.acc.flags.c_contiguous
        keep = None
        if nodes is not None:
            d = self.dim
            keep = np.ascontiguousarray(np.asarray(nodes, np.float64)[:, :d + d * d])
            self.S.given_nodes = keep.ctypes.data_as(C.POINTER(C.c_double))
        else:
            self.S.given_nodes = None
        lib().ora_advance(C.byref(self.S), int(step0), int(nsteps), st.y.shape[0], _p(st.y), _p(st.acc),
                          _p(st.status), _p(st.batch), 1 if reset_acc else 0)
        self.S.given_nodes = None
        del keep
        return st


def dep_struct(wl=None, *, dim=None, N=None, kernel=None, h_min=None, h_max=None, p=None,
               window_dt=None, per_cell=False, fp32_decision=False, plain=False, fold=None, mlp=None) -> _Dep:
    """Deposit settings.  plain: det J decided in single precision (plain mode);
    fold: per-droplet flags of J given as the fold guard's double-precision copy
    (the array is kept alive on the returned struct)."""
    D = _Dep()
    D.dim = dim if dim is not None else wl.dim
    D.N = N if N is not None else wl.n_cells_axis
    D.kernel = kernel if kernel is not None else wl.kernel
    D.h_min = h_min if h_min is not None else wl.h_min
    D.h_max = h_max if h_max is not None else wl.h_max
    D.p = p if p is not None else (wl.p if wl is not None else 1.0)
    D.window_dt = window_dt if window_dt is not None else wl.window * wl.dt
    D.per_cell = 1 if per_cell else 0
    D.fp32_decision = 1 if fp32_decision else 0
    D.plain = 1 if plain else 0
    if fold is not None:
        D._fold_keep = np.ascontiguousarray(fold, dtype=np.int32)
        D.fold = D._fold_keep.ctypes.data
    else:
        D.fold = None
    if mlp is not None:
        D._mlp_keep = np.ascontiguousarray(mlp, dtype=np.float32)
        D.mlp = D._mlp_keep.ctypes.data
    else:
        D.mlp = None
    return D


def nw_deposit(D: _Dep, x, J, acc, status, batch, n0, h0, cells=None):
    """Brute-force Nadaraya-Watson deposit; returns (S_mass, S_mom, Dsum)."""
    d = D.dim
    x, J, acc = _f64(x).reshape(-1, d), _f64(J).reshape(-1, d * d), _f64(acc).reshape(-1, 1 + d)
    status, batch = _i32(status), _i32(batch)
    n = x.shape[0]
    if cells is None:
        n_out = D.N ** d
        cptr = None
    else:
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        n_out = cells.shape[0]
        cptr = _p(cells)
    Sm = np.zeros(n_out)
    Sv = np.zeros((n_out, d))
    Ds = np.zeros(n_out)
    lib().ora_nw_deposit(C.byref(D), n, _p(x), _p(J), _p(acc), _p(status), _p(batch),
                         _p(_f64(n0)), _p(_f64(h0)), n_out, cptr, _p(Sm), _p(Sv), _p(Ds))
    return Sm, Sv, Ds


def nw_deposit_celllist(D: _Dep, x, J, acc, status, batch, n0, h0, cells=None):
    """Cell-list deposit (bit-identical to the brute force); cells limits it to a list."""
    d = D.dim
    x, J, acc = _f64(x).reshape(-1, d), _f64(J).reshape(-1, d * d), _f64(acc).reshape(-1, 1 + d)
    status, batch = _i32(status), _i32(batch)
    if cells is None:
        n_out, cptr = D.N ** d, None
    else:
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        n_out, cptr = cells.shape[0], _p(cells)
    Sm = np.zeros(n_out)
    Sv = np.zeros((n_out, d))
    Ds = np.zeros(n_out)
    lib().ora_nw_deposit_celllist_cells(C.byref(D), x.shape[0], _p(x), _p(J), _p(acc), _p(status), _p(batch),
                                        _p(_f64(n0)), _p(_f64(h0)), n_out, cptr, _p(Sm), _p(Sv), _p(Ds))
    return Sm, Sv, Ds


def decision_audit(D: _Dep, x, J, acc, status, batch, n0, h0, cells, max_out=100_000):
    """Pairs whose single-precision truncation decision (D.fp32_decision = 1) differs
    from q <= 9 in double: (list positions of the cells, droplets, q in double) and
    the number of pairs inside the double-precision support."""
    assert D.fp32_decision == 1
    d = D.dim
    x, J, acc = _f64(x).reshape(-1, d), _f64(J).reshape(-1, d * d), _f64(acc).reshape(-1, 1 + d)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    oc = np.zeros(max_out, np.int64)
    od = np.zeros(max_out, np.int32)
    oq = np.zeros(max_out)
    inside = C.c_long(0)
    found = lib().ora_decision_audit(C.byref(D), x.shape[0], _p(x), _p(J), _p(acc), _p(_i32(status)),
                                     _p(_i32(batch)), _p(_f64(n0)), _p(_f64(h0)), cells.shape[0], _p(cells),
                                     max_out, _p(oc), _p(od), _p(oq), C.byref(inside))
    k = min(found, max_out)
    return oc[:k], od[:k], oq[:k], int(found), int(inside.value)


def kernel_on_cells(D: _Dep, x, J, n0: float, h0: float, normalised: bool) -> np.ndarray:
    d = D.dim
    out = np.zeros(D.N ** d)
    lib().ora_kernel_on_cells(C.byref(D), _p(_f64(x)), _p(_f64(J).ravel()), n0, h0,
                              1 if normalised else 0, _p(out))
    return out


def records(D: _Dep, x, J, acc, batch, n0, h0) -> np.ndarray:
    """Per droplet (n, det J, h, prefactor)."""
    d = D.dim
    x, J, acc = _f64(x).reshape(-1, d), _f64(J).reshape(-1, d * d), _f64(acc).reshape(-1, 1 + d)
    out = np.zeros((x.shape[0], 4))
    lib().ora_records(C.byref(D), x.shape[0], _p(x), _p(J), _p(acc), _p(_i32(batch)),
                      _p(_f64(n0)), _p(_f64(h0)), _p(out))
    return out


def cell_keys(d: int, N: int, x, status, fp32: bool) -> np.ndarray:
    x = _f64(x).reshape(-1, d)
    keys = np.zeros(x.shape[0], np.uint32)
    lib().ora_cell_keys(d, N, x.shape[0], _p(x), _p(_i32(status)), 1 if fp32 else 0, _p(keys))
    return keys


def sort_and_bins(keys: np.ndarray, n_cells: int):
    """Stable sort of (key, index) and bin starts: the cell list of the deposits."""
    perm = np.argsort(keys, kind="stable").astype(np.uint32)
    sk = keys[perm]
    bin_start = np.searchsorted(sk, np.arange(n_cells + 1, dtype=np.uint64), side="left").astype(np.uint32)
    return sk, perm, bin_start


def cic(D: _Dep, x, acc, status, batch, w, brute: bool = False, fp32_keys: bool = False):
    """Cloud-In-Cell sources (tent weights to the cell centres around each parcel)
    and the box counts (keys in single precision with fp32_keys); brute: over every
    parcel for each cell, else the cell list."""
    d = D.dim
    x, acc = _f64(x).reshape(-1, d), _f64(acc).reshape(-1, 1 + d)
    nc = D.N ** d
    counts = np.zeros(nc, np.uint32)
    Sm = np.zeros(nc)
    Sv = np.zeros((nc, d))
    f = lib().ora_cic if brute else lib().ora_cic_celllist
    f(C.byref(D), x.shape[0], _p(x), _p(acc), _p(_i32(status)), _p(_i32(batch)), _p(_f64(w)), 1 if fp32_keys else 0,
      _p(counts), _p(Sm), _p(Sv))
    return counts, Sm, Sv


def psicell(D: _Dep, x, acc, status, batch, w, fp32_keys: bool):
    d = D.dim
    x, acc = _f64(x).reshape(-1, d), _f64(acc).reshape(-1, 1 + d)
    nc = D.N ** d
    counts = np.zeros(nc, np.uint32)
    Sm = np.zeros(nc)
    Sv = np.zeros((nc, d))
    lib().ora_psicell(C.byref(D), x.shape[0], _p(x), _p(acc), _p(_i32(status)), _p(_i32(batch)),
                      _p(_f64(w)), 1 if fp32_keys else 0, _p(counts), _p(Sm), _p(Sv))
    return counts, Sm, Sv


def run(wl, cloud=None, *, nsteps=None, use_mesh=True, deposit_every_window=False, advancer=None):
    """Integrate a workload's cloud from step 0 with window resets; returns the final
    state (window sums cover the last window)."""
    cloud = cloud if cloud is not None else wl.fla
    nsteps = wl.nsteps if nsteps is None else nsteps
    adv = advancer or Advancer(wl, cloud, use_mesh=use_mesh)
    st = initial_state(cloud, wl.dim)
    s = 0
    while s < nsteps:
        k = min(wl.window, nsteps - s)
        adv.advance(st, s, k, reset_acc=True)
        s += k
    return st


# ---------------------------------------------------------------------------
# Learned bandwidth correction (no counterpart in the paper)

MLP_IN, MLP_HIDDEN = 6, 64


def mlp_nparam() -> int:
    return lib().ora_mlp_nparam()


class exact_mlp:
    """Context: evaluate the network without any bfloat16 rounding."""

    def __enter__(self):
        lib().ora_mlp_set_exact(1)

    def __exit__(self, *a):
        lib().ora_mlp_set_exact(0)


def mlp_features(d: int, J, n0, h0, dx: float) -> np.ndarray:
    J = _f64(J).reshape(-1, d * d)
    n = J.shape[0]
    n0 = np.broadcast_to(np.asarray(n0, np.float64), (n,))
    h0 = np.broadcast_to(np.asarray(h0, np.float64), (n,))
    out = np.zeros((n, MLP_IN))
    for i in range(n):
        f = np.zeros(MLP_IN)
        lib().ora_mlp_features(d, _p(_f64(J[i])), float(n0[i]), float(h0[i]), float(dx), _p(f))
        out[i] = f
    return out


def mlp_forward(params, F, FE=None):
    """c = g(f) for each row of F and the bound on a single-precision forward's deviation."""
    P = np.ascontiguousarray(params, dtype=np.float32)
    F = _f64(F).reshape(-1, MLP_IN)
    c = np.zeros(F.shape[0])
    b = np.zeros(F.shape[0])
    FE = None if FE is None else _f64(FE).reshape(-1, MLP_IN)
    lib().ora_mlp_forward_batch(_p(P), F.shape[0], _p(F), _p(FE) if FE is not None else None, _p(c), _p(b))
    return c, b


def mlp_backward(params, f, dLdc: float) -> np.ndarray:
    P = np.ascontiguousarray(params, dtype=np.float32)
    g = np.zeros(mlp_nparam())
    lib().ora_mlp_backward(_p(P), _p(_f64(f)), float(dLdc), _p(g))
    return g


def learn_loss_grad(D: _Dep, x, J, acc, status, batch, n0, h0, cells, target, with_grad=True):
    """Training loss of the learned correction at the listed cells and its gradient."""
    d = D.dim
    x, J, acc = _f64(x).reshape(-1, d), _f64(J).reshape(-1, d * d), _f64(acc).reshape(-1, 1 + d)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    target = _f64(target).reshape(-1, 1 + d)
    loss = np.zeros(1)
    grad = np.zeros(mlp_nparam()) if with_grad else None
    rc = lib().ora_learn_loss_grad(C.byref(D), x.shape[0], _p(x), _p(J), _p(acc), _p(_i32(status)), _p(_i32(batch)),
                                   _p(_f64(n0)), _p(_f64(h0)), cells.shape[0], _p(cells), _p(target), _p(loss),
                                   _p(grad) if grad is not None else None)
    assert rc == 0
    return float(loss[0]), grad


def learn_records(D: _Dep, x, J, acc, batch, n0, h0):
    """Per droplet: the network output c, whether h moves with c, and h."""
    d = D.dim
    x, J, acc = _f64(x).reshape(-1, d), _f64(J).reshape(-1, d * d), _f64(acc).reshape(-1, 1 + d)
    n = x.shape[0]
    c, act, h = np.zeros(n), np.zeros(n, np.int32), np.zeros(n)
    lib().ora_learn_records(C.byref(D), n, _p(x), _p(J), _p(acc), _p(_i32(batch)), _p(_f64(n0)), _p(_f64(h0)),
                            _p(c), _p(act), _p(h))
    return c, act.astype(bool), h
