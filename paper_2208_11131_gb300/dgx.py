"""ctypes binding of the C ABI in include/dgx.h (libdgx.so, built in-tree for sm_103a).

Argument marshalling only: every step of the hot path runs in the CUDA kernels
of libdgx.so.  There is no CPU fallback: if the library is missing or cannot
be loaded, ``lib()`` raises.

Functions keep the C names (``dg_create``, ``dg_set_state``, ``dg_rhs``,
``dg_step``, ``dg_get_state``, ``dg_max_dt`` ...).  ``Simulation`` is a small
convenience wrapper around one handle.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgx.so")

DG_OK, DG_EINVAL, DG_ENOMEM, DG_ECUDA, DG_ENONPHYS, DG_ETIMEOUT, DG_EUNSUPPORTED = range(7)
DG_BC_PERIODIC, DG_BC_OUTFLOW = 0, 1
DG_FP64, DG_FP32_BULK = 0, 1

# every entry point declared in include/dgx.h
EXPORTS = (
    "dg_default_params", "dg_create", "dg_destroy", "dg_set_params", "dg_get_params", "dg_sizes",
    "dg_set_stream", "dg_set_state", "dg_get_state", "dg_set_state_device", "dg_get_state_device",
    "dg_rhs", "dg_rhs_device", "dg_step", "dg_steps", "dg_step_timed", "dg_sync", "dg_max_dt", "dg_conserved_sums",
    "dg_get_aux", "dg_set_aux", "dg_last_error", "dg_status_string", "dg_max_dt_noalloc",
    "dg_batch_create", "dg_batch_step", "dg_batch_sync", "dg_batch_last_error", "dg_batch_destroy",
    "dg_get_forcing", "dg_set_forcing",
)


class dg_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("bc", ctypes.c_int * 3)]


class dg_params(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("rk_stages", ctypes.c_int), ("cfl", ctypes.c_double),
                ("av_on", ctypes.c_int), ("av_scale", ctypes.c_double), ("f_v", ctypes.c_double),
                ("f_tau", ctypes.c_double), ("f_w", ctypes.c_double), ("s_onset", ctypes.c_double),
                ("positivity_on", ctypes.c_int), ("forcing_on", ctypes.c_int), ("force_amp", ctypes.c_double),
                ("force_ts", ctypes.c_double), ("force_dt", ctypes.c_double), ("force_seed", ctypes.c_ulonglong),
                ("tracer_on", ctypes.c_int), ("tracer_eta", ctypes.c_double), ("basis", ctypes.c_int)]

DG_BASIS_TENSOR = 0
DG_BASIS_TOTAL = 1

FORCING_STATE = 97  # DG_FORCING_STATE


class DGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


_lib = None


def lib(path: str = LIB_PATH):
    """Load libdgx.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2208_11131_gb300.build.build()")
    L = ctypes.CDLL(path)
    H = ctypes.c_void_p
    P = ctypes.POINTER(ctypes.c_double)
    I = ctypes.c_int
    sig = {
        "dg_default_params": (I, [ctypes.POINTER(dg_params)]),
        "dg_create": (I, [ctypes.POINTER(dg_grid), I, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                          ctypes.POINTER(H)]),
        "dg_destroy": (None, [H]),
        "dg_set_params": (I, [H, ctypes.POINTER(dg_params)]),
        "dg_get_params": (I, [H, ctypes.POINTER(dg_params)]),
        "dg_sizes": (I, [H, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(ctypes.c_longlong)]),
        "dg_set_stream": (I, [H, ctypes.c_void_p]),
        "dg_set_state": (I, [H, P]), "dg_get_state": (I, [H, P]),
        "dg_set_state_device": (I, [H, ctypes.c_void_p]), "dg_get_state_device": (I, [H, ctypes.c_void_p]),
        "dg_rhs": (I, [H, P]), "dg_rhs_device": (I, [H, ctypes.c_void_p]),
        "dg_step": (I, [H, ctypes.c_double]), "dg_steps": (I, [H, I, ctypes.c_double]),
        "dg_step_timed": (I, [H, ctypes.c_double, ctypes.POINTER(ctypes.c_float), I]),
        "dg_sync": (I, [H]), "dg_max_dt": (I, [H, P]), "dg_conserved_sums": (I, [H, P]),
        "dg_get_aux": (I, [H, P, P, P]), "dg_set_aux": (I, [H, P, P, P]),
        "dg_last_error": (ctypes.c_char_p, [H]), "dg_status_string": (ctypes.c_char_p, [I]),
        "dg_batch_create": (I, [ctypes.POINTER(H), I, ctypes.POINTER(H)]),
        "dg_batch_step": (I, [H, I, ctypes.c_double]), "dg_batch_sync": (I, [H]),
        "dg_batch_last_error": (ctypes.c_char_p, [H]), "dg_batch_destroy": (None, [H]),
        "dg_max_dt_noalloc": (I, [ctypes.POINTER(dg_grid), I, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p]),
        "dg_get_forcing": (I, [H, P]), "dg_set_forcing": (I, [H, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(h, code):
    if code != DG_OK:
        msg = lib().dg_last_error(h).decode() if h else lib().dg_status_string(code).decode()
        raise DGError(code, msg or lib().dg_status_string(code).decode())


# ---------------------------------------------------------------- C-named wrappers

def dg_default_params() -> dg_params:
    p = dg_params()
    lib().dg_default_params(ctypes.byref(p))
    return p


def dg_create(grid: dg_grid, degree: int, gamma: float, nu: float, kappa: float):
    h = ctypes.c_void_p()
    code = lib().dg_create(ctypes.byref(grid), int(degree), float(gamma), float(nu), float(kappa), ctypes.byref(h))
    _check(None, code)
    return h


def dg_destroy(h):
    lib().dg_destroy(h)


def dg_set_params(h, p: dg_params):
    _check(h, lib().dg_set_params(h, ctypes.byref(p)))


def dg_get_params(h) -> dg_params:
    p = dg_params()
    _check(h, lib().dg_get_params(h, ctypes.byref(p)))
    return p


def dg_sizes(h):
    nf, nm, nc = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    _check(h, lib().dg_sizes(h, ctypes.byref(nf), ctypes.byref(nm), ctypes.byref(nc)))
    return nf.value, nm.value, nc.value


def dg_set_stream(h, stream_ptr: int):
    _check(h, lib().dg_set_stream(h, ctypes.c_void_p(stream_ptr)))


def dg_set_state(h, w: np.ndarray):
    _check(h, lib().dg_set_state(h, _dp(w)))


def dg_get_state(h, out: np.ndarray):
    _check(h, lib().dg_get_state(h, _dp(out)))


def dg_set_state_device(h, dev_ptr: int):
    _check(h, lib().dg_set_state_device(h, ctypes.c_void_p(dev_ptr)))


def dg_get_state_device(h, dev_ptr: int):
    _check(h, lib().dg_get_state_device(h, ctypes.c_void_p(dev_ptr)))


def dg_rhs(h, out: np.ndarray):
    _check(h, lib().dg_rhs(h, _dp(out)))


def dg_rhs_device(h, dev_ptr: int):
    _check(h, lib().dg_rhs_device(h, ctypes.c_void_p(dev_ptr)))


def dg_step(h, dt: float = 0.0):
    _check(h, lib().dg_step(h, float(dt)))


def dg_steps(h, nsteps: int, dt: float = 0.0):
    _check(h, lib().dg_steps(h, int(nsteps), float(dt)))


def dg_step_timed(h, dt: float = 0.0, nlaunch: int = 7):
    ms = (ctypes.c_float * 7)()
    _check(h, lib().dg_step_timed(h, float(dt), ms, 7))
    return list(ms)[:nlaunch]


def dg_sync(h):
    _check(h, lib().dg_sync(h))


def dg_max_dt(h) -> float:
    d = ctypes.c_double()
    _check(h, lib().dg_max_dt(h, ctypes.byref(d)))
    return d.value


def dg_conserved_sums(h, nc: int) -> np.ndarray:
    out = np.zeros(nc)
    _check(h, lib().dg_conserved_sums(h, _dp(out)))
    return out


def dg_get_aux(h, ncell: int):
    S = np.zeros(ncell)
    wig = np.zeros(ncell)
    scal = np.zeros(3)
    _check(h, lib().dg_get_aux(h, _dp(S), _dp(wig), _dp(scal)))
    return S, wig, scal


def dg_set_aux(h, S_prev=None, wig=None, scal=None):
    cv = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
    S_prev, wig, scal = cv(S_prev), cv(wig), cv(scal)
    _check(h, lib().dg_set_aux(h, _dp(S_prev), _dp(wig), _dp(scal)))


def dg_get_forcing(h) -> np.ndarray:
    out = np.zeros(FORCING_STATE)
    _check(h, lib().dg_get_forcing(h, _dp(out)))
    return out


def dg_set_forcing(h, state):
    state = np.ascontiguousarray(state, dtype=np.float64)
    assert state.shape == (FORCING_STATE,)
    _check(h, lib().dg_set_forcing(h, _dp(state)))


def dg_max_dt_noalloc(grid: dg_grid, degree: int, gamma: float, cfl: float, dev_state_ptr: int, dev_dt_ptr: int,
                      stream_ptr: int = 0):
    """CFL step into a caller-owned device double; allocates nothing (see include/dgx.h)."""
    code = lib().dg_max_dt_noalloc(ctypes.byref(grid), int(degree), float(gamma), float(cfl),
                                   ctypes.c_void_p(dev_state_ptr), ctypes.c_void_p(dev_dt_ptr),
                                   ctypes.c_void_p(stream_ptr))
    _check(None, code)


def _bcheck(b, code):
    if code != DG_OK:
        msg = lib().dg_batch_last_error(b).decode() if b else lib().dg_status_string(code).decode()
        raise DGError(code, msg or lib().dg_status_string(code).decode())


def dg_batch_create(handles):
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    b = ctypes.c_void_p()
    _bcheck(None, lib().dg_batch_create(arr, len(handles), ctypes.byref(b)))
    return b


def dg_batch_step(b, nsteps: int, dt: float = 0.0):
    _bcheck(b, lib().dg_batch_step(b, int(nsteps), float(dt)))


def dg_batch_sync(b):
    _bcheck(b, lib().dg_batch_sync(b))


def dg_batch_destroy(b):
    lib().dg_batch_destroy(b)


# ---------------------------------------------------------------- convenience wrapper

def make_grid(dim, N, lo, hi, bc=(0, 0, 0)) -> dg_grid:
    g = dg_grid()
    g.dim = dim
    for a in range(3):
        g.n[a] = int(N[a]) if a < len(N) else 1
        g.lo[a] = float(lo[a]) if a < len(lo) else 0.0
        g.hi[a] = float(hi[a]) if a < len(hi) else 1.0
        g.bc[a] = int(bc[a]) if a < len(bc) else 0
    return g


class Simulation:
    """One simulation handle built from an ``inputs.Workload``-like description."""

    def __init__(self, wl, precision: int = DG_FP64, rk_stages: int = 0, cfl: float | None = None):
        self.wl = wl
        grid = make_grid(wl.dim, wl.N[: wl.dim], wl.lo[: wl.dim], wl.hi[: wl.dim], wl.bc[: wl.dim])
        self.h = dg_create(grid, wl.n, wl.gamma, wl.nu, wl.kappa)
        p = dg_default_params()
        p.precision = precision
        p.rk_stages = rk_stages
        p.cfl = wl.cfl if cfl is None else cfl
        p.av_on = int(wl.av_on)
        p.positivity_on = int(getattr(wl, "positivity_on", 0))
        p.basis = int(getattr(wl, "basis", 0))
        if getattr(wl, "tracer_on", 0):
            p.tracer_on = 1
            p.tracer_eta = float(wl.eta)
        if getattr(wl, "forcing_on", 0):
            p.forcing_on = 1
            p.force_amp, p.force_ts, p.force_dt = wl.force_amp, wl.force_ts, wl.force_dt
            p.force_seed = int(wl.force_seed) & 0xFFFFFFFFFFFFFFFF
        dg_set_params(self.h, p)
        self.nf, self.M, self.ncell = dg_sizes(self.h)
        self.nc = wl.dim + 2 + (1 if getattr(wl, "tracer_on", 0) else 0)

    def close(self):
        if self.h:
            dg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.nf, self.ncell, self.M)

    def set_stream(self, stream_ptr: int):
        dg_set_stream(self.h, stream_ptr)

    def set_state(self, w: np.ndarray):
        w = np.ascontiguousarray(w, dtype=np.float64)
        assert w.shape == self.shape, (w.shape, self.shape)
        dg_set_state(self.h, w)

    def get_state(self) -> np.ndarray:
        out = np.empty(self.shape)
        dg_get_state(self.h, out)
        return out

    def rhs(self) -> np.ndarray:
        out = np.empty(self.shape)
        dg_rhs(self.h, out)
        return out

    def step(self, dt: float = 0.0):
        dg_step(self.h, dt)

    def steps(self, n: int, dt: float = 0.0):
        dg_steps(self.h, n, dt)

    def sync(self):
        dg_sync(self.h)

    def max_dt(self) -> float:
        return dg_max_dt(self.h)

    def conserved_sums(self) -> np.ndarray:
        return dg_conserved_sums(self.h, self.nc)

    def get_forcing(self) -> np.ndarray:
        return dg_get_forcing(self.h)

    def set_forcing(self, state):
        dg_set_forcing(self.h, state)

    def get_aux(self):
        return dg_get_aux(self.h, self.ncell)

    def set_aux(self, S_prev=None, wig=None, scal=None):
        dg_set_aux(self.h, S_prev, wig, scal)
