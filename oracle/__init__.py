"""FP64 CPU oracle of the modal DG hot path of arXiv 2208.11131.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code,
table or constant with the CUDA path in ``paper_2208_11131_gb300``.

The arithmetic lives in ``dg_oracle.c`` (plain C, FP64, direct modal sums,
compiled with ``-ffp-contract=off``); this module only marshals arguments and
adds the small host-side pieces the tests need:

* ``project``    -- initial projection w_l = (1/|K|) int u phi_l  (Eq. weights_equation),
                    with an elevated n+3 point Gauss rule (Sec. 5.1, Sec. 6);
* ``l1_error``   -- the L1 norm of Eq. l1_norm with an n+2 point rule (Sec. 5.1);
* thin wrappers of every C entry point.

The state layout is ``[field][cell][mode]`` with cells x-fastest and the mode
index l = l_x + (n+1)(l_y + (n+1) l_z); fields are (rho, rho v_x, rho v_y,
[rho v_z], e) followed by the artificial-viscosity field alpha when it is on.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK = 0
EINVAL = 1
ENONPHYS = 4


def build(force: bool = False) -> str:
    """Compile dg_oracle.c into liboracle.so (gcc, -O2 -ffp-contract=off -fopenmp)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Cfg(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int), ("N", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("bc", ctypes.c_int * 3),
        ("gamma", ctypes.c_double), ("nu", ctypes.c_double), ("kappa", ctypes.c_double),
        ("av_on", ctypes.c_int), ("av_scale", ctypes.c_double), ("f_v", ctypes.c_double),
        ("f_tau", ctypes.c_double), ("f_w", ctypes.c_double), ("s_onset", ctypes.c_double),
        ("positivity_on", ctypes.c_int), ("cfl", ctypes.c_double), ("rk_stages", ctypes.c_int),
        ("forcing_on", ctypes.c_int), ("force_amp", ctypes.c_double), ("force_ts", ctypes.c_double),
        ("force_dt", ctypes.c_double), ("force_seed", ctypes.c_ulonglong),
        ("tracer_on", ctypes.c_int), ("eta", ctypes.c_double), ("basis", ctypes.c_int),
        ("s_floor", ctypes.c_double),
    ]

FMODES = 16  # forcing-state mode stride
FSTATE = 1 + 6 * FMODES


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D = ctypes.c_double
        P = ctypes.POINTER(ctypes.c_double)
        I = ctypes.c_int
        C = ctypes.POINTER(Cfg)
        sig = {
            "or_pt": (D, [I, D]), "or_dpt": (D, [I, D]), "or_gauss": (I, [I, P, P]),
            "or_recovery_matrices": (I, [I, D, P, P]), "or_overlap_fraction": (D, [I]),
            "or_hllc": (I, [I, I, D, P, P, P]), "or_ns_flux": (I, [I, I, D, D, D, P, P, P]),
            "or_rhs": (I, [C, P, P, P]), "or_max_speeds": (I, [C, P, P, P]), "or_max_dt": (I, [C, P, P]),
            "or_sensor": (I, [C, P, P]), "or_wiggle": (I, [C, P, P, P, D, ctypes.c_long]),
            "or_positivity": (I, [C, P]), "or_rk_stages": (I, [I]), "or_rk_table": (I, [I, P, P]),
            "or_step": (I, [C, P, P, P, P, D, P]), "or_basis_eval": (I, [I, I, I, P, P]),
            "or_num_threads": (I, []), "or_set_num_threads": (None, [I]),
            "or_face_recovery": (I, [C, P, ctypes.c_long, ctypes.c_long, I, P, P]),
            "or_rhs_forced": (I, [C, P, P, P, P]), "or_step_forced": (I, [C, P, P, P, P, P, D, P]),
            "or_forcing_modes": (I, [I, ctypes.POINTER(ctypes.c_int)]),
            "or_forcing_uniform": (D, [ctypes.c_ulonglong, ctypes.c_ulonglong]),
            "or_forcing_normal": (D, [ctypes.c_ulonglong, ctypes.c_ulonglong]),
            "or_forcing_update": (I, [C, P, D]), "or_forcing_eval": (I, [C, P, I, P, P]),
            "or_hllc_tracer": (I, [I, I, D, P, P, P]),
            "or_num_modes": (I, [I, I, I]), "or_basis_eval_b": (I, [I, I, I, I, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------- basics

def pt(l: int, x: float) -> float:
    """Scaled Legendre polynomial sqrt(2l+1) P_l(x)."""
    return lib().or_pt(l, x)


def dpt(l: int, x: float) -> float:
    return lib().or_dpt(l, x)


def gauss(q: int):
    x = np.zeros(q)
    w = np.zeros(q)
    if lib().or_gauss(q, _p(x), _p(w)) != OK:
        raise ValueError(q)
    return x, w


def recovery_matrices(n: int, f: float | None = None):
    if f is None:
        f = lib().or_overlap_fraction(n)
    Am = np.zeros((n + 1) * (n + 2))
    Ap = np.zeros((n + 1) * (n + 2))
    lib().or_recovery_matrices(n, f, _p(Am), _p(Ap))
    return Am.reshape(n + 1, n + 2), Ap.reshape(n + 1, n + 2), f


def hllc(dim: int, axis: int, gamma: float, uL, uR):
    """HLLC flux of the Euler fields; with d+3 components the last is a passive tracer rho c"""
    uL = np.ascontiguousarray(uL, dtype=np.float64)
    uR = np.ascontiguousarray(uR, dtype=np.float64)
    tr = uL.size == dim + 3
    F = np.zeros(dim + 2 + tr)
    fn = lib().or_hllc_tracer if tr else lib().or_hllc
    st = fn(dim, axis, gamma, _p(uL), _p(uR), _p(F))
    return F, st


def ns_flux(dim: int, axis: int, gamma: float, nu: float, kappa: float, u, grad):
    u = np.ascontiguousarray(u, dtype=np.float64)
    grad = np.ascontiguousarray(grad, dtype=np.float64).reshape(dim, dim + 2)
    F = np.zeros(dim + 2)
    st = lib().or_ns_flux(dim, axis, gamma, nu, kappa, _p(u), _p(grad), _p(F))
    return F, st


def rk_table(stages: int):
    a = np.zeros(36)
    b = np.zeros(36)
    if lib().or_rk_table(stages, _p(a), _p(b)) != OK:
        raise ValueError(stages)
    return a.reshape(6, 6), b.reshape(6, 6)


def rk_stages(n: int) -> int:
    return lib().or_rk_stages(n)


def basis_eval(dim: int, n: int, xi: np.ndarray, basis: int = 0) -> np.ndarray:
    """phi_l at reference points xi [npts, dim] -> [npts, M]; basis 1: the total-degree modes"""
    xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(-1, dim)
    M = lib().or_num_modes(dim, n, basis)
    out = np.zeros((xi.shape[0], M))
    lib().or_basis_eval_b(dim, n, basis, xi.shape[0], _p(xi), _p(out))
    return out


def set_threads(t: int) -> None:
    lib().or_set_num_threads(int(t))


def num_threads() -> int:
    return lib().or_num_threads()


# ---------------------------------------------------------------- problem description

@dataclass
class Problem:
    """Grid, degree, gas and dissipation parameters of one simulation."""
    dim: int
    n: int
    N: tuple
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    bc: tuple = (0, 0, 0)
    gamma: float = 5.0 / 3.0
    nu: float = 0.0
    kappa: float = 0.0
    av_on: int = 0
    av_scale: float = 1.0
    f_v: float = 2.5
    f_tau: float = 0.5
    f_w: float = 0.2
    s_onset: float = 1e-4
    positivity_on: int = 0
    cfl: float = 0.5
    rk_stages: int = 0
    forcing_on: int = 0
    force_amp: float = 0.0
    force_ts: float = 1.0
    force_dt: float = 0.01
    force_seed: int = 0
    tracer_on: int = 0
    eta: float = 0.0
    basis: int = 0  # 0 tensor product, 1 total degree l_x + l_y + l_z <= n (Sec. 2.3)
    # floor of the oscillation sensor in the wiggle source, as a fraction of the onset threshold
    # s_onset/P^2 (the reading of Sec. 4.1's d log S/dt; a parameter only so that tests can show
    # what the floor does)
    s_floor: float = 1e-4

    def cfg(self) -> Cfg:
        c = Cfg()
        c.dim, c.n = self.dim, self.n
        N = list(self.N) + [1] * (3 - len(self.N))
        lo = list(self.lo) + [0.0] * (3 - len(self.lo))
        hi = list(self.hi) + [1.0] * (3 - len(self.hi))
        bc = list(self.bc) + [0] * (3 - len(self.bc))
        for a in range(3):
            c.N[a], c.lo[a], c.hi[a], c.bc[a] = int(N[a]), float(lo[a]), float(hi[a]), int(bc[a])
        c.gamma, c.nu, c.kappa = self.gamma, self.nu, self.kappa
        c.av_on, c.av_scale, c.f_v, c.f_tau, c.f_w, c.s_onset = (int(self.av_on), self.av_scale, self.f_v,
                                                                self.f_tau, self.f_w, self.s_onset)
        c.positivity_on, c.cfl, c.rk_stages = int(self.positivity_on), self.cfl, int(self.rk_stages)
        c.forcing_on, c.force_amp, c.force_ts, c.force_dt = (int(self.forcing_on), self.force_amp, self.force_ts,
                                                             self.force_dt)
        c.force_seed = int(self.force_seed) & 0xFFFFFFFFFFFFFFFF
        c.tracer_on, c.eta = int(self.tracer_on), float(self.eta)
        c.basis = int(self.basis)
        c.s_floor = float(self.s_floor)
        return c

    @property
    def ncell(self) -> int:
        return int(np.prod(self.N[: self.dim]))

    @property
    def M(self) -> int:
        return lib().or_num_modes(self.dim, self.n, int(self.basis))

    @property
    def nfields(self) -> int:
        return self.dim + 2 + (1 if self.tracer_on else 0) + (1 if self.av_on else 0)

    @property
    def h(self):
        return [(self.hi[a] - self.lo[a]) / self.N[a] for a in range(self.dim)]

    def shape(self):
        return (self.nfields, self.ncell, self.M)

    def cell_centres(self) -> np.ndarray:
        """[ncell, dim] cell centres, x fastest."""
        axes = [self.lo[a] + (np.arange(self.N[a]) + 0.5) * self.h[a] for a in range(self.dim)]
        grids = np.meshgrid(*axes[::-1], indexing="ij")  # slowest axis first
        return np.stack([g.reshape(-1) for g in grids[::-1]], axis=1)


def _ref_points(dim: int, q: int):
    x, w = gauss(q)
    grids = np.meshgrid(*([x] * dim)[::-1], indexing="ij")
    xi = np.stack([g.reshape(-1) for g in grids[::-1]], axis=1)  # axis 0 fastest
    wg = np.meshgrid(*([w] * dim)[::-1], indexing="ij")
    G = np.prod(np.stack([g.reshape(-1) for g in wg], axis=1), axis=1)
    return xi, G


def project(prob: Problem, func, q: int | None = None) -> np.ndarray:
    """w_l = (1/|K|) int_K u phi_l dV with a q-point Gauss rule (default n+3).

    ``func(X)`` receives points [npts, dim] and returns the fields [nf, npts].
    """
    q = prob.n + 3 if q is None else q
    xi, G = _ref_points(prob.dim, q)
    phi = basis_eval(prob.dim, prob.n, xi, prob.basis)  # [nq, M]
    xc = prob.cell_centres()
    h = np.array(prob.h)
    X = xc[:, None, :] + 0.5 * h[None, None, :] * xi[None, :, :]  # [ncell, nq, dim]
    U = np.asarray(func(X.reshape(-1, prob.dim)), dtype=np.float64)
    U = U.reshape(U.shape[0], prob.ncell, xi.shape[0])
    w = np.einsum("fkj,j,jl->fkl", U, G, phi) / 2.0 ** prob.dim
    return np.ascontiguousarray(w)


def evaluate(prob: Problem, w: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """values of every field at reference points xi [npts, dim] of every cell -> [nf, ncell, npts]."""
    phi = basis_eval(prob.dim, prob.n, xi, prob.basis)
    return np.einsum("fkl,jl->fkj", w, phi)


def l1_error(prob: Problem, w: np.ndarray, func, field: int = 0, q: int | None = None) -> float:
    """Domain-averaged L1 norm of Eq. l1_norm for one field, n+2 point Gauss rule."""
    q = prob.n + 2 if q is None else q
    xi, G = _ref_points(prob.dim, q)
    xc = prob.cell_centres()
    h = np.array(prob.h)
    X = xc[:, None, :] + 0.5 * h[None, None, :] * xi[None, :, :]
    U = np.asarray(func(X.reshape(-1, prob.dim)), dtype=np.float64)
    U = U.reshape(U.shape[0], prob.ncell, xi.shape[0])[field]
    Uh = evaluate(prob, w[field:field + 1], xi)[0]
    return float(np.sum(np.abs(U - Uh) * G[None, :]) / (2.0 ** prob.dim) / prob.ncell)


# ---------------------------------------------------------------- operator calls

def rhs(prob: Problem, w: np.ndarray, wig: np.ndarray | None = None, fst: np.ndarray | None = None):
    """dw/dt; with forcing on, ``fst`` is the forcing state whose driving field is added."""
    c = prob.cfg()
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros_like(w)
    wp = _p(np.ascontiguousarray(wig, dtype=np.float64)) if wig is not None else None
    fp = _p(np.ascontiguousarray(fst, dtype=np.float64)) if fst is not None else None
    st = lib().or_rhs_forced(ctypes.byref(c), _p(w), wp, fp, _p(out))
    return out, st


# ---------------------------------------------------------------- turbulence driving (Sec. 7.1)

def forcing_modes(dim: int) -> np.ndarray:
    """[nmodes, 3] integer wave vectors of the driving (one of every +-k pair)."""
    k = (ctypes.c_int * (3 * FMODES))()
    n = lib().or_forcing_modes(dim, k)
    return np.array(k[: 3 * n], dtype=int).reshape(n, 3)


def forcing_uniform(seed: int, i: int) -> float:
    return lib().or_forcing_uniform(seed & 0xFFFFFFFFFFFFFFFF, i)


def forcing_normal(seed: int, c: int) -> float:
    return lib().or_forcing_normal(seed & 0xFFFFFFFFFFFFFFFF, c)


def forcing_state() -> np.ndarray:
    """a fresh forcing state: no update applied yet"""
    f = np.zeros(FSTATE)
    f[0] = -1.0
    return f


def forcing_update(prob: Problem, fst: np.ndarray, t: float) -> int:
    """in place: apply every OU update due at time t"""
    c = prob.cfg()
    return lib().or_forcing_update(ctypes.byref(c), _p(fst), float(t))


def forcing_eval(prob: Problem, fst: np.ndarray, X: np.ndarray) -> np.ndarray:
    """driving acceleration at physical points X [npts, dim] -> [npts, 3]"""
    c = prob.cfg()
    X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.zeros((X.shape[0], 3))
    st = lib().or_forcing_eval(ctypes.byref(c), _p(np.ascontiguousarray(fst)), X.shape[0], _p(X), _p(out))
    if st != OK:
        raise ValueError(st)
    return out


def face_recovery(prob: Problem, w: np.ndarray, KL: int, KR: int, axis: int):
    """recovered state [NQF, nf] and physical gradient [NQF, 3, nf] on the face between cells KL | KR."""
    c = prob.cfg()
    nqf = (prob.n + 1) ** (prob.dim - 1)
    nf = prob.dim + 2
    ut = np.zeros((nqf, nf))
    gt = np.zeros((nqf, 3, nf))
    st = lib().or_face_recovery(ctypes.byref(c), _p(np.ascontiguousarray(w)), KL, KR, axis, _p(ut), _p(gt))
    if st != OK:
        raise ValueError(st)
    return ut, gt


def max_speeds(prob: Problem, w: np.ndarray):
    c = prob.cfg()
    cm = ctypes.c_double()
    vm = ctypes.c_double()
    st = lib().or_max_speeds(ctypes.byref(c), _p(np.ascontiguousarray(w)), ctypes.byref(cm), ctypes.byref(vm))
    return cm.value, vm.value, st


def max_dt(prob: Problem, w: np.ndarray):
    c = prob.cfg()
    dt = ctypes.c_double()
    st = lib().or_max_dt(ctypes.byref(c), _p(np.ascontiguousarray(w)), ctypes.byref(dt))
    return dt.value, st


def sensor(prob: Problem, w: np.ndarray) -> np.ndarray:
    c = prob.cfg()
    S = np.zeros(prob.ncell)
    lib().or_sensor(ctypes.byref(c), _p(np.ascontiguousarray(w)), _p(S))
    return S


def positivity(prob: Problem, w: np.ndarray) -> int:
    """in place"""
    c = prob.cfg()
    return lib().or_positivity(ctypes.byref(c), _p(w))


@dataclass
class Sim:
    """Oracle simulation: state + the per-cell and scalar auxiliary data of a step."""
    prob: Problem
    w: np.ndarray
    S_prev: np.ndarray = None
    wig: np.ndarray = None
    scal: np.ndarray = field(default_factory=lambda: np.zeros(3))  # dt_prev, step, t
    fst: np.ndarray = None  # forcing state (Sec. 7.1 driving)

    def __post_init__(self):
        self.w = np.ascontiguousarray(self.w, dtype=np.float64).copy()
        if self.fst is None:
            self.fst = forcing_state()
        if self.S_prev is None:
            self.S_prev = np.zeros(self.prob.ncell)
        if self.wig is None:
            self.wig = np.zeros(self.prob.ncell)

    def step(self, dt: float = 0.0):
        c = self.prob.cfg()
        used = ctypes.c_double()
        st = lib().or_step_forced(ctypes.byref(c), _p(self.w), _p(self.S_prev), _p(self.wig), _p(self.scal),
                                  _p(self.fst), float(dt), ctypes.byref(used))
        return used.value, st

    @property
    def t(self) -> float:
        return float(self.scal[2])
