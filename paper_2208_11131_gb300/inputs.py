"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the one piece shared by the CUDA path's callers (tests,
``bench.py``) and by the oracle's tests.  It holds none of the right-hand-side,
time-step or limiter arithmetic.  It only

* describes a workload (grid, degree, gas, dissipation switches, step count),
* draws seeded random numbers, and
* projects analytic initial conditions onto the cell-local scaled-Legendre
  basis (Eq. weights_equation, w_l = (1/|K|) int_K u phi_l dV) with an n+3 point
  Gauss rule taken from ``numpy.polynomial.legendre`` (Sec. 5.1 and Sec. 6 use
  an elevated rule for the projection).

State layout: float64 ``[field][cell][mode]``, cells x-fastest, mode index
l = l_x + (n+1)(l_y + (n+1) l_z), fields (rho, rho v_x, rho v_y, [rho v_z], e)
and then the artificial-viscosity field alpha when ``av_on``.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np
from numpy.polynomial import legendre as npleg

BASE_SEED = 20220823


@dataclass(frozen=True)
class Workload:
    name: str
    dim: int
    n: int
    N: tuple
    lo: tuple
    hi: tuple
    bc: tuple = (0, 0, 0)  # 0 periodic, 1 outflow
    gamma: float = 5.0 / 3.0
    nu: float = 0.0
    kappa: float = 0.0
    av_on: int = 0
    positivity_on: int = 0
    cfl: float = 0.5
    steps: int = 1
    # turbulence driving (Sec. 7.1): amplitude of the |k| = 1 modes, OU correlation time, update
    # interval, generator seed
    forcing_on: int = 0
    force_amp: float = 0.0
    force_ts: float = 1.0
    force_dt: float = 0.01
    force_seed: int = 0
    # passive tracer (Sec. 3.4): conserved field rho c after the energy, diffusivity eta
    tracer_on: int = 0
    eta: float = 0.0
    basis: int = 0  # 0 tensor product, 1 total degree l_x + l_y + l_z <= n (Sec. 2.3)

    @property
    def ncell(self) -> int:
        return int(np.prod(self.N[: self.dim]))

    @property
    def M(self) -> int:
        return len(mode_exponents(self.dim, self.n, self.basis))

    @property
    def nfields(self) -> int:
        return self.ncons + (1 if self.av_on else 0)

    @property
    def ncons(self) -> int:
        return self.dim + 2 + (1 if self.tracer_on else 0)

    @property
    def dofs(self) -> int:
        """conserved degrees of freedom: cells x modes x (d+2)"""
        return self.ncell * self.M * self.ncons

    @property
    def h(self):
        return [(self.hi[a] - self.lo[a]) / self.N[a] for a in range(self.dim)]

    def shape(self):
        return (self.nfields, self.ncell, self.M)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def mode_exponents(dim: int, n: int, basis: int = 0) -> np.ndarray:
    """[M, dim] Legendre degrees of the modes in state order: tensor order with x fastest, all l_a <= n
    (basis 0) or only l_x + l_y + l_z <= n (basis 1, the paper's total-degree truncation)"""
    grids = np.meshgrid(*([np.arange(n + 1)] * dim)[::-1], indexing="ij")
    e = np.stack([g.reshape(-1) for g in grids[::-1]], axis=1)
    return e[e.sum(1) <= n] if basis == 1 else e


# ------------------------------------------------------------------ the five paper-shaped workloads

def isentropic_vortex(N: int = 32, n: int = 3) -> Workload:
    """2-D Euler isentropic vortex of Sec. 5.1: periodic [-5,5]^2, gamma=1.4, beta=5 (steady)."""
    return Workload("isentropic_vortex_2d", 2, n, (N, N, 1), (-5.0, -5.0, 0.0), (5.0, 5.0, 1.0), gamma=1.4,
                    cfl=0.3, steps=100)


def gaussian_pulse(N: int = 16, n: int = 2) -> Workload:
    """2-D diffusion of a Gaussian tracer pulse (Sec. 5.2): gas at rest (rho = p = 1, gamma = 1.4) on
    the periodic [-0.5,0.5]^2, tracer diffusivity eta = 1/128."""
    return Workload("gaussian_pulse_2d", 2, n, (N, N, 1), (-0.5, -0.5, 0.0), (0.5, 0.5, 1.0), gamma=1.4, cfl=0.3,
                    steps=100, tracer_on=1, eta=1.0 / 128.0)


def c1_density_wave(N: int = 32, n: int = 2) -> Workload:
    """2-D Euler, gamma=5/3, periodic [0,1]^2, rho = 1 + 0.2 sin 2pi(x+y), v=(1,1), P=1."""
    return Workload("density_wave_2d", 2, n, (N, N, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), gamma=5.0 / 3.0,
                    cfl=0.3, steps=20)


def c2_shear_layer(N: int = 256, n: int = 3) -> Workload:
    """2-D compressible Navier-Stokes shear layer, [0,1]x[0,2], NxN cells (h_y = 2 h_x), nu=kappa=1e-5, AV on."""
    return Workload("ns_shear_layer_2d", 2, n, (N, N, 1), (0.0, 0.0, 0.0), (1.0, 2.0, 1.0), gamma=5.0 / 3.0,
                    nu=1e-5, kappa=1e-5, av_on=1, cfl=0.5, steps=500)


def c3_sod_blast(N: int = 64, n: int = 3) -> Workload:
    """3-D rotated Sod plane + spherical blast, outflow boundaries, AV and positivity limiter on."""
    return Workload("sod_blast_3d", 3, n, (N, N, N), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), bc=(1, 1, 1), gamma=1.4,
                    av_on=1, positivity_on=1, cfl=0.3, steps=200)


def c4_turbulence_box(N: int = 128, n: int = 3) -> Workload:
    """3-D periodic subsonic turbulence box, gamma=1.001, nu=kappa=1e-4, AV on, driven (Sec. 7.1):
    modes 1 <= |k| <= 2, amplitude 0.03 |k|^(-5/3) (rms acceleration about 0.1, which brings the
    gas started at rest with c_s = 1 to Mach ~0.3 within a few time units), OU correlation time 1,
    update interval 0.01."""
    return Workload("turbulence_box_3d", 3, n, (N, N, N), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), gamma=1.001,
                    nu=1e-4, kappa=1e-4, av_on=1, cfl=0.5, steps=100, forcing_on=1, force_amp=0.03,
                    force_ts=1.0, force_dt=0.01, force_seed=BASE_SEED + 4)


# ------------------------------------------------------------------ projection (numpy Gauss rule)

def _pt_table(n: int, x: np.ndarray) -> np.ndarray:
    """[len(x), n+1] scaled Legendre values sqrt(2l+1) P_l(x) via numpy's Legendre series."""
    V = npleg.legvander(x, n)
    return V * np.sqrt(2.0 * np.arange(n + 1) + 1.0)[None, :]


def _cell_centres(wl: Workload) -> np.ndarray:
    axes = [wl.lo[a] + (np.arange(wl.N[a]) + 0.5) * wl.h[a] for a in range(wl.dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return np.stack([g.reshape(-1) for g in grids[::-1]], axis=1)


def project(wl: Workload, func, q: int | None = None, chunk: int = 1 << 15) -> np.ndarray:
    """Project ``func(X) -> [nfields, npts]`` onto the basis of every cell (x fastest)."""
    q = wl.n + 3 if q is None else q
    x, g = npleg.leggauss(q)
    B = _pt_table(wl.n, x)  # [q, n+1]
    d = wl.dim
    grids = np.meshgrid(*([x] * d)[::-1], indexing="ij")
    xi = np.stack([gg.reshape(-1) for gg in grids[::-1]], axis=1)  # [q^d, d], axis 0 fastest
    idx = np.stack([gg.reshape(-1) for gg in np.meshgrid(*([np.arange(q)] * d)[::-1], indexing="ij")[::-1]], 1)
    G = np.prod(g[idx], axis=1)
    midx = mode_exponents(d, wl.n, wl.basis)  # [M, d]
    phi = np.ones((xi.shape[0], wl.M))
    for a in range(d):
        phi *= B[idx[:, a]][:, midx[:, a]]
    xc = _cell_centres(wl)
    h = np.array(wl.h)
    out = np.empty(wl.shape())
    for c0 in range(0, wl.ncell, chunk):
        c1 = min(wl.ncell, c0 + chunk)
        X = xc[c0:c1, None, :] + 0.5 * h[None, None, :] * xi[None, :, :]
        U = np.asarray(func(X.reshape(-1, d)), dtype=np.float64).reshape(-1, c1 - c0, xi.shape[0])
        out[:, c0:c1, :] = np.einsum("fkj,j,jl->fkl", U, G, phi) / 2.0 ** d
    return np.ascontiguousarray(out)


def _cons(gamma, rho, vel, p, extra=None):
    e = p / (gamma - 1.0) + 0.5 * rho * sum(v * v for v in vel)
    fields = [rho] + [rho * v for v in vel] + [e]
    if extra is not None:
        fields.append(extra)
    return np.stack(fields)


# ------------------------------------------------------------------ initial conditions

def density_wave_ic(wl: Workload, t: float = 0.0):
    """exact solution of the advected density wave: rho(x - t, y - t), v=(1,1), P=1"""
    def f(X):
        x, y = X[:, 0], X[:, 1]
        rho = 1.0 + 0.2 * np.sin(2.0 * np.pi * (x + y - 2.0 * t))
        one = np.ones_like(x)
        return _cons(wl.gamma, rho, [one, one], one, np.zeros_like(x) if wl.av_on else None)
    return f


def isentropic_vortex_ic(wl: Workload, beta: float = 5.0):
    """the vortex of Sec. 5.1 (Yee's original set-up, background rho = p = 1) centred at the origin:
    v = beta/(2 pi) e^((1-r^2)/2) (-y, x), specific internal energy
    u = 1/(gamma-1) - beta^2/(8 gamma pi^2) e^(1-r^2), rho = ((gamma-1) u)^(1/(gamma-1)),
    p = (gamma-1) rho u; isentropic (p = rho^gamma) and in radial balance dp/dr = rho v^2/r, so it is
    also the exact solution at every time"""
    g = wl.gamma

    def f(X):
        x, y = X[:, 0], X[:, 1]
        r2 = x * x + y * y
        a = beta / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
        u = 1.0 / (g - 1.0) - beta * beta / (8.0 * g * np.pi ** 2) * np.exp(1.0 - r2)
        rho = ((g - 1.0) * u) ** (1.0 / (g - 1.0))
        p = (g - 1.0) * rho * u
        return _cons(g, rho, [-a * y, a * x], p, np.zeros_like(x) if wl.av_on else None)
    return f


def gaussian_pulse_ic(wl: Workload, t: float, c_b: float = 0.1, c_g: float = 1.0):
    """exact tracer field of Sec. 5.2 at time t: c = c_b + sum_j c_g/(2 pi s^2) exp(-|x-j|^2/(2 s^2)),
    s^2 = 2 eta t, summed over the periodic images j of the unit box; gas at rest, rho = p = 1"""
    s2 = 2.0 * wl.eta * t

    def f(X):
        x, y = X[:, 0], X[:, 1]
        c = np.full_like(x, c_b)
        for jx in range(-4, 5):
            for jy in range(-4, 5):
                c += c_g / (2.0 * np.pi * s2) * np.exp(-((x - jx) ** 2 + (y - jy) ** 2) / (2.0 * s2))
        one = np.ones_like(x)
        zero = np.zeros_like(x)
        fields = [one, zero, zero, one / (wl.gamma - 1.0), c]
        if wl.av_on:
            fields.append(zero)
        return np.stack(fields)
    return f


def shear_layer_ic(wl: Workload, seed: int = BASE_SEED):
    """smooth Kelvin-Helmholtz shear layer (Sec. 6 set-up): a=0.05, y1=0.5, y2=1.5, u_flow=1,
    density contrast 2 (Delta rho/rho0 = 1), A=0.01, sigma=0.2, P0=10, seeded phase of the perturbation."""
    rng = np.random.default_rng(seed)
    phase = float(rng.uniform(0.0, 2.0 * np.pi))
    a, y1, y2, A, sig, P0, drho = 0.05, 0.5, 1.5, 0.01, 0.2, 10.0, 1.0

    def f(X):
        x, y = X[:, 0], X[:, 1]
        th = np.tanh((y - y1) / a) - np.tanh((y - y2) / a)
        rho = 1.0 + drho * 0.5 * th
        vx = 1.0 * (th - 1.0)
        vy = A * np.sin(2.0 * np.pi * x + phase) * (np.exp(-((y - y1) ** 2) / sig**2) +
                                                    np.exp(-((y - y2) ** 2) / sig**2))
        p = P0 * np.ones_like(x)
        return _cons(wl.gamma, rho, [vx, vy], p, np.zeros_like(x) if wl.av_on else None)
    return f


def sod_blast_ic(wl: Workload, seed: int = BASE_SEED):
    """Sod states (1,1 | 0.125,0.1) across a plane through the box centre with a seeded unit normal,
    plus p=100 inside a sphere of radius 0.1 around a seeded centre in [0.25,0.75]^d."""
    rng = np.random.default_rng(seed + 3)
    nrm = rng.normal(size=wl.dim)
    nrm /= np.linalg.norm(nrm)
    ctr = rng.uniform(0.25, 0.75, size=wl.dim)

    def f(X):
        s = (X - 0.5) @ nrm
        left = s < 0.0
        rho = np.where(left, 1.0, 0.125)
        p = np.where(left, 1.0, 0.1)
        r2 = np.sum((X - ctr) ** 2, axis=1)
        p = np.where(r2 < 0.01, 100.0, p)
        zero = np.zeros_like(rho)
        return _cons(wl.gamma, rho, [zero] * wl.dim, p, zero if wl.av_on else None)
    return f


def rest_state(wl: Workload) -> np.ndarray:
    """modes of gas at rest with uniform density 1 and pressure 1/gamma (sound speed 1): the
    starting state of the driven-turbulence runs of Sec. 7"""
    w = np.zeros(wl.shape())
    w[0, :, 0] = 1.0
    w[wl.dim + 1, :, 0] = 1.0 / (wl.gamma * (wl.gamma - 1.0))
    return w


def turbulence_modes(seed: int = BASE_SEED + 6, kmax2: int = 9, slope: float = -11.0 / 6.0):
    """Seeded solenoidal Fourier amplitudes of a random velocity field on the unit periodic cube:
    integer wave vectors with 1 <= |k|^2 <= kmax2 (|k| <= 3), one of each +-k pair (first non-zero
    component positive), complex vector amplitudes with normal real and imaginary parts times
    |k|^slope (slope -11/6: a k^(-5/3) shell spectrum), projected onto the plane normal to k.
    Returns (k [nm, 3] int, A [nm, 3] complex); v(x) = sum_m Re(A_m exp(2 pi i k_m . x))."""
    ks = []
    for kz in range(-3, 4):
        for ky in range(-3, 4):
            for kx in range(-3, 4):
                k2 = kx * kx + ky * ky + kz * kz
                first = kx if kx != 0 else (ky if ky != 0 else kz)
                if 1 <= k2 <= kmax2 and first > 0:
                    ks.append((kx, ky, kz))
    k = np.array(ks, dtype=np.int64)
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((len(k), 3)) + 1j * rng.standard_normal((len(k), 3))
    kk = k.astype(np.float64)
    A *= (np.sqrt((kk * kk).sum(1)) ** slope)[:, None]
    A -= kk * ((A * kk).sum(1) / (kk * kk).sum(1))[:, None]
    return k, A


def turbulence_ic_state(wl: Workload, v_rms: float = 0.3, seed: int = BASE_SEED + 6) -> np.ndarray:
    """Modes of the driven-turbulence box started already turbulent: uniform density 1 and pressure
    1/gamma (sound speed 1) with the solenoidal random velocity of ``turbulence_modes`` scaled to the
    rms speed v_rms (rms Mach number v_rms), on a periodic cube.  Projected with the n+3 point Gauss
    rule like ``project``, but by separable per-axis tables of exp(2 pi i k x), one z-layer of cells
    at a time (128^3 cells at degree 3 take some tens of seconds)."""
    assert wl.dim == 3 and wl.basis == 0
    k, A = turbulence_modes(seed)
    A = A * (v_rms / np.sqrt(0.5 * np.sum(np.abs(A) ** 2)))  # <|v|^2> = sum |A|^2 / 2
    n, q = wl.n, wl.n + 3
    Q = n + 1
    x, g = npleg.leggauss(q)
    Bp = 0.5 * (g[:, None] * _pt_table(n, x))  # [q, Q]: (1/2) int over one axis of a cell
    N = wl.N
    L = [wl.hi[a] - wl.lo[a] for a in range(3)]
    # per-axis phase tables E[a][kk + 3][cell * q + j] = exp(2 pi i kk x_j / L_a)
    E = []
    for a in range(3):
        X = wl.lo[a] + (np.arange(N[a])[:, None] + 0.5 + 0.5 * x[None, :]) * (L[a] / N[a])
        E.append(np.exp(2j * np.pi * np.arange(-3, 4)[:, None] * X.reshape(1, -1) / L[a]))
    # amplitudes on the dense 7^3 cube of wave vectors
    C = np.zeros((7, 7, 7, 3), dtype=np.complex128)
    for m in range(len(k)):
        C[k[m, 0] + 3, k[m, 1] + 3, k[m, 2] + 3] += A[m]
    T1 = np.einsum("xX,xyzc->Xyzc", E[0], C)          # [Nx q, ky, kz, c]
    T2 = np.einsum("Xyzc,yY->cXYz", T1, E[1])         # [c, Nx q, Ny q, kz]
    T2r = np.ascontiguousarray(T2.real).reshape(-1, 7)
    T2i = np.ascontiguousarray(T2.imag).reshape(-1, 7)
    del T1, T2
    nf = wl.nfields
    out = np.zeros((nf, N[2], N[1], N[0], Q, Q, Q))   # [f][cz][cy][cx][lz][ly][lx]
    p0 = 1.0 / wl.gamma
    for cz in range(N[2]):
        Ez = E[2][:, cz * q:(cz + 1) * q]              # [kz, q]
        v = T2r @ Ez.real - T2i @ Ez.imag              # Re of the kz sum
        v = v.reshape(3, N[0], q, N[1], q, q)           # [c][cx][jx][cy][jy][jz]
        fields = [None, v[0], v[1], v[2], p0 / (wl.gamma - 1.0) + 0.5 * (v * v).sum(0)]
        for f in range(1, 5):
            # (1/|K|) int_K u phi_l: (1/2) g_j Pt_l(x_j) summed along each axis in turn (z, y, x)
            t = np.tensordot(fields[f], Bp, axes=([4], [0]))   # [cx, jx, cy, jy, lz]
            t = np.tensordot(t, Bp, axes=([3], [0]))           # [cx, jx, cy, lz, ly]
            t = np.tensordot(t, Bp, axes=([1], [0]))           # [cx, cy, lz, ly, lx]
            out[f, cz] = t.transpose(1, 0, 2, 3, 4)
    out[0, :, :, :, 0, 0, 0] = 1.0
    return np.ascontiguousarray(out.reshape(nf, wl.ncell, Q * Q * Q))


def sod_tube_ic(wl: Workload, axis: int = 0, x0: float = 0.5):
    """planar Sod shock tube along one axis (the 1-D Riemann problem embedded in 2-D/3-D)"""
    def f(X):
        left = X[:, axis] < x0
        rho = np.where(left, 1.0, 0.125)
        p = np.where(left, 1.0, 0.1)
        zero = np.zeros_like(rho)
        return _cons(wl.gamma, rho, [zero] * wl.dim, p, zero if wl.av_on else None)
    return f


def random_modal_state(wl: Workload, seed: int, amp: float = 0.05, decay: float = 0.5,
                       alpha_level: float = 0.3) -> np.ndarray:
    """A physical random state for operator parity: cell means rho~1, |v|~0.3, p~1 (varying from cell to
    cell) and higher modes drawn with amplitude amp * decay^(l_x+l_y+l_z) relative to the mean."""
    rng = np.random.default_rng(seed)
    d, n = wl.dim, wl.n
    midx = mode_exponents(d, n, wl.basis)
    scale = decay ** midx.sum(1)
    scale[0] = 0.0
    K = wl.ncell
    rho0 = 1.0 + 0.2 * rng.uniform(-1, 1, K)
    vel0 = [0.3 * rng.uniform(-1, 1, K) for _ in range(d)]
    p0 = 1.0 + 0.3 * rng.uniform(-1, 1, K)
    mean = _cons(wl.gamma, rho0, vel0, p0, alpha_level * rng.uniform(0, 1, K) if wl.av_on else None)
    if wl.tracer_on:  # rho c with c in [0.2, 1], inserted after the energy
        mean = np.insert(mean, d + 2, rho0 * rng.uniform(0.2, 1.0, K), axis=0)
    w = np.zeros(wl.shape())
    w[:, :, 0] = mean
    hi = rng.uniform(-1, 1, (wl.nfields, K, wl.M)) * scale[None, None, :] * amp
    w += hi * np.abs(mean)[:, :, None].clip(min=0.2)
    return np.ascontiguousarray(w)


# ------------------------------------------------------------------ batched ensemble (64 uneven 2-D runs)

def _proj1d(n: int, N: int, lo: float, hi: float, func, q: int | None = None) -> np.ndarray:
    """[N, n+1] coefficients of the 1-D projection of func onto Pt_l in each of N equal cells."""
    q = n + 3 if q is None else q
    x, g = npleg.leggauss(q)
    B = _pt_table(n, x)  # [q, n+1]
    h = (hi - lo) / N
    xc = lo + (np.arange(N) + 0.5) * h
    X = xc[:, None] + 0.5 * h * x[None, :]
    return 0.5 * np.einsum("kj,j,jl->kl", func(X), g, B)


def _outer2d(A: np.ndarray, Bm: np.ndarray) -> np.ndarray:
    """2-D modes from per-axis factors: w[iy*Nx+ix][lx + Q ly] = A[ix][lx] B[iy][ly]."""
    Nx, Q = A.shape
    Ny = Bm.shape[0]
    w = np.einsum("xa,yb->yxba", A, Bm)  # [iy][ix][ly][lx]
    return w.reshape(Ny * Nx, Q * Q)


@dataclass(frozen=True)
class Member:
    wl: Workload
    kind: str  # "wave" or "sod"
    axis: int  # shock-tube axis


def c5_manifest(seed: int = BASE_SEED, count: int = 64, log2_cells=(6, 10)):
    """64 independent 2-D runs: cells per axis drawn from {64,128,256,512} (log-uniform; log2_cells
    gives the half-open range of log2 of the cells per axis), degree uniform in 1..5, half smooth
    density waves (periodic) and half Sod tubes along a seeded axis (outflow along it, positivity
    limiter on), half of all members with NS (nu = kappa = 1e-4); AV on for all."""
    rng = np.random.default_rng(seed + 5)
    out = []
    for i in range(count):
        N = int(2 ** rng.integers(*log2_cells))
        n = int(rng.integers(1, 6))
        kind = "wave" if rng.random() < 0.5 else "sod"
        axis = int(rng.integers(0, 2))
        ns = rng.random() < 0.5
        bc = (0, 0, 0)
        gamma = 5.0 / 3.0
        if kind == "sod":
            bc = (1, 0, 0) if axis == 0 else (0, 1, 0)
            gamma = 1.4
        nu = 1e-4 if ns else 0.0
        wl = Workload(f"member{i}", 2, n, (N, N, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), bc=bc, gamma=gamma, nu=nu,
                      kappa=nu, av_on=1, cfl=0.3, steps=50, positivity_on=1 if kind == "sod" else 0)
        out.append(Member(wl, kind, axis))
    return out


def member_state(m: Member) -> np.ndarray:
    """initial modes of an ensemble member by separable projection (exact for these initial states)"""
    wl = m.wl
    n, N = wl.n, wl.N[0]
    Q = n + 1
    w = np.zeros(wl.shape())
    if m.kind == "wave":
        # rho = 1 + 0.2 sin 2pi(x+y) = 1 + 0.2 (sin 2pi x cos 2pi y + cos 2pi x sin 2pi y); v = (1,1); p = 1
        Sx = _proj1d(n, N, 0.0, 1.0, lambda X: np.sin(2 * np.pi * X))
        Cx = _proj1d(n, N, 0.0, 1.0, lambda X: np.cos(2 * np.pi * X))
        rho = 0.2 * (_outer2d(Sx, Cx) + _outer2d(Cx, Sx))
        rho[:, 0] += 1.0
        w[0] = rho
        w[1] = rho
        w[2] = rho
        w[3] = rho
        w[3][:, 0] += 1.0 / (wl.gamma - 1.0)
    else:
        step = lambda lo_v, hi_v: (lambda X: np.where(X < 0.5, lo_v, hi_v))
        r1 = _proj1d(n, N, 0.0, 1.0, step(1.0, 0.125))
        p1 = _proj1d(n, N, 0.0, 1.0, step(1.0, 0.1))
        one = np.zeros((N, Q))
        one[:, 0] = 1.0
        if m.axis == 0:
            w[0] = _outer2d(r1, one)
            w[3] = _outer2d(p1, one) / (wl.gamma - 1.0)
        else:
            w[0] = _outer2d(one, r1)
            w[3] = _outer2d(one, p1) / (wl.gamma - 1.0)
    return np.ascontiguousarray(w)
