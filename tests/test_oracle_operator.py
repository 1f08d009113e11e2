"""Whole-operator pins of the oracle (CPU only): (b) free-stream preservation, (c) conservation on
periodic domains, (d) order n+1 convergence on the advected density wave, (e) the exact Riemann
solution of a shock tube embedded in 2-D, plus the viscous shear-wave decay (Sec. 3.3) and the
decay of the artificial-viscosity field (Eq. timedependentviscosity) under the Runge-Kutta scheme.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import riemann
from paper_2208_11131_gb300 import inputs


def _cons_const(g, rho, v, p):
    v = np.asarray(v, dtype=float)
    return np.concatenate([[rho], rho * v, [p / (g - 1) + 0.5 * rho * v @ v]])


@pytest.mark.parametrize("dim,n,nu,av", [(2, 0, 0.0, 0), (2, 2, 0.0, 0), (2, 3, 1e-2, 1), (3, 1, 0.0, 1),
                                         (3, 2, 1e-3, 1)])
def test_free_stream_preserved(dim, n, nu, av):
    g = 1.4
    P = oracle.Problem(dim=dim, n=n, N=(4, 3, 2)[:dim], hi=(1.0, 2.0, 0.5)[:dim], gamma=g, nu=nu, kappa=nu,
                       av_on=av)
    w = np.zeros(P.shape())
    w[:dim + 2, :, 0] = _cons_const(g, 1.3, [0.4, -0.2, 0.7][:dim], 0.9)[:, None]
    if av:
        w[-1, :, 0] = 0.6  # uniform alpha: only its decay term acts
    r, st = oracle.rhs(P, w)
    assert st == 0
    assert np.abs(r[:dim + 2]).max() < 1e-13
    if av:
        cs = math.sqrt(g * 0.9 / 1.3)
        tau = 0.5 * min(P.h) / ((n + 1) * cs)
        assert abs(r[-1, :, 0] + 0.6 / tau).max() < 1e-12
        assert np.abs(r[-1, :, 1:]).max() < 1e-12


@pytest.mark.parametrize("dim,n,nu,av", [(2, 1, 0.0, 0), (2, 3, 3e-3, 1), (3, 2, 1e-3, 1)])
def test_conservation_periodic(dim, n, nu, av):
    wl = inputs.Workload("t", dim, n, (5, 4, 3)[:dim] + (1,) * (3 - dim), (0, 0, 0), (1.0, 1.5, 0.8), gamma=1.4,
                         nu=nu, kappa=nu, av_on=av)
    P = oracle.Problem(dim=dim, n=n, N=wl.N[:dim], hi=wl.hi[:dim], gamma=1.4, nu=nu, kappa=nu, av_on=av)
    w = inputs.random_modal_state(wl, seed=5)
    wig = np.random.default_rng(1).uniform(0, 1, P.ncell)
    r, st = oracle.rhs(P, w, wig)
    assert st == 0
    vol = np.prod(P.h)
    for f in range(dim + 2):
        tot = vol * r[f, :, 0].sum()
        assert abs(tot) < 1e-13 * vol * np.abs(r[f, :, 0]).sum()
    # and over whole SSP-RK steps
    s = oracle.Sim(P, w)
    m0 = s.w[:dim + 2, :, 0].sum(1)
    for _ in range(3):
        _, st = s.step()
        assert st == 0
    assert np.allclose(s.w[:dim + 2, :, 0].sum(1), m0, rtol=1e-13, atol=1e-13 * np.abs(m0).max())


@pytest.mark.parametrize("n,Ns", [(1, (8, 16)), (2, (8, 16)), (3, (6, 12))])
def test_convergence_order_density_wave(n, Ns):
    """(d) order n+1 on the smoothly advected density wave (2-D Euler, gamma=5/3, v=(1,1), P=1)."""
    T = 0.05
    errs = []
    for N in Ns:
        wl = inputs.c1_density_wave(N=N, n=n)
        P = oracle.Problem(dim=2, n=n, N=(N, N), gamma=wl.gamma, cfl=0.3)
        s = oracle.Sim(P, oracle.project(P, inputs.density_wave_ic(wl, 0.0)))
        while s.t < T - 1e-14:
            dt, _ = oracle.max_dt(P, s.w)
            s.step(min(dt, T - s.t))
        errs.append(oracle.l1_error(P, s.w, inputs.density_wave_ic(wl, T)))
    slope = math.log(errs[0] / errs[1]) / math.log(Ns[1] / Ns[0])
    assert n + 1 - 0.35 < slope < n + 1 + 0.6, (errs, slope)


def test_convergence_order_3d():
    T = 0.02
    errs = []
    for N in (4, 8):
        P = oracle.Problem(dim=3, n=1, N=(N, N, N), gamma=1.4, cfl=0.3)

        def ex(t):
            def f(X):
                rho = 1 + 0.2 * np.sin(2 * np.pi * (X[:, 0] + X[:, 1] + X[:, 2] - 1.5 * t))
                one = np.ones_like(rho)
                return np.stack([rho, 0.5 * rho, 0.5 * rho, 0.5 * rho, one / 0.4 + 0.5 * rho * 0.75])
            return f
        s = oracle.Sim(P, oracle.project(P, ex(0)))
        while s.t < T - 1e-14:
            dt, _ = oracle.max_dt(P, s.w)
            s.step(min(dt, T - s.t))
        errs.append(oracle.l1_error(P, s.w, ex(T)))
    assert 1.6 < math.log2(errs[0] / errs[1]) < 2.8, errs


def test_shock_tube_embedded_in_2d_vs_exact_riemann():
    """(e) Sod tube along x in a 2-D box (outflow in x, periodic in y), AV + positivity, n=2:
    first-order L1 convergence towards the exact Riemann solution and exact y-independence."""
    g, T = 1.4, 0.2
    errs = []
    for N in (48, 96):
        P = oracle.Problem(dim=2, n=2, N=(N, 2), hi=(1.0, 2.0 / N), bc=(1, 0), gamma=g, av_on=1, positivity_on=1,
                           cfl=0.3)
        wl = inputs.Workload("sod", 2, 2, (N, 2, 1), (0, 0, 0), (1.0, 2.0 / N, 1.0), bc=(1, 0, 0), gamma=g, av_on=1)
        s = oracle.Sim(P, oracle.project(P, inputs.sod_tube_ic(wl)))
        while s.t < T - 1e-14:
            dt, _ = oracle.max_dt(P, s.w)
            _, st = s.step(min(dt, T - s.t))
            assert st == 0

        def ex(X):
            r, u, p = riemann.sample((1, 0, 1), (0.125, 0, 0.1), g, (X[:, 0] - 0.5) / T)
            return np.stack([r, r * u, 0 * r, p / (g - 1) + 0.5 * r * u * u, 0 * r])
        errs.append(oracle.l1_error(P, s.w, ex))
        assert np.array_equal(s.w[:, :N], s.w[:, N:])
    assert errs[0] < 0.009 and errs[1] < 0.005 and errs[0] / errs[1] > 1.5, errs


@pytest.mark.parametrize("n,tol", [(2, 3e-3), (3, 5e-4)])
def test_viscous_shear_wave_decay(n, tol):
    """v_x = A sin(2 pi y): linear momentum decays as exp(-nu (2 pi)^2 t) (Sec. 3.3 stress tensor),
    reached through the recovered interface gradients (Sec. 3.2)."""
    g, nu, A, T = 1.4, 0.01, 1e-3, 0.5
    P = oracle.Problem(dim=2, n=n, N=(8, 8), gamma=g, nu=nu, cfl=0.3)

    def ic(X):
        y = X[:, 1]
        vx = A * np.sin(2 * np.pi * y)
        one = np.ones_like(y)
        return np.stack([one, vx, 0 * y, one / (g - 1) + 0.5 * vx**2])
    w0 = oracle.project(P, ic)
    s = oracle.Sim(P, w0)
    while s.t < T - 1e-14:
        dt, _ = oracle.max_dt(P, s.w)
        s.step(min(dt, T - s.t))
    amp = np.sum(s.w[1] * w0[1]) / np.sum(w0[1] * w0[1])
    assert abs(amp / math.exp(-nu * (2 * math.pi) ** 2 * T) - 1) < tol


@pytest.mark.parametrize("n", [2, 3])
def test_alpha_field_decay_follows_rk_stability_polynomial(n):
    """uniform flow, no compression, no wiggles: d alpha/dt = -alpha/tau, tau = f_tau h/(P c_s)
    (Eq. timedependentviscosity); one SSP-RK step multiplies alpha by R(-dt/tau)."""
    g = 1.4
    P = oracle.Problem(dim=2, n=n, N=(4, 4), gamma=g, av_on=1, cfl=0.3)

    def ic(X):
        x = X[:, 0]
        one = np.ones_like(x)
        return np.stack([one, 0.3 * one, 0.1 * one, one / (g - 1) + 0.05 * one, 0.5 + 0.1 * np.sin(2 * np.pi * x)])
    s = oracle.Sim(P, oracle.project(P, ic))
    a0 = s.w[4].copy()
    tau = 0.5 * 0.25 / ((n + 1) * math.sqrt(g))
    fac = 1.0
    if n == 2:
        R = lambda z: 1 + z + z * z / 2 + z**3 / 6
    else:
        al, be = oracle.rk_table(5)
        A = np.zeros((6, 6))
        for i in range(1, 6):
            for k in range(i):
                A[i] += al[i, k] * A[k]
                A[i, k] += be[i, k]
        b, Am = A[5, :5], A[:5, :5]
        R = lambda z: 1 + z * b @ np.linalg.solve(np.eye(5) - z * Am, np.ones(5))
    for _ in range(6):
        dt, st = s.step()
        assert st == 0
        fac *= R(-dt / tau)
    assert np.abs(s.w[4] - a0 * fac).max() < 1e-13
    assert np.abs(s.w[:4, :, 1:]).max() < 1e-13


def test_inputs_projection_matches_oracle_projection():
    """the seeded generator's numpy projection and the oracle's own projection agree"""
    wl = inputs.c2_shear_layer(N=8, n=3)
    P = oracle.Problem(dim=2, n=3, N=(8, 8), hi=(1.0, 2.0), gamma=wl.gamma, av_on=1)
    a = inputs.project(wl, inputs.shear_layer_ic(wl))
    b = oracle.project(P, inputs.shear_layer_ic(wl))
    assert np.abs(a - b).max() < 1e-13


def test_ensemble_separable_projection_matches_full_projection():
    """the fast separable projection of the ensemble's initial states equals the full 2-D projection"""
    for m in inputs.c5_manifest(count=6):
        wl = m.wl.with_(N=(8, 8, 1))
        mm = inputs.Member(wl, m.kind, m.axis)
        P = oracle.Problem(dim=2, n=wl.n, N=(8, 8), gamma=wl.gamma, av_on=1)
        if m.kind == "wave":
            ref = oracle.project(P, inputs.density_wave_ic(wl, 0.0))
        else:
            ref = oracle.project(P, inputs.sod_tube_ic(wl, axis=m.axis))
        assert np.abs(inputs.member_state(mm) - ref).max() < 1e-13


@pytest.mark.parametrize("n", [1, 2, 3])
def test_isentropic_vortex_convergence_order(n):
    """Sec. 5.1: the steady isentropic vortex converges at order n+1 in the cell size (t = 1)"""
    errs = []
    for N in (16, 32):
        wl = inputs.isentropic_vortex(N=N, n=n)
        P = oracle.Problem(dim=2, n=n, N=(N, N), lo=(-5.0, -5.0), hi=(5.0, 5.0), gamma=1.4, cfl=0.3)
        s = oracle.Sim(P, oracle.project(P, inputs.isentropic_vortex_ic(wl)))
        while s.t < 1.0 - 1e-14:
            dt, _ = oracle.max_dt(P, s.w)
            _, st = s.step(min(dt, 1.0 - s.t))
            assert st == 0
        errs.append(oracle.l1_error(P, s.w, inputs.isentropic_vortex_ic(wl)))
    slope = math.log2(errs[0] / errs[1])
    assert n + 1 - 0.3 < slope < n + 1 + 0.5, (errs, slope)


def test_isentropic_vortex_exponential_in_order():
    """Sec. 5.1: at a fixed grid the error falls exponentially with the order (here by more than 5x
    per degree, n = 1..4 on 16^2 cells at t = 1)"""
    errs = []
    for n in (1, 2, 3, 4):
        wl = inputs.isentropic_vortex(N=16, n=n)
        P = oracle.Problem(dim=2, n=n, N=(16, 16), lo=(-5.0, -5.0), hi=(5.0, 5.0), gamma=1.4, cfl=0.3)
        s = oracle.Sim(P, oracle.project(P, inputs.isentropic_vortex_ic(wl)))
        while s.t < 1.0 - 1e-14:
            dt, _ = oracle.max_dt(P, s.w)
            _, st = s.step(min(dt, 1.0 - s.t))
            assert st == 0
        errs.append(oracle.l1_error(P, s.w, inputs.isentropic_vortex_ic(wl)))
    assert all(errs[k] / errs[k + 1] > 5.0 for k in range(3)), errs


def test_isentropic_vortex_initial_state_is_steady_and_isentropic():
    """the set-up is an exact steady solution: p = rho^gamma and dp/dr = rho v_theta^2 / r"""
    wl = inputs.isentropic_vortex(N=8, n=1)
    r = np.linspace(0.05, 4.0, 400)
    X = np.stack([r, 0 * r], 1)
    U = inputs.isentropic_vortex_ic(wl)(X)
    g = wl.gamma
    rho, vy = U[0], U[2] / U[0]
    p = (g - 1) * (U[3] - 0.5 * rho * vy * vy)
    assert np.allclose(p, rho ** g, rtol=1e-13)
    # radial balance by the derivative of the closed form p = rho^gamma
    dr = 1e-6
    Up = inputs.isentropic_vortex_ic(wl)(np.stack([r + dr, 0 * r], 1))
    Um = inputs.isentropic_vortex_ic(wl)(np.stack([r - dr, 0 * r], 1))
    dpdr = (Up[0] ** g - Um[0] ** g) / (2 * dr)
    assert np.allclose(dpdr, rho * vy * vy / r, rtol=1e-6, atol=1e-9)  # difference roundoff ~ eps p / dr
    # background state of Yee's set-up
    far = inputs.isentropic_vortex_ic(wl)(np.array([[5.0, 5.0]]))
    assert abs(far[0, 0] - 1.0) < 1e-9
