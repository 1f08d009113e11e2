"""Pins of the oracle's turbulence driving (Sec. 7.1, "Driving"), CPU only.

What the paper fixes: modes with 2pi/L <= |k| <= 2 (2pi/L), amplitude proportional to |k|^(-5/3),
Ornstein-Uhlenbeck phases updated at intervals with correlation time t_s, the solenoidal
projection (delta_ij - k_i k_j / k^2), a momentum source rho s and an energy source rho s.v,
integrated with the Gauss rule.  Each pin below would fail on a plausible mistake: a missing
projection (divergence), a k=0 or wrong-shell mode (Fourier support), a wrong OU decay or noise
factor (stationary variance, lag correlation), a wrong amplitude law (shell power ratio), a wrong
quadrature weight, node coordinate or field in the source (independent numpy assembly), an
update schedule off by one (update count).
"""
import math

import numpy as np
import pytest

import oracle


def _prob(dim=3, n=2, N=4, hi=None, **kw):
    hi = hi or (1.0,) * dim
    args = dict(dim=dim, n=n, N=(N,) * dim, hi=hi, gamma=1.001, forcing_on=1, force_amp=0.7, force_ts=1.0,
                force_dt=0.01, force_seed=1234)
    args.update(kw)
    return oracle.Problem(**args)


def test_modes_are_the_half_shell_1_to_2():
    for dim, count in ((2, 6), (3, 16)):
        k = oracle.forcing_modes(dim)
        assert len(k) == count
        k2 = (k * k).sum(1)
        assert k2.min() == 1 and k2.max() == 4
        # exactly one of every +-k pair, and every integer vector of the shell is covered
        full = {tuple(v) for v in k} | {tuple(-v) for v in k}
        rng = range(-2, 3)
        shell = {(a, b, c) for a in rng for b in rng for c in (rng if dim == 3 else [0])
                 if 1 <= a * a + b * b + c * c <= 4}
        assert full == shell and len(full) == 2 * count


def test_uniform_and_normal_draws():
    u = np.array([oracle.forcing_uniform(99, i) for i in range(40000)])
    assert u.min() > 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 4 * 0.2887 / math.sqrt(u.size)
    z = np.array([oracle.forcing_normal(99, c) for c in range(40000)])
    assert abs(z.mean()) < 4 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 0.03
    assert abs(np.mean(z ** 4) - 3.0) < 0.15  # Gaussian kurtosis
    # counters are independent streams: a different seed gives different draws
    assert oracle.forcing_normal(98, 5) != oracle.forcing_normal(99, 5)


def test_ou_stationary_variance_and_lag_correlation():
    P = _prob(dim=3, force_dt=0.1, force_ts=1.0)
    f = oracle.forcing_state()
    xs = []
    for j in range(1500):
        assert oracle.forcing_update(P, f, j * 0.1 + 1e-9) == 0
        assert f[0] == j
        xs.append(f[1:].copy())
    X = np.array(xs)  # [updates, 96]
    assert abs(X.var() - 1.0) < 0.04
    a, b = X[:-1].ravel(), X[1:].ravel()
    corr = np.mean(a * b) / np.sqrt(np.mean(a * a) * np.mean(b * b))
    assert abs(corr - math.exp(-0.1)) < 0.02, corr


def test_update_schedule():
    P = _prob(dim=2, force_dt=0.01)
    f = oracle.forcing_state()
    for t, expect in ((0.0, 0), (0.0099, 0), (0.01, 1), (0.0375, 3), (0.0375, 3), (0.1, 10)):
        oracle.forcing_update(P, f, t)
        assert f[0] == expect
    # components beyond d stay zero in 2-D
    assert np.all(f[1:].reshape(16, 6)[:, [2, 5]] == 0.0)


def _field_on_grid(P, f, G):
    d = P.dim
    ax = [P.lo[a] + (P.hi[a] - P.lo[a]) * np.arange(G) / G for a in range(d)]
    mesh = np.meshgrid(*ax, indexing="ij")
    X = np.stack([m.ravel() for m in mesh], 1)
    return oracle.forcing_eval(P, f, X)[:, :d].reshape((G,) * d + (d,))


@pytest.mark.parametrize("dim,hi", [(2, (1.0, 2.0)), (3, (1.0, 1.0, 1.0)), (3, (1.0, 0.5, 2.0))])
def test_field_is_solenoidal_zero_mean_and_band_limited(dim, hi):
    P = _prob(dim=dim, hi=hi)
    f = oracle.forcing_state()
    oracle.forcing_update(P, f, 0.37)
    # divergence by central differences at random points
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 1, (64, dim)) * np.array(hi)
    eps = 1e-5
    div = np.zeros(len(X))
    gscale = 0.0
    for a in range(dim):
        e = np.zeros(dim)
        e[a] = eps
        dsa = (oracle.forcing_eval(P, f, X + e) - oracle.forcing_eval(P, f, X - e)) / (2 * eps)
        div += dsa[:, a]
        gscale = max(gscale, np.abs(dsa).max())
    assert np.abs(div).max() < 1e-7 * gscale
    # Fourier analysis on an 8^d grid (exact for |k_a| <= 2)
    G = 8
    S = _field_on_grid(P, f, G)
    assert np.abs(S.mean(axis=tuple(range(dim)))).max() < 1e-14 * np.abs(S).max()
    Fh = np.fft.fftn(S, axes=tuple(range(dim))) / G ** dim
    kint = np.fft.fftfreq(G, 1.0 / G).astype(int)
    Kg = np.stack(np.meshgrid(*([kint] * dim), indexing="ij"), -1)  # integer wave vectors
    k2 = (Kg * Kg).sum(-1)
    outside = (k2 < 1) | (k2 > 4)
    assert np.abs(Fh[outside]).max() < 1e-13 * np.abs(Fh).max()
    # each retained coefficient is normal to its physical wave vector and has the prescribed size
    L = np.array(hi)
    kmodes = oracle.forcing_modes(dim)
    for m, k in enumerate(kmodes):
        kk = k[:dim]
        c = Fh[tuple(kk % G)]  # coefficient of exp(+i K.x): half the complex amplitude s_m
        Kp = 2 * np.pi * kk / L
        assert abs(np.dot(Kp, c)) < 1e-12 * np.abs(c).max() * np.linalg.norm(Kp)
        X_ = f[1 + 6 * m: 1 + 6 * m + dim]
        Y_ = f[4 + 6 * m: 4 + 6 * m + dim]
        z = X_ + 1j * Y_
        z = z - Kp * np.dot(Kp, z) / np.dot(Kp, Kp)
        expect = 0.5 * 0.7 * np.linalg.norm(kk) ** (-5.0 / 3.0) * z
        assert np.allclose(c, expect, rtol=1e-12, atol=1e-14)


def test_shell_power_follows_k_to_minus_five_thirds():
    """ensemble over OU states: mean |s_k|^2 at |k| = 2 over that at |k| = 1 is 2^(-10/3)
    (the solenoidal projection keeps (d-1)/d of an isotropic vector's variance at every k)"""
    P = _prob(dim=3, force_dt=1.0, force_ts=0.05)  # nearly independent draws per update
    f = oracle.forcing_state()
    k = oracle.forcing_modes(3)
    k2 = (k * k).sum(1)
    p1, p4 = [], []
    for j in range(3000):
        oracle.forcing_update(P, f, float(j))
        X = f[1:].reshape(16, 6)
        for m in range(16):
            Kp = 2 * np.pi * k[m]
            z = X[m, :3] + 1j * X[m, 3:]
            z = z - Kp * np.dot(Kp, z) / np.dot(Kp, Kp)
            amp2 = (0.7 * math.sqrt(k2[m]) ** (-5.0 / 3.0)) ** 2 * np.vdot(z, z).real
            (p1 if k2[m] == 1 else p4 if k2[m] == 4 else []).append(amp2)
    ratio = np.mean(p4) / np.mean(p1)
    assert abs(ratio / 2 ** (-10.0 / 3.0) - 1) < 0.05
    assert abs(np.mean(p1) / (0.7 ** 2 * 2 * 2) - 1) < 0.05  # 2 of 3 components x (re, im)


@pytest.mark.parametrize("dim,n", [(2, 2), (3, 1), (3, 3)])
def test_rhs_source_equals_independent_gauss_assembly(dim, n):
    """uniform state: every flux term cancels and the right-hand side is the driving source alone,
    2^-d sum_j G_j phi_l(xi_j) S(x_j) with S = (0, rho s, s.(rho v)) -- assembled here in numpy"""
    N = 3
    P = _prob(dim=dim, n=n, N=N, hi=(1.0, 1.5, 0.75)[:dim])
    f = oracle.forcing_state()
    oracle.forcing_update(P, f, 0.05)
    rho, v, p = 1.3, np.array([0.2, -0.1, 0.3])[:dim], 0.8
    w = np.zeros(P.shape())
    w[0, :, 0] = rho
    w[1:dim + 1, :, 0] = (rho * v)[:, None]
    w[dim + 1, :, 0] = p / (P.gamma - 1) + 0.5 * rho * v @ v
    r, st = oracle.rhs(P, w, fst=f)
    assert st == 0
    xg, wg = np.polynomial.legendre.leggauss(n + 1)
    idx = np.stack(np.meshgrid(*([np.arange(n + 1)] * dim), indexing="ij")[::-1], -1).reshape(-1, dim)
    xi = xg[idx]  # [Q^d, d], axis 0 fastest
    G = np.prod(wg[idx], 1)
    midx = idx  # same ordering for modes
    phi = np.ones((len(xi), len(midx)))
    for a in range(dim):
        Pt = np.stack([math.sqrt(2 * l + 1) * np.polynomial.legendre.legval(xi[:, a], [0] * l + [1])
                       for l in range(n + 1)], 1)
        phi *= Pt[:, midx[:, a]]
    xc = P.cell_centres()
    h = np.array(P.h)
    X = (xc[:, None, :] + 0.5 * h * xi[None]).reshape(-1, dim)
    s = oracle.forcing_eval(P, f, X)[:, :dim].reshape(P.ncell, len(xi), dim)
    src = np.zeros((dim + 2, P.ncell, len(xi)))
    src[1:dim + 1] = np.moveaxis(rho * s, -1, 0)
    src[dim + 1] = s @ (rho * v)
    expect = np.einsum("fkj,j,jl->fkl", src, G, phi) / 2.0 ** dim
    # the flux terms of the uniform state cancel to rounding of the flux size (e + p)|v| 2/h
    # (e = 800 at gamma = 1.001)
    e = w[dim + 1, 0, 0]
    flux = (np.abs(e) + p) * np.abs(v).max() * 2.0 / min(h) + np.abs(expect).max()
    assert np.abs(r[:dim + 2] - expect).max() < 2e-14 * flux
    assert np.abs(r[0]).max() < 2e-14 * flux


def test_step_from_rest_injects_no_net_momentum_and_does_work():
    """from rest at uniform density: one forward-Euler stage adds dt * int rho s = 0 net momentum
    and no energy (s.(rho v) = 0 at rest); over later steps the drive does positive work"""
    dim = 3
    P = _prob(dim=dim, n=1, N=4, cfl=0.3, rk_stages=1)
    w = np.zeros(P.shape())
    w[0, :, 0] = 1.0
    w[dim + 1, :, 0] = 1.0 / (P.gamma * (P.gamma - 1))
    sim = oracle.Sim(P, w)
    e0 = sim.w[dim + 1, :, 0].sum()
    _, st = sim.step(0.01)
    assert st == 0
    mom = sim.w[1:dim + 1, :, 0].sum(1)
    assert np.abs(mom).max() < 1e-14 * np.abs(sim.w[1:dim + 1, :, 0]).max() * P.ncell
    assert abs(sim.w[dim + 1, :, 0].sum() - e0) < 1e-14 * abs(e0)
    P3 = _prob(dim=dim, n=1, N=4, cfl=0.3)
    sim = oracle.Sim(P3, w)
    for _ in range(3):
        _, st = sim.step(0.01)
        assert st == 0
    assert sim.fst[0] == 2  # updates at the step starts t = 0, 0.01, 0.02
    assert sim.w[dim + 1, :, 0].sum() > e0 * (1 + 1e-9)
