"""Pins of the oracle's artificial-viscosity dynamics (Sec. 4.1) by what they must do, not by their
formulas, CPU only.

* The wiggle source f_w max(0, d ln S/dt) [S > S_onset] takes the logarithm of the oscillation
  sensor of the previous step.  Ahead of a discontinuity the higher density modes of a uniform cell
  are rounding noise, so the sensor there is noise too; the reading floors S at 1e-4 S_onset inside
  the logarithm.  Two states that differ only by rounding-level values in their top density modes
  must then give the same alpha field; with a floor at rounding level (1e-30) they do not, because
  the wiggle source of the cells the wave reaches becomes ln(noise) / dt.
* Sec. 4.1 measures the width of a Mach-3 shock (gamma = 5/3, into gas at rest with unit density
  and pressure, h = 1/21, shock at x = 0.5) between 20% and 80% of the density jump and finds it
  proportional to 1/p for p >= 2.  The oracle's AV (epsilon = alpha c_s h / P, alpha equation,
  sensor, wiggle term) must reproduce that law; planting epsilon = alpha c_s h (no 1/P) breaks it.
"""
import numpy as np
import pytest

import oracle
from paper_2208_11131_gb300 import inputs


def _sod_pair():
    wl = inputs.Workload("sod", 2, 3, (24, 2, 1), (0, 0, 0), (1.0, 2.0 / 24, 1.0), bc=(1, 0, 0), gamma=1.4,
                         av_on=1, positivity_on=1, cfl=0.3)
    wA = inputs.project(wl, inputs.sod_tube_ic(wl))
    Q = wl.n + 1
    top = [l for l in range(Q * Q) if (l % Q == wl.n or l // Q == wl.n)]
    # the discontinuity sits on a face: every cell starts uniform, its top modes rounding noise
    assert np.abs(wA[0][:, top]).max() < 1e-15
    wB = wA.copy()
    wB[0][:, top] += 1e-14 * np.random.default_rng(3).standard_normal((wl.ncell, len(top)))
    return wA, wB


def _alpha_gap(s_floor, steps=3):
    wA, wB = _sod_pair()
    P = oracle.Problem(dim=2, n=3, N=(24, 2), hi=(1.0, 2.0 / 24), bc=(1, 0), gamma=1.4, av_on=1, positivity_on=1,
                       cfl=0.3, s_floor=s_floor)
    a, b = oracle.Sim(P, wA), oracle.Sim(P, wB)
    gap = 0.0
    for _ in range(steps):
        dt, st = a.step()
        assert st == 0
        _, st = b.step(dt)
        assert st == 0
        gap = max(gap, float(np.abs(a.w[4] - b.w[4]).max()))
    assert np.abs(a.w[4]).max() > 0.5  # the wave switched the viscosity on
    return gap


def test_wiggle_source_ignores_rounding_noise_of_the_sensor():
    assert _alpha_gap(oracle.Problem(dim=2, n=1, N=(1, 1)).s_floor) < 1e-10


def test_rounding_level_floor_lets_noise_into_alpha():
    """the same pair with the sensor floored at 1e-30 instead: alpha differs at order one"""
    s_on = 1e-4 / 16
    assert _alpha_gap(1e-30 / s_on) > 0.1


def _mach3_width(n, av_scale=1.0, N=21):
    """width (in cells) between 20% and 80% of the density jump of a Mach-3 shock reaching x = 0.5"""
    g, M = 5.0 / 3.0, 3.0
    r2 = (g + 1) * M * M / ((g - 1) * M * M + 2)  # Rankine-Hugoniot: 3
    p2 = (2 * g * M * M - (g - 1)) / (g + 1)       # 11
    vs = M * np.sqrt(g)
    u2 = vs * (1 - 1 / r2)
    x0 = 5.0 / N
    # the positivity limiter of Sec. 4.2 is on, as in the paper's runs (the first steps of a projected
    # strong jump are non-physical at some Gauss points without it)
    P = oracle.Problem(dim=2, n=n, N=(N, 1), hi=(1.0, 1.0 / N), bc=(1, 0), gamma=g, av_on=1, cfl=0.3,
                       positivity_on=1, av_scale=av_scale)
    wl = inputs.Workload("m3", 2, n, (N, 1, 1), (0, 0, 0), (1.0, 1.0 / N, 1.0), bc=(1, 0, 0), gamma=g, av_on=1)

    def ic(X):
        left = X[:, 0] < x0
        z = np.zeros(len(X))
        return inputs._cons(g, np.where(left, r2, 1.0), [np.where(left, u2, 0.0), z], np.where(left, p2, 1.0), z)

    sim = oracle.Sim(P, inputs.project(wl, ic))
    T = (0.5 - x0) / vs
    while sim.t < T - 1e-14:
        dt, _ = oracle.max_dt(P, sim.w)
        _, st = sim.step(min(dt, T - sim.t))
        assert st == 0
    m = 40 * N * (n + 1)
    xs = (np.arange(m) + 0.5) / m
    cell = np.minimum((xs * N).astype(int), N - 1)
    xi = 2 * (xs * N - cell) - 1
    rho = np.einsum("kl,kl->k", sim.w[0][cell], oracle.basis_eval(2, n, np.stack([xi, np.zeros_like(xi)], 1)))
    i20 = np.max(np.nonzero(rho > 1.0 + 0.2 * (r2 - 1.0))[0])
    i80 = np.max(np.nonzero(rho > 1.0 + 0.8 * (r2 - 1.0))[0])
    return (xs[i20] - xs[i80]) * N


def test_shock_width_scales_as_one_over_p():
    widths = {n + 1: _mach3_width(n) for n in range(1, 6)}
    wp = np.array([w * p for p, w in widths.items()])
    # width * p / h constant to within 15% over p = 2..6 (the oracle gives 2.4 - 2.7 cells)
    assert wp.max() / wp.min() < 1.15, widths
    assert widths[6] < 0.4 * widths[2], widths
    # and sub-cell at high order
    assert widths[6] < 0.5


def test_shock_width_law_fails_without_the_order_factor_of_epsilon():
    """planted: epsilon = alpha c_s h (av_scale = P cancels the 1/P): the width no longer falls as 1/p"""
    w2 = _mach3_width(1, av_scale=2.0)
    w6 = _mach3_width(5, av_scale=6.0)
    assert w6 * 6 > 2.0 * w2 * 2
