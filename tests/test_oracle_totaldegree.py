"""Pins of the oracle's total-degree basis (Sec. 2.3: products of scaled Legendre polynomials with
l_x + l_y + l_z <= n), CPU only.

* the mode counts are the paper's: (n+1)(n+2)/2 in 2-D and the N3D(n) that the memory table of
  Sec. 8.3 is printed with (tests/golden/memory_table.txt);
* projection of a total-degree-n polynomial is exact;
* on a state in the total-degree space the right-hand side equals the tensor-basis right-hand
  side restricted to the total-degree modes (the two bases share every quadrature point and the
  total-degree modes are a subset of the orthonormal tensor modes, so the Galerkin projection
  onto the smaller space is the restriction) -- a check against the separately pinned tensor path;
* free stream, conservation and order n+1 convergence on the density wave;
* the oscillation sensor's "high" modes are those with l_x + l_y + l_z = n (A-12).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2208_11131_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_mode_counts_match_paper():
    for n in range(0, 8):
        assert oracle.lib().or_num_modes(2, n, 1) == (n + 1) * (n + 2) // 2
        assert len(inputs.mode_exponents(2, n, 1)) == (n + 1) * (n + 2) // 2
    # Sec. 8.3: words = (3 + d + f_t) N3D(n) Nc^3 with N3D the oracle's 3-D total-degree count
    units = {"MB": 2**20, "GB": 2**30, "TB": 2**40}
    rows = [l.split() for l in open(os.path.join(GOLDEN, "memory_table.txt")) if l.strip() and l[0] != "#"]
    checked = 0
    for nc, deg, val, unit in rows:
        nc, deg = int(nc), int(deg)
        if deg > 7:
            continue
        n3d = oracle.lib().or_num_modes(3, deg, 1)
        words = (3 + 3 + oracle.rk_stages(deg)) * n3d * nc**3
        assert abs(words * 8 - float(val) * units[unit]) / (float(val) * units[unit]) < 5e-4
        checked += 1
    assert checked == 8


@pytest.mark.parametrize("dim,n", [(2, 2), (2, 4), (3, 2), (3, 3)])
def test_projection_exact_for_total_degree_polynomials(dim, n):
    rng = np.random.default_rng(dim * 10 + n)
    ex = inputs.mode_exponents(dim, n, 1)
    coef = rng.normal(size=len(ex))

    def poly(X):
        return sum(c * np.prod(X ** e[None, :dim], axis=1) for c, e in zip(coef, ex))
    P = oracle.Problem(dim=dim, n=n, N=(3, 2, 2)[:dim], hi=(0.9, 1.2, 0.7)[:dim], basis=1)
    w = oracle.project(P, lambda X: np.stack([poly(X)] * (dim + 2)))
    assert w.shape == (dim + 2, P.ncell, len(ex))
    rng2 = np.random.default_rng(1)
    xi = rng2.uniform(-1, 1, (17, dim))
    vals = oracle.evaluate(P, w[:1], xi)[0]  # [ncell, pts]
    X = P.cell_centres()[:, None, :] + 0.5 * np.array(P.h) * xi[None]
    assert np.allclose(vals, poly(X.reshape(-1, dim)).reshape(P.ncell, -1), atol=1e-12, rtol=1e-12)


def _embed(w_td, dim, n):
    """total-degree modes placed at their tensor positions, zeros elsewhere"""
    ex_t = inputs.mode_exponents(dim, n, 0)
    keep = ex_t.sum(1) <= n
    out = np.zeros(w_td.shape[:2] + (len(ex_t),))
    out[:, :, keep] = w_td
    return out, keep


@pytest.mark.parametrize("dim,n,nu,av,tr", [(2, 1, 0.0, 0, 0), (2, 3, 1e-3, 1, 0), (2, 4, 0.0, 1, 1),
                                           (3, 2, 1e-3, 1, 0), (3, 3, 0.0, 0, 1)])
def test_rhs_equals_tensor_rhs_restricted(dim, n, nu, av, tr):
    N = (5, 4, 3)[:dim] + (1,) * (3 - dim)
    wl = inputs.Workload("td", dim, n, N, (0, 0, 0), (1.0, 1.3, 0.8), gamma=1.4, nu=nu, kappa=nu, av_on=av,
                         tracer_on=tr, eta=2e-3 if tr else 0.0, basis=1)
    w = inputs.random_modal_state(wl, seed=9 + n)
    kw = dict(dim=dim, n=n, N=N[:dim], hi=(1.0, 1.3, 0.8)[:dim], gamma=1.4, nu=nu, kappa=nu, av_on=av,
              tracer_on=tr, eta=wl.eta)
    Ptd = oracle.Problem(basis=1, **kw)
    Pt = oracle.Problem(basis=0, **kw)
    r_td, st = oracle.rhs(Ptd, w)
    assert st == 0
    we, keep = _embed(w, dim, n)
    r_t, st = oracle.rhs(Pt, we)
    assert st == 0
    scale = np.abs(r_t).reshape(r_t.shape[0], -1).max(1)[:, None, None]
    assert np.all(np.abs(r_td - r_t[:, :, keep]) <= 1e-12 * scale)


@pytest.mark.parametrize("dim,n", [(2, 3), (3, 2)])
def test_free_stream_and_conservation(dim, n):
    g = 1.4
    P = oracle.Problem(dim=dim, n=n, N=(4, 3, 3)[:dim], hi=(1.0, 1.5, 0.8)[:dim], gamma=g, nu=1e-3, kappa=1e-3,
                       av_on=1, basis=1)
    w = np.zeros(P.shape())
    v = np.array([0.4, -0.2, 0.3])[:dim]
    w[:dim + 2, :, 0] = np.concatenate([[1.2], 1.2 * v, [0.9 / (g - 1) + 0.5 * 1.2 * v @ v]])[:, None]
    r, st = oracle.rhs(P, w)
    assert st == 0 and np.abs(r[:dim + 2]).max() < 1e-13
    wl = inputs.Workload("td", dim, n, (4, 3, 3)[:dim] + (1,) * (3 - dim), (0, 0, 0), (1.0, 1.5, 0.8),
                         gamma=g, nu=1e-3, kappa=1e-3, av_on=1, basis=1)
    w = inputs.random_modal_state(wl, seed=2)
    r, st = oracle.rhs(P, w)
    vol = np.prod(P.h)
    for f in range(dim + 2):
        assert abs(vol * r[f, :, 0].sum()) < 1e-13 * vol * np.abs(r[f, :, 0]).sum()


@pytest.mark.parametrize("n", [1, 2, 3])
def test_density_wave_order(n):
    T = 0.05
    errs = []
    for N in (8, 16):
        wl = inputs.c1_density_wave(N=N, n=n).with_(basis=1)
        P = oracle.Problem(dim=2, n=n, N=(N, N), gamma=wl.gamma, cfl=0.3, basis=1)
        s = oracle.Sim(P, oracle.project(P, inputs.density_wave_ic(wl, 0.0)))
        while s.t < T - 1e-14:
            dt, _ = oracle.max_dt(P, s.w)
            s.step(min(dt, T - s.t))
        errs.append(oracle.l1_error(P, s.w, inputs.density_wave_ic(wl, T)))
    slope = math.log2(errs[0] / errs[1])
    assert n + 1 - 0.4 < slope < n + 1 + 0.6, (errs, slope)


def test_sensor_high_modes_are_total_degree_n():
    n = 3
    P = oracle.Problem(dim=2, n=n, N=(3, 1), basis=1)
    ex = inputs.mode_exponents(2, n, 1)
    for k, e in enumerate(ex):
        if k == 0:
            continue
        w = np.zeros(P.shape())
        w[0, :, 0] = 1.0
        w[0, :, k] = 0.5
        S = oracle.sensor(P, w)
        expect = 0.25 / 1.25 if e.sum() == n else 0.0
        assert np.allclose(S, expect, atol=1e-15), (e, S)
