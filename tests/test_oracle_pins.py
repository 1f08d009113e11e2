"""Pins of the oracle's building blocks against closed forms, textbook values,
invariants and the paper's printed numbers (CPU only).

Each test names the passage of arXiv 2208.11131 (or the mathematics) it rests on.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import riemann
from paper_2208_11131_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Gauss rule (Sec. 2.4)

def test_gauss_two_point_closed_form():
    x, w = oracle.gauss(2)
    assert np.allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=3e-16, rtol=0)
    assert np.allclose(w, [1.0, 1.0], atol=1e-15, rtol=0)


@pytest.mark.parametrize("q", range(1, 9))
def test_gauss_exact_to_degree_2q_minus_1(q):
    x, w = oracle.gauss(q)
    for k in range(2 * q):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x**k) - exact) < 1e-14
    # and not exact one degree higher (the rule is exactly of degree 2q-1)
    k = 2 * q
    assert abs(np.dot(w, x**k) - 2.0 / (k + 1)) > 1e-8


# ---------------------------------------------------------------- scaled Legendre basis (Sec. 2.3)

def test_scaled_legendre_closed_forms():
    for x in np.linspace(-1, 1, 7):
        assert abs(oracle.pt(0, x) - 1.0) < 1e-15
        assert abs(oracle.pt(1, x) - math.sqrt(3) * x) < 1e-15
        assert abs(oracle.pt(2, x) - math.sqrt(5) * (1.5 * x * x - 0.5)) < 1e-14
        assert abs(oracle.pt(3, x) - math.sqrt(7) * (2.5 * x**3 - 1.5 * x)) < 1e-14
        assert abs(oracle.dpt(2, x) - math.sqrt(5) * 3 * x) < 1e-14
        assert abs(oracle.dpt(3, x) - math.sqrt(7) * (7.5 * x * x - 1.5)) < 1e-13


def test_basis_gram_is_twice_identity():
    """int_{-1}^{1} Pt_l Pt_m = 2 delta (Sec. 2.3), so (1/|K|) int phi_l phi_m = delta."""
    x, w = oracle.gauss(12)
    for n in range(0, 8):
        B = np.array([[oracle.pt(l, xi) for l in range(n + 1)] for xi in x])
        assert np.allclose(B.T @ (w[:, None] * B), 2 * np.eye(n + 1), atol=1e-13)


@pytest.mark.parametrize("dim,n", [(2, 0), (2, 2), (2, 4), (3, 1), (3, 3)])
def test_projection_round_trip_of_tensor_polynomials(dim, n):
    """(a) projection of a polynomial of degree <= n per axis is exact; evaluation gives it back."""
    rng = np.random.default_rng(1)
    coef = rng.normal(size=(n + 1,) * dim)

    def poly(X):
        v = np.zeros(X.shape[0])
        for idx in np.ndindex(*coef.shape):
            term = coef[idx] * np.ones(X.shape[0])
            for a in range(dim):
                term = term * X[:, a] ** idx[a]
            v += term
        return v

    P = oracle.Problem(dim=dim, n=n, N=(3, 2, 2)[:dim], hi=(1.0, 0.7, 1.3)[:dim])
    w = oracle.project(P, lambda X: np.stack([poly(X)] * (dim + 2)))
    xi = rng.uniform(-1, 1, size=(11, dim))
    vals = oracle.evaluate(P, w, xi)[0]
    xc = P.cell_centres()
    X = xc[:, None, :] + 0.5 * np.array(P.h)[None, None, :] * xi[None, :, :]
    ref = poly(X.reshape(-1, dim)).reshape(P.ncell, -1)
    assert np.abs(vals - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    assert oracle.l1_error(P, w, lambda X: np.stack([poly(X)] * (dim + 2))) < 1e-13


def test_cell_mean_is_mode_zero():
    P = oracle.Problem(dim=2, n=3, N=(4, 4))
    w = oracle.project(P, lambda X: np.stack([np.exp(np.sin(6 * X[:, 0]) + X[:, 1])] * 4), q=12)
    # w_0 = (1/|K|) int u: compare with a fine Gauss rule average
    x, g = oracle.gauss(12)
    xc = P.cell_centres()[5]
    h = P.h
    tot = 0.0
    for i in range(12):
        for j in range(12):
            X = np.array([[xc[0] + 0.5 * h[0] * x[i], xc[1] + 0.5 * h[1] * x[j]]])
            tot += g[i] * g[j] * np.exp(np.sin(6 * X[0, 0]) + X[0, 1]) / 4
    assert abs(w[0, 5, 0] - tot) < 1e-14


# ---------------------------------------------------------------- interface recovery (Sec. 3.2)

def test_recovery_piecewise_constant_gradient_closed_form():
    """n=0, f=3/4: the recovered gradient of piecewise constants is (u+ - u-)/h n (Sec. 3.2)."""
    P = oracle.Problem(dim=2, n=0, N=(2, 1), hi=(0.8, 0.3))
    w = np.zeros(P.shape())
    w[:, 0, 0] = [1.0, 0.2, -0.1, 3.0]
    w[:, 1, 0] = [1.6, -0.4, 0.5, 2.1]
    ut, gt = oracle.face_recovery(P, w, 0, 1, 0)
    h = P.h[0]
    assert np.allclose(gt[:, 0, :], (w[:, 1, 0] - w[:, 0, 0]) / h, atol=1e-14, rtol=0)
    assert np.allclose(gt[:, 1, :], 0.0, atol=1e-14)
    assert np.allclose(ut, 0.5 * (w[:, 1, 0] + w[:, 0, 0]), atol=1e-14)


@pytest.mark.parametrize("dim,n,axis", [(2, 1, 0), (2, 2, 1), (2, 3, 0), (2, 4, 1), (3, 2, 2), (3, 3, 1)])
def test_recovery_exact_for_global_polynomials(dim, n, axis):
    """a polynomial of degree <= n per axis spanning both cells is recovered exactly, with its gradient."""
    rng = np.random.default_rng(7 + n)
    coef = rng.normal(size=(n + 1,) * dim)

    def poly(X, grad_axis=None):
        v = np.zeros(X.shape[0])
        for idx in np.ndindex(*coef.shape):
            term = coef[idx] * np.ones(X.shape[0])
            for a in range(dim):
                if a == grad_axis:
                    term = term * (idx[a] * X[:, a] ** max(idx[a] - 1, 0))
                else:
                    term = term * X[:, a] ** idx[a]
            v += term
        return v

    N = [1] * dim
    N[axis] = 2
    hi = [0.9, 1.1, 0.6][:dim]
    P = oracle.Problem(dim=dim, n=n, N=tuple(N), hi=tuple(hi))
    w = oracle.project(P, lambda X: np.stack([poly(X)] * (dim + 2)))
    ut, gt = oracle.face_recovery(P, w, 0, 1, axis)
    # face points: x_axis = h_axis, transverse at the Gauss nodes of each transverse cell
    x, _ = oracle.gauss(n + 1)
    ta = [a for a in range(dim) if a != axis]
    pts = []
    for k in range((n + 1) ** (dim - 1)):
        kk = [(k // (n + 1) ** i) % (n + 1) for i in range(dim - 1)]
        X = np.zeros(dim)
        X[axis] = P.h[axis]
        for i, a in enumerate(ta):
            X[a] = 0.5 * P.h[a] * (1 + x[kk[i]])
        pts.append(X)
    pts = np.array(pts)
    scale = max(1.0, np.abs(coef).sum())
    assert np.abs(ut[:, 0] - poly(pts)).max() < 1e-12 * scale
    for a in range(dim):
        assert np.abs(gt[:, a, 0] - poly(pts, grad_axis=a)).max() < 1e-10 * scale


@pytest.mark.parametrize("n", range(0, 7))
def test_recovery_overlap_mirror_symmetry(n):
    """mirror x -> -x maps the left overlap integral onto the right one: A+_ml = (-1)^(m+l) A-_ml."""
    Am, Ap, f = oracle.recovery_matrices(n)
    assert f == (0.75 if n <= 2 else 1.0)  # Sec. 3.2 choice of the overlap fraction
    sgn = (-1.0) ** (np.arange(n + 1)[:, None] + np.arange(n + 2)[None, :])
    assert np.allclose(Ap, sgn * Am, atol=1e-14)


def test_recovery_f1_reproduces_cell_data():
    """f=1: K* is the union of both cells, so projecting the joint degree-(n+1) polynomial back onto a
    single-cell constant reproduces the cell means: (A-^T)_0 column gives each cell half the weight."""
    for n in range(0, 6):
        Am, Ap, _ = oracle.recovery_matrices(n, 1.0)
        # q_0 = (w0- + w0+)/2 when f = 1 (mean over the union of the two cells)
        assert abs(0.5 * Am[0, 0] - 0.5) < 1e-14 and abs(0.5 * Ap[0, 0] - 0.5) < 1e-14
        assert np.allclose(Am[1:, 0], 0.0, atol=1e-14)


# ---------------------------------------------------------------- HLLC (Sec. 2.2) and Euler flux (Eq. flux_matrix)

def _cons(g, rho, v, p):
    v = np.asarray(v, dtype=float)
    return np.concatenate([[rho], rho * v, [p / (g - 1) + 0.5 * rho * v @ v]])


def _euler_flux(g, u, ax):
    d = len(u) - 2
    rho = u[0]
    v = u[1:1 + d] / rho
    p = (g - 1) * (u[-1] - 0.5 * rho * v @ v)
    F = np.zeros(d + 2)
    F[0] = rho * v[ax]
    F[1:1 + d] = rho * v[ax] * v
    F[1 + ax] += p
    F[-1] = (u[-1] + p) * v[ax]
    return F


@pytest.mark.parametrize("dim", [2, 3])
def test_hllc_consistency(dim):
    rng = np.random.default_rng(3)
    g = 1.4
    for _ in range(20):
        u = _cons(g, rng.uniform(0.2, 2), rng.uniform(-2, 2, dim), rng.uniform(0.1, 3))
        for ax in range(dim):
            F, st = oracle.hllc(dim, ax, g, u, u)
            assert st == 0
            assert np.allclose(F, _euler_flux(g, u, ax), rtol=1e-13, atol=1e-13)


def test_hllc_resolves_isolated_contact():
    g = 5 / 3
    for v in (0.4, -0.7):
        uL = _cons(g, 1.0, [v, 0.3], 2.0)
        uR = _cons(g, 0.25, [v, -0.5], 2.0)
        F, _ = oracle.hllc(2, 0, g, uL, uR)
        upwind = uL if v > 0 else uR
        assert np.allclose(F, _euler_flux(g, upwind, 0), rtol=1e-13, atol=1e-13)


def test_hllc_supersonic_upwinding():
    g = 1.4
    uL = _cons(g, 1.0, [5.0, 0.1, 0.2], 1.0)
    uR = _cons(g, 0.5, [4.5, -0.3, 0.0], 0.8)
    F, _ = oracle.hllc(3, 0, g, uL, uR)
    assert np.allclose(F, _euler_flux(g, uL, 0), rtol=1e-14)
    F, _ = oracle.hllc(3, 0, g, _cons(g, 1, [-5, 0, 0], 1), _cons(g, 2, [-6, 0, 0], 1))
    assert np.allclose(F, _euler_flux(g, _cons(g, 2, [-6, 0, 0], 1), 0), rtol=1e-14)


def test_hllc_rotation_and_mirror_invariance():
    g = 1.4
    rng = np.random.default_rng(5)
    for _ in range(10):
        uL = _cons(g, rng.uniform(0.5, 2), rng.uniform(-1, 1, 2), rng.uniform(0.5, 2))
        uR = _cons(g, rng.uniform(0.5, 2), rng.uniform(-1, 1, 2), rng.uniform(0.5, 2))
        Fx, _ = oracle.hllc(2, 0, g, uL, uR)
        sw = lambda u: u[[0, 2, 1, 3]]
        Fy, _ = oracle.hllc(2, 1, g, sw(uL), sw(uR))
        assert np.allclose(Fx, sw(Fy), rtol=1e-13, atol=1e-14)
        mir = lambda u: u * np.array([1, -1, 1, 1])
        Fm, _ = oracle.hllc(2, 0, g, mir(uR), mir(uL))
        assert np.allclose(Fx, -mir(Fm), rtol=1e-13, atol=1e-14)


# ---------------------------------------------------------------- Navier-Stokes flux (Sec. 3.3)

def test_ns_stress_is_trace_free_and_vanishes_for_dilatation():
    """zero bulk viscosity: a pure dilatation grad v = a I gives Pi = 0; Pi is symmetric and trace free."""
    g, nu = 1.4, 0.3
    rho, v = 1.7, np.array([0.2, -0.1, 0.4])
    u = _cons(g, rho, v, 1.0)
    a = 0.37
    grad = np.zeros((3, 5))
    for b in range(3):
        grad[b, 1 + b] = rho * a  # d(rho v_b)/dx_b with rho uniform
    for ax in range(3):
        F, _ = oracle.ns_flux(3, ax, g, nu, 0.0, u, grad)
        assert np.allclose(F[1:4], 0.0, atol=1e-15)
    rng = np.random.default_rng(2)
    grad = rng.normal(size=(3, 5))
    Pi = np.array([oracle.ns_flux(3, ax, g, nu, 0.0, u, grad)[0][1:4] for ax in range(3)])
    assert np.allclose(Pi, Pi.T, atol=1e-14)
    assert abs(np.trace(Pi)) < 1e-14


def test_ns_simple_shear_and_heat_flux_closed_forms():
    """v_x(y) shear: Pi_xy = nu rho dv_x/dy; at rest with uniform rho the heat flux of Sec. 3.3,
    chi (gamma-1) rho grad u_int, reduces to chi grad p."""
    g, nu, chi = 5 / 3, 0.02, 0.05
    rho = 1.3
    u = _cons(g, rho, [0.0, 0.0], 2.0)
    grad = np.zeros((2, 4))
    grad[1, 1] = rho * 0.8  # d(rho v_x)/dy, rho uniform -> dv_x/dy = 0.8
    F, _ = oracle.ns_flux(2, 1, g, nu, 0.0, u, grad)
    assert abs(F[1] - nu * rho * 0.8) < 1e-15 and abs(F[2]) < 1e-15
    grad = np.zeros((2, 4))
    grad[0, 3] = 0.9  # de/dx at rest, rho uniform -> dp/dx = (g-1) 0.9
    F, _ = oracle.ns_flux(2, 0, g, 0.0, chi, u, grad)
    assert abs(F[3] - chi * (g - 1) * 0.9) < 1e-15


# ---------------------------------------------------------------- oscillation sensor (Eq. discontinuity_sensor2)

def test_sensor_closed_forms():
    for dim, n in [(2, 1), (2, 3), (3, 2)]:
        P = oracle.Problem(dim=dim, n=n, N=(2,) * dim)
        w = np.zeros(P.shape())
        rng = np.random.default_rng(n)
        M = P.M
        midx = np.array([[(l // (n + 1) ** a) % (n + 1) for a in range(dim)] for l in range(M)])
        top = midx.max(1) == n
        # cell 0: degree-(n-1) data only -> S = 0
        w[0, 0, ~top] = rng.normal(size=(~top).sum())
        # cell 1: a single top mode -> S = 1
        w[0, 1, np.nonzero(top)[0][0]] = 0.3
        # cell 2: known mixture
        w[0, 2, 0] = 2.0
        w[0, 2, np.nonzero(top)[0][-1]] = 1.0
        # cell 3: zero density data -> S = 0 by definition
        S = oracle.sensor(P, w)
        assert S[0] == 0.0 and abs(S[1] - 1.0) < 1e-15 and abs(S[2] - 0.2) < 1e-15 and S[3] == 0.0
        w = rng.normal(size=P.shape())
        S = oracle.sensor(P, w)
        assert np.all((S >= 0) & (S <= 1))
    P = oracle.Problem(dim=2, n=0, N=(2, 2))
    assert np.all(oracle.sensor(P, np.ones(P.shape())) == 0.0)


# ---------------------------------------------------------------- SSP Runge-Kutta (Sec. 2.5)

def _butcher(stages):
    al, be = oracle.rk_table(stages)
    A = np.zeros((stages + 1, stages + 1))
    for i in range(1, stages + 1):
        assert abs(al[i, :i].sum() - 1.0) < 1e-14  # convex combination
        assert np.all(al[i] >= 0) and np.all(be[i] >= 0)  # SSP: non-negative coefficients
        for k in range(i):
            A[i] += al[i, k] * A[k]
            A[i, k] += be[i, k]
    return A[stages, :stages], A[:stages, :stages]


@pytest.mark.parametrize("stages,order", [(1, 1), (2, 2), (3, 3), (5, 4)])
def test_rk_order_conditions(stages, order):
    b, A = _butcher(stages)
    c = A.sum(1)
    conds = [(b.sum(), 1.0)]
    if order >= 2:
        conds += [(b @ c, 0.5)]
    if order >= 3:
        conds += [(b @ c**2, 1 / 3), (b @ A @ c, 1 / 6)]
    if order >= 4:
        conds += [(b @ c**3, 1 / 4), (b @ (c * (A @ c)), 1 / 8), (b @ A @ c**2, 1 / 12), (b @ A @ A @ c, 1 / 24)]
    for v, t in conds:
        assert abs(v - t) < 1e-14


def test_rk_stage_rule_reproduces_paper_memory_table():
    """Sec. 8.3: words = (3 + d + f_t(p)) N3D(n) Nc^3; f_t is the stage count of the SSP scheme
    (P stages for P = n+1 <= 3, else 5).  The printed table pins that rule (d = 3, 8-byte words)."""
    units = {"MB": 2**20, "GB": 2**30, "TB": 2**40}
    rows = [l.split() for l in open(os.path.join(GOLDEN, "memory_table.txt")) if l.strip() and l[0] != "#"]
    for nc, deg, val, unit in rows:
        nc, deg = int(nc), int(deg)
        n3d = (deg + 1) * (deg + 2) * (deg + 3) // 6
        words = (3 + 3 + oracle.rk_stages(deg)) * n3d * nc**3
        printed = float(val) * units[unit]
        assert abs(words * 8 - printed) / printed < 5e-4, (nc, deg)


# ---------------------------------------------------------------- time step (Eq. timestep)

@pytest.mark.parametrize("dim,n", [(2, 0), (2, 2), (3, 3)])
def test_max_dt_uniform_state_closed_form(dim, n):
    g = 1.4
    P = oracle.Problem(dim=dim, n=n, N=(5, 3, 2)[:dim], hi=(1.0, 0.45, 0.8)[:dim], gamma=g, cfl=0.3)
    v = np.array([0.3, -0.4, 0.12])[:dim]
    w = np.zeros(P.shape())
    w[:, :, 0] = _cons(g, 1.3, v, 0.7)[:, None]
    dt, st = oracle.max_dt(P, w)
    cs = math.sqrt(g * 0.7 / 1.3)
    hmin = min(P.h)
    assert st == 0
    assert abs(dt - 0.3 * hmin / (2 * (n + 1) * (cs + np.linalg.norm(v)))) < 1e-15


# ---------------------------------------------------------------- positivity limiter (Sec. 4.2)

def test_positivity_limiter_properties():
    g = 1.4
    P = oracle.Problem(dim=2, n=3, N=(3, 3), gamma=g)
    rng = np.random.default_rng(11)
    # smooth data: limiter is the identity
    w = oracle.project(P, lambda X: np.stack([1 + 0.1 * np.sin(6 * X[:, 0]), 0 * X[:, 0], 0 * X[:, 0],
                                              2.5 + 0 * X[:, 0]]))
    w0 = w.copy()
    assert oracle.positivity(P, w) == 0
    assert np.array_equal(w, w0)
    # strongly oscillating density with negative point values: limited, means unchanged
    w = w0.copy()
    w[0, :, 1:] += rng.normal(scale=0.8, size=w[0, :, 1:].shape)
    w[3, :, 1:] += rng.normal(scale=2.0, size=w[3, :, 1:].shape)
    means = w[:, :, 0].copy()
    assert oracle.positivity(P, w) == 0
    assert np.array_equal(w[:, :, 0], means)
    x, _ = oracle.gauss(4)
    pts = [(a, b) for a in x for b in x] + [(s, b) for s in (-1, 1) for b in x] + [(b, s) for s in (-1, 1) for b in x]
    vals = oracle.evaluate(P, w, np.array(pts))
    rho = vals[0]
    p = (g - 1) * (vals[3] - 0.5 * (vals[1] ** 2 + vals[2] ** 2) / rho)
    # limited to the floors up to rounding of the cell mean
    assert np.all(rho >= (1e-6 - 1e-12) * means[0][:, None])
    pm = (g - 1) * (means[3] - 0.5 * (means[1] ** 2 + means[2] ** 2) / means[0])
    assert np.all(p >= (1e-6 - 1e-10) * pm[:, None])
    assert np.any(w[0, :, 1:] != w0[0, :, 1:])


# ---------------------------------------------------------------- exact Riemann solver (textbook)

def test_exact_riemann_sod_star_state_textbook_values():
    vals = [l.split() for l in open(os.path.join(GOLDEN, "sod_star.txt")) if l.strip() and l[0] != "#"][0]
    ps, us, rl, rr = map(float, vals)
    p, u = riemann.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
    assert abs(p - ps) < 5e-6 and abs(u - us) < 5e-6
    r, _, _ = riemann.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4, [u - 1e-9, u + 1e-9])
    assert abs(r[0] - rl) < 5e-6 and abs(r[1] - rr) < 5e-6


def test_exact_riemann_rankine_hugoniot_across_shock():
    g = 1.4
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    ps, us = riemann.star_state(left, right, g)
    r2 = riemann.sample(left, right, g, [us + 1e-9])[0][0]
    # shock speed from mass conservation, then momentum and energy jumps must match
    rR, uR, pR = right
    S = (r2 * us - rR * uR) / (r2 - rR)
    mom = lambda r, u, p: r * u * u + p
    ene = lambda r, u, p: (p / (g - 1) + 0.5 * r * u * u + p) * u
    E = lambda r, u, p: p / (g - 1) + 0.5 * r * u * u
    assert abs((mom(r2, us, ps) - mom(*right)) - S * (r2 * us - rR * uR)) < 1e-12
    assert abs((ene(r2, us, ps) - ene(*right)) - S * (E(r2, us, ps) - E(*right))) < 1e-12


def test_av_defaults_golden():
    vals = dict(l.split() for l in open(os.path.join(GOLDEN, "av_defaults.txt")) if l.strip() and l[0] != "#")
    P = oracle.Problem(dim=2, n=1, N=(1, 1))
    assert (P.av_scale, P.f_v, P.f_tau, P.f_w, P.s_onset) == tuple(
        float(vals[k]) for k in ("av_scale", "f_v", "f_tau", "f_w", "s_onset"))
    assert P.cfl == float(vals["cfl"])


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_recovery_is_the_l2_projection_of_discontinuous_data(n):
    """Sec. 3.2 by brute force: the L2 projection of the two cells' (discontinuous, random) data
    onto Legendre polynomials of degree n+1 on K* (f h on each side), by dense Gauss quadrature split
    at the interface, gives the recovered value and normal derivative at the interface."""
    from numpy.polynomial import legendre as L
    rng = np.random.default_rng(30 + n)
    hx, hy = 0.7, 0.4
    P = oracle.Problem(dim=2, n=n, N=(2, 1), hi=(2 * hx, hy))
    w = rng.normal(size=P.shape())
    ut, gt = oracle.face_recovery(P, w, 0, 1, 0)
    f = 0.75 if n <= 2 else 1.0
    Q = n + 1
    yg, _ = L.leggauss(Q)
    xq, wq = L.leggauss(60)
    Pt = lambda l, x: math.sqrt(2 * l + 1) * L.legval(x, [0] * l + [1])
    sl, sr = 0.5 * (xq - 1), 0.5 * (xq + 1)  # K* coordinate on [-1,0] and [0,1]
    for k in range(Q):
        for fld in range(P.dim + 2):
            def side(c, xi):
                return sum(w[fld, c, lx + Q * ly] * Pt(lx, xi) * Pt(ly, yg[k]) for ly in range(Q) for lx in range(Q))
            # physical offset from the interface x = s f hx: cell 0 at xi = 1 + 2 f s, cell 1 at xi = -1 + 2 f s
            q = []
            for l in range(n + 2):
                Pl = L.legval(sl, [0] * l + [1]), L.legval(sr, [0] * l + [1])
                integ = 0.5 * np.sum(wq * side(0, 1 + 2 * f * sl) * Pl[0]) + 0.5 * np.sum(wq * side(1, -1 + 2 * f * sr) * Pl[1])
                q.append(integ * (2 * l + 1) / 2)
            assert abs(L.legval(0.0, q) - ut[k, fld]) < 1e-12
            assert abs(L.legval(0.0, L.legder(q)) / (f * hx) - gt[k, 0, fld]) < 1e-11


@pytest.mark.parametrize("dim,n,N", [(2, 3, (1, 1)), (2, 2, (7, 1)), (2, 3, (1, 5)), (3, 2, (1, 2, 3))])
def test_periodic_degenerate_grids_conserve(dim, n, N):
    """one cell along an axis of a periodic grid: the cell is its own neighbour, every face flux
    still leaves one cell and enters another (here the same one), so the cell-mean right-hand sides
    of the conserved fields sum to zero (Sec. 3, manifest conservation), and a uniform state is a
    steady state"""
    P = oracle.Problem(dim=dim, n=n, N=N, hi=(1.0, 0.7, 0.9)[:dim], gamma=1.4, nu=1e-3, kappa=1e-3, av_on=1)
    Nf = tuple(N) + (1,) * (3 - dim)
    wl = inputs.Workload("deg", dim, n, Nf, (0, 0, 0), (1.0, 0.7, 0.9), gamma=1.4, nu=1e-3, kappa=1e-3, av_on=1)
    w = inputs.random_modal_state(wl, seed=3)
    r, st = oracle.rhs(P, w)
    assert st == 0
    for f in range(dim + 2):
        assert abs(r[f, :, 0].sum()) < 1e-13 * max(1.0, np.abs(r[f]).max())
    u = np.zeros_like(w)
    v = np.array([0.3, -0.2, 0.1])[:dim]
    u[0, :, 0] = 1.1
    u[1:dim + 1, :, 0] = (1.1 * v)[:, None]
    u[dim + 1, :, 0] = 1.0 / 0.4 + 0.5 * 1.1 * v @ v
    r0, st = oracle.rhs(P, u)
    assert st == 0 and np.abs(r0[:dim + 2]).max() < 1e-13


def test_wiggle_source_closed_form():
    """Sec. 4.1 wiggle term of the alpha source, one value per cell per step: f_w max(0, d ln S / dt)
    where the sensor S exceeds s_onset / P^2, else 0, with d ln S / dt the difference of ln S between
    the starts of this and the previous step over the previous step's dt (S floored at
    1e-4 s_onset / P^2), and zero at the first step.  Each cell carries one top density mode of
    amplitude a on a unit mean, so S = a^2 / (1 + a^2) exactly."""
    n, g = 3, 1.4
    P = n + 1
    prob = oracle.Problem(dim=2, n=n, N=(7, 1), gamma=g, av_on=1)
    s_on = prob.s_onset / P**2
    floor = 1e-4 * s_on
    # above the onset and growing / shrinking; growing below the onset; a floored history; below the
    # floor; unchanged; between s_onset / P^2 and s_onset (on only with the 1 / P^2)
    a = np.array([0.1, 0.1, 1e-3, 0.02, 1e-6, 0.05, 0.005])
    S = a**2 / (1 + a**2)
    assert s_on < S[6] < prob.s_onset
    S_prev = np.array([S[0] / 2, 2 * S[1], S[2] / 10, 1e-14, 1e-20, S[5], S[6] / 3])
    w = np.zeros(prob.shape())
    w[0, :, 0] = 1.0
    w[0, :, n] = a  # mode (l_x, l_y) = (n, 0)
    w[3, :, 0] = 1.0 / (g - 1)  # at rest, p = 1
    dt_prev = 0.01
    expect = np.where(S > s_on, prob.f_w * np.maximum(0.0, (np.log(np.maximum(S, floor)) -
                                                           np.log(np.maximum(S_prev, floor))) / dt_prev), 0.0)
    assert expect[0] > 0 and expect[3] > 0 and expect[6] > 0 and not np.any(expect[[1, 2, 4, 5]])
    sim = oracle.Sim(prob, w, S_prev=S_prev.copy(), scal=np.array([dt_prev, 1.0, 0.0]))
    _, st = sim.step(1e-9)
    assert st == 0
    assert np.allclose(sim.wig, expect, rtol=1e-12, atol=0.0)
    assert np.allclose(sim.S_prev, S, rtol=1e-13, atol=0.0)  # the history now holds this step's sensor
    first = oracle.Sim(prob, w, S_prev=S_prev.copy(), scal=np.array([0.0, 0.0, 0.0]))
    _, st = first.step(1e-9)
    assert st == 0 and not np.any(first.wig)


def test_artificial_viscosity_diffuses_a_density_wave_at_rest():
    """Sec. 4.1 artificial viscosity alone: gas at rest at uniform pressure carrying a small density
    sine along x, with alpha = 1.  Every face sees a stationary contact, which HLLC returns exactly
    (no mass or energy flux, the same pressure on both sides), so the only flux is eps grad u with
    eps = av_scale clip(alpha, 0, 1) c_s h / P, h = min_a h_a (here h_x: the cells are twice as tall
    as wide).  The cell-mean density right-hand side is then eps_0 times the cell average of rho''
    (up to O(delta) from the variation of c_s and the recovery error, which falls with h), and
    momentum and energy do not change."""
    g, delta, n = 1.4, 1e-5, 3
    errs = []
    for N in (8, 16, 32):
        P = oracle.Problem(dim=2, n=n, N=(N, N), hi=(1.0, 2.0), gamma=g, av_on=1)

        def ic(X):
            one = np.ones(len(X))
            return np.stack([1 + delta * np.sin(2 * np.pi * X[:, 0]), 0 * one, 0 * one, one / (g - 1), one])
        w = oracle.project(P, ic)
        r, st = oracle.rhs(P, w)
        assert st == 0
        h = 1.0 / N
        eps0 = P.av_scale * np.sqrt(g) * h / (n + 1)  # c_s = sqrt(gamma p / rho) = sqrt(gamma)
        xc = P.cell_centres()[:, 0]
        avg_rho2 = -(2 * np.pi) * delta * (np.cos(2 * np.pi * (xc - h / 2)) - np.cos(2 * np.pi * (xc + h / 2))) / h
        expect = eps0 * avg_rho2
        errs.append(np.abs(r[0, :, 0] - expect).max() / np.abs(expect).max())
        assert np.abs(r[1:4]).max() < 1e-12
    assert errs[1] < 1e-4 and errs[2] < errs[1] / 4 and errs[1] < errs[0] / 4, errs


def test_alpha_compression_source():
    """Sec. 4.1 source of the artificial-viscosity field: f_v max(0, -div v) at every volume node,
    projected with the Gauss rule.  With alpha = 0 (no decay term, no viscosity), no wiggle term and
    the periodic velocity v_x = -a sin 2 pi x (compression where cos 2 pi x > 0), the cell mean of
    the alpha right-hand side is 2^-d sum_j g_j f_v max(0, 2 pi a cos 2 pi x_j); the DG divergence
    at the nodes differs from the exact one by O(h^n)."""
    g, a, n = 1.4, 0.1, 3
    errs = []
    for N in (8, 16, 32):
        P = oracle.Problem(dim=2, n=n, N=(N, N), hi=(1.0, 2.0), gamma=g, av_on=1)

        def ic(X):
            one = np.ones(len(X))
            v = -a * np.sin(2 * np.pi * X[:, 0])
            return np.stack([one, v, 0 * one, one / (g - 1) + 0.5 * v * v, 0 * one])
        w = oracle.project(P, ic)
        r, st = oracle.rhs(P, w)
        assert st == 0
        xg, wg = np.polynomial.legendre.leggauss(n + 1)
        X = P.cell_centres()[:, :1] + 0.5 * P.h[0] * xg[None, :]
        src = P.f_v * np.maximum(0.0, 2 * np.pi * a * np.cos(2 * np.pi * X))
        expect = (src * wg[None, :]).sum(1) / 2.0  # the field is constant in y: the y-rule sums to 2
        errs.append(np.abs(r[4, :, 0] - expect).max() / np.abs(expect).max())
    assert errs[1] < 1e-5 and errs[2] < errs[1] / 8 and errs[1] < errs[0] / 8, errs


def test_outflow_faces_carry_the_physical_flux_of_the_interior_trace():
    """Outflow boundaries (the reading taken where the paper is silent: the ghost trace is the
    interior trace, so the face flux is the physical Euler flux of the interior trace and no
    dissipative flux crosses the boundary).  One cell with outflow at both x faces, varying in x only, Navier-Stokes on: the cell
    mean changes by -(F(u(+1)) - F(u(-1))) / h_x with u(+-1) the cell's own traces (the y faces are
    periodic onto the cell itself and cancel; the volume terms do not reach the cell mean)."""
    g, n, hx = 1.4, 2, 0.5
    P = oracle.Problem(dim=2, n=n, N=(1, 1), hi=(hx, 0.7), bc=(1, 0), gamma=g, nu=1e-2, kappa=1e-2, av_on=0)
    w = np.zeros(P.shape())
    w[0, 0, :3] = (1.0, 0.1, 0.05)  # modes l_x = 0, 1, 2 with l_y = 0
    w[1, 0, :2] = (0.3, 0.05)
    w[2, 0, 0] = 0.1
    w[3, 0, :2] = (2.5, 0.1)
    r, st = oracle.rhs(P, w)
    assert st == 0

    def flux(x):
        u = np.array([sum(w[f, 0, l] * oracle.pt(l, x) for l in range(n + 1)) for f in range(4)])
        rho, mx, my, e = u
        vx, vy = mx / rho, my / rho
        p = (g - 1) * (e - 0.5 * rho * (vx * vx + vy * vy))
        return np.array([mx, mx * vx + p, mx * vy, (e + p) * vx])
    expect = -(flux(1.0) - flux(-1.0)) / hx
    assert np.allclose(r[:4, 0, 0], expect, rtol=1e-13, atol=1e-13), (r[:4, 0, 0], expect)
