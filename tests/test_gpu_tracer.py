"""Passive tracer (Sec. 3.4) on the GPU against the oracle: right-hand side (2-D/3-D, n = 0..4,
with and without diffusion, NS and AV, FP64 and FP32-bulk), whole steps with the limiter, the
Gaussian pulse of Sec. 5.2 step by step and its convergence against the closed form, and the
conservation sums.  Tolerances as in test_gpu_parity."""
import math

import numpy as np
import pytest

import oracle
from paper_2208_11131_gb300 import build as B
from paper_2208_11131_gb300 import dgx, inputs

from .helpers import problem, rel_l1, rhs_err, state_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    dgx.lib()


def _wl(dim, n, N, hi, nu=0.0, av=0, eta=3e-3, lim=0):
    N = tuple(N) + (1,) * (3 - len(N))
    hi = tuple(hi) + (1.0,) * (3 - len(hi))
    return inputs.Workload(f"tr{dim}{n}", dim, n, N, (0.0, 0.0, 0.0), hi, gamma=1.4, nu=nu, kappa=nu, av_on=av,
                           positivity_on=lim, cfl=0.3, tracer_on=1, eta=eta)


def _state(wl, seed):
    """random physical flow with a random tracer concentration field in [0.2, 1]"""
    w = inputs.random_modal_state(wl.with_(tracer_on=0), seed=seed)
    c = inputs.random_modal_state(wl.with_(tracer_on=0, av_on=0), seed=seed + 1)[0]
    c = 0.2 + 0.8 * (c - c[:, 0].min()) / (np.ptp(c[:, 0]) + 1e-12)
    rc = w[0] * 0  # rho c to first order: cell means multiplied, higher modes from c
    rc[:, 0] = w[0, :, 0] * c[:, 0]
    rc[:, 1:] = 0.5 * c[:, 1:]
    d = wl.dim
    return np.ascontiguousarray(np.concatenate([w[:d + 2], rc[None], w[d + 2:]]))


CASES = [
    (2, 0, (7, 5), (1.0, 1.3), 0.0, 0, 3e-3),
    (2, 2, (9, 7), (1.0, 2.0), 0.0, 0, 3e-3),
    (2, 3, (13, 10), (1.0, 2.0), 1e-3, 1, 3e-3),
    (2, 4, (6, 6), (1.0, 1.0), 0.0, 1, 0.0),
    (2, 1, (17, 9), (1.0, 1.0), 1e-3, 0, 0.0),
    (3, 1, (5, 4, 3), (1.0, 1.0, 0.5), 0.0, 1, 3e-3),
    (3, 2, (4, 4, 3), (1.0, 1.0, 1.0), 1e-3, 1, 3e-3),
    (3, 3, (3, 3, 3), (1.0, 1.0, 1.0), 0.0, 0, 3e-3),
]


@pytest.mark.parametrize("prec", [dgx.DG_FP64, dgx.DG_FP32_BULK])
@pytest.mark.parametrize("dim,n,N,hi,nu,av,eta", CASES)
def test_tracer_rhs_parity(dim, n, N, hi, nu, av, eta, prec):
    wl = _wl(dim, n, N, hi, nu, av, eta)
    P = problem(wl)
    w = _state(wl, seed=3 + n)
    ref, st = oracle.rhs(P, w)
    assert st == 0
    sim = dgx.Simulation(wl, precision=prec)
    assert sim.shape == w.shape
    sim.set_state(w)
    out = sim.rhs()
    assert rhs_err(out, ref, P, w) < (1e-13 if prec == dgx.DG_FP64 else 1e-5)
    sim.close()


@pytest.mark.parametrize("prec", [dgx.DG_FP64, dgx.DG_FP32_BULK])
def test_tracer_steps_with_limiter(prec):
    wl = _wl(2, 3, (12, 10), (1.0, 1.0), 1e-3, 1, 2e-3, lim=1)
    P = problem(wl)
    w = _state(wl, seed=21)
    ref = oracle.Sim(P, w)
    sim = dgx.Simulation(wl, precision=prec)
    sim.set_state(w)
    for _ in range(4):
        _, st = ref.step()
        assert st == 0
        sim.step()
    out = sim.get_state()
    if prec == dgx.DG_FP64:
        assert state_err(out, ref.w, P) < 1e-11
    else:
        assert rel_l1(out, ref.w, 0) < 1e-5 and rel_l1(out, ref.w, 4) < 1e-5
    tot = sim.conserved_sums()  # FP64 sums of the cell means, the tracer included
    assert tot.shape == (5,)
    assert abs(tot[4] - np.prod(P.h) * out[4, :, 0].sum()) < 1e-12 * abs(tot[4])
    sim.close()


def test_gaussian_pulse_per_step_parity():
    wl = inputs.gaussian_pulse(N=16, n=3)
    P = problem(wl)
    w0 = inputs.project(wl, inputs.gaussian_pulse_ic(wl, 1.0))
    ref = oracle.Sim(P, w0)
    sim = dgx.Simulation(wl)
    sim.set_state(w0)
    for _ in range(10):
        _, st = ref.step()
        assert st == 0
        sim.step()
        assert state_err(sim.get_state(), ref.w, P) < 1e-12


@pytest.mark.parametrize("prec", [dgx.DG_FP64, dgx.DG_FP32_BULK])
@pytest.mark.parametrize("n,lo,hi", [(1, 1.7, 2.5), (2, 1.8, 2.5), (3, 3.7, 4.6)])
def test_gaussian_pulse_convergence(n, lo, hi, prec):
    """the orders the oracle gives (order 2 at n = 2: the recovery of Sec. 3.2 with the paper's overlap
    fraction f = 3/4 gives 2 there, f = 1 would give 3)"""
    errs = []
    for N in (16, 32):
        wl = inputs.gaussian_pulse(N=N, n=n)
        P = problem(wl)
        sim = dgx.Simulation(wl, precision=prec)
        sim.set_state(inputs.project(wl, inputs.gaussian_pulse_ic(wl, 1.0)))
        t = 0.0
        while t < 0.5 - 1e-14:
            dt = min(sim.max_dt(), 0.5 - t)
            sim.step(dt)
            t += dt
        errs.append(oracle.l1_error(P, sim.get_state(), inputs.gaussian_pulse_ic(wl, 1.5), field=4))
        sim.close()
    slope = math.log2(errs[0] / errs[1])
    assert lo < slope < hi, (errs, slope)


def test_batch_rejects_tracer_members():
    s = dgx.Simulation(_wl(2, 3, (8, 8), (1.0, 1.0), 0.0, 1))
    with pytest.raises(dgx.DGError) as e:
        dgx.dg_batch_create([s.h])
    assert e.value.code == dgx.DG_EUNSUPPORTED
    s.close()
