"""Turbulence driving (Sec. 7.1) on the GPU against the oracle, through the C ABI.

* right-hand side with a given driving state (dg_set_forcing): same tolerances as the undriven
  right-hand side (flux-term scale, FP64 1e-13, FP32-bulk 1e-5), and the driving contribution
  itself must be far above that tolerance so that the comparison tests it;
* whole steps at a fixed dt that crosses several update instants: the update counter equals the
  oracle's exactly, the OU vector agrees to the rounding of log/cos in the normal draws, and the
  state agrees within the step tolerances of the undriven parity tests;
* a restart from dg_get_state / dg_get_aux / dg_get_forcing continues bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2208_11131_gb300 import build as B
from paper_2208_11131_gb300 import dgx, inputs

from .helpers import problem, rel_l1, rhs_err, state_err

pytestmark = pytest.mark.gpu

FP64_RHS_TOL = 1e-13
FP64_STEP_TOL = 1e-11
FP32_RHS_TOL = 1e-5
FP32_L1_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    dgx.lib()


def _wl(dim, n, N, hi, nu=0.0, av=0, amp=0.5, gamma=1.4):
    N = tuple(N) + (1,) * (3 - len(N))
    hi = tuple(hi) + (1.0,) * (3 - len(hi))
    return inputs.Workload(f"f{dim}{n}", dim, n, N, (0.0, 0.0, 0.0), hi, gamma=gamma, nu=nu, kappa=nu, av_on=av,
                           cfl=0.3, forcing_on=1, force_amp=amp, force_ts=0.7, force_dt=0.01, force_seed=77 + n)


CASES = [
    (2, 2, (7, 5), (1.0, 1.5), 0.0, 0),
    (2, 3, (19, 10), (1.0, 2.0), 1e-3, 1),
    (2, 5, (6, 6), (1.0, 1.0), 0.0, 1),
    (3, 1, (5, 4, 3), (1.0, 1.0, 0.5), 0.0, 1),
    (3, 3, (5, 4, 4), (1.0, 1.0, 1.0), 1e-3, 1),
]


@pytest.mark.parametrize("prec", [dgx.DG_FP64, dgx.DG_FP32_BULK])
@pytest.mark.parametrize("dim,n,N,hi,nu,av", CASES)
def test_forced_rhs_parity(dim, n, N, hi, nu, av, prec):
    wl = _wl(dim, n, N, hi, nu, av)
    P = problem(wl)
    w = inputs.random_modal_state(wl, seed=11 + n)
    fst = oracle.forcing_state()
    assert oracle.forcing_update(P, fst, 0.123) == 0  # 12 updates after the initial draw
    ref, st = oracle.rhs(P, w, None, fst)
    assert st == 0
    unforced, _ = oracle.rhs(problem(wl, forcing_on=0), w)
    sim = dgx.Simulation(wl, precision=prec)
    sim.set_state(w)
    sim.set_forcing(fst)
    out = sim.rhs()
    tol = FP64_RHS_TOL if prec == dgx.DG_FP64 else FP32_RHS_TOL
    assert rhs_err(out, ref, P, w) < tol
    assert rhs_err(unforced, ref, P, w) > 1e3 * tol  # the driving term is what is being compared
    assert np.array_equal(sim.get_forcing(), fst)  # dg_rhs does not advance the driving
    sim.close()


@pytest.mark.parametrize("prec", [dgx.DG_FP64, dgx.DG_FP32_BULK])
@pytest.mark.parametrize("dim,n,N,hi,nu,av", [CASES[1], CASES[3], CASES[4]])
def test_forced_steps_parity(dim, n, N, hi, nu, av, prec):
    wl = _wl(dim, n, N, hi, nu, av)
    P = problem(wl)
    w = inputs.random_modal_state(wl, seed=21 + n)
    ref = oracle.Sim(P, w)
    sim = dgx.Simulation(wl, precision=prec)
    sim.set_state(w)
    f0 = sim.get_forcing()
    assert f0[0] == -1 and not np.any(f0[1:])
    dt = 0.0043  # update instants 0.01, 0.02 fall inside steps 3 and 5
    for k in range(6):
        _, st = ref.step(dt)
        assert st == 0
        sim.step(dt)
        fg = sim.get_forcing()
        assert fg[0] == ref.fst[0]
        assert np.abs(fg[1:] - ref.fst[1:]).max() < 1e-14 * np.abs(ref.fst[1:]).max()
    out = sim.get_state()
    if prec == dgx.DG_FP64:
        assert state_err(out, ref.w, P) < FP64_STEP_TOL
    else:
        assert rel_l1(out, ref.w, 0) < FP32_L1_TOL
        assert state_err(out, ref.w, P) < 1e-5
    sim.close()


def test_forced_restart_is_bitwise():
    wl = _wl(3, 2, (6, 5, 4), (1.0, 1.0, 1.0), 1e-3, 1)
    w = inputs.random_modal_state(wl, seed=5)
    a = dgx.Simulation(wl, precision=dgx.DG_FP32_BULK)
    b = dgx.Simulation(wl, precision=dgx.DG_FP32_BULK)
    for s in (a, b):
        s.set_state(w)
    for _ in range(7):
        a.step()
    for _ in range(4):
        b.step()
    c = dgx.Simulation(wl, precision=dgx.DG_FP32_BULK)
    c.set_state(b.get_state())
    c.set_aux(*b.get_aux())
    c.set_forcing(b.get_forcing())
    for _ in range(3):
        c.step()
    assert np.array_equal(a.get_state(), c.get_state())
    assert np.array_equal(a.get_forcing(), c.get_forcing())
    for s in (a, b, c):
        s.close()


def test_forcing_state_calls_need_forcing_on():
    wl = _wl(2, 1, (4, 4), (1.0, 1.0)).with_(forcing_on=0)
    s = dgx.Simulation(wl)
    with pytest.raises(dgx.DGError) as e:
        s.get_forcing()
    assert e.value.code == dgx.DG_EINVAL
    s.close()


def test_batch_rejects_forced_members():
    s = dgx.Simulation(_wl(2, 3, (8, 8), (1.0, 1.0), 0.0, 1))
    with pytest.raises(dgx.DGError) as e:
        dgx.dg_batch_create([s.h])
    assert e.value.code == dgx.DG_EUNSUPPORTED
    s.close()
