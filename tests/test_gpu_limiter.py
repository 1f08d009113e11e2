"""Positivity limiter (Sec. 4.2) on the GPU against the oracle: one whole step on states whose
troubled cells have negative point densities and pressures, and per-step parity on a small
version of the 3-D rotated-Sod + blast workload (AV + limiter)."""
import numpy as np
import pytest

import oracle
from paper_2208_11131_gb300 import build as B
from paper_2208_11131_gb300 import dgx, inputs

from .helpers import problem, rel_l1, state_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    dgx.lib()


def troubled_state(wl, seed):
    """random smooth state with a few cells whose higher density and energy modes are blown up"""
    w = inputs.random_modal_state(wl, seed=seed, amp=0.02)
    rng = np.random.default_rng(seed + 1)
    cells = rng.choice(wl.ncell, size=max(2, wl.ncell // 6), replace=False)
    for c in cells:
        w[0, c, 1:] *= 40.0
        w[wl.dim + 1, c, 1:] *= 40.0
    return w, cells


@pytest.mark.parametrize("dim,n,N", [(2, 2, (9, 7)), (2, 3, (12, 10)), (3, 1, (5, 4, 3)), (3, 2, (4, 5, 3)),
                                     (3, 3, (4, 3, 3))])
@pytest.mark.parametrize("prec", [dgx.DG_FP64, dgx.DG_FP32_BULK])
def test_limited_step_matches_oracle(dim, n, N, prec):
    wl = inputs.Workload("lim", dim, n, tuple(N) + (1,) * (3 - len(N)), (0, 0, 0), (1.0, 1.0, 1.0), gamma=1.4,
                         av_on=1, positivity_on=1, cfl=0.3)
    w, cells = troubled_state(wl, seed=7 + n)
    P = problem(wl)
    # the input is non-physical at points of the troubled cells, and the limiter changes the step
    lim = oracle.Sim(P, w)
    dt, st = lim.step()
    assert st == 0
    nolim = oracle.Sim(problem(wl, positivity_on=0), w)
    nolim.step(dt)
    assert not np.allclose(lim.w, nolim.w, atol=1e-3)
    sim = dgx.Simulation(wl, precision=prec)
    sim.set_state(w)
    sim.step(dt)
    out = sim.get_state()
    if prec == dgx.DG_FP64:
        assert state_err(out, lim.w, P) < 1e-11
    else:
        assert rel_l1(out, lim.w, 0) < 1e-5
    sim.close()


def test_sod_blast_3d_per_step_parity():
    """8^3 cells, degree 3, outflow, AV + limiter: every step compared on identical input."""
    wl = inputs.c3_sod_blast(N=8, n=3)
    w0 = inputs.project(wl, inputs.sod_blast_ic(wl))
    P = problem(wl)
    sim = dgx.Simulation(wl)
    sim.set_state(w0)
    for _ in range(6):
        wg = sim.get_state()
        S, wig, scal = sim.get_aux()
        ref = oracle.Sim(P, wg, S_prev=S.copy(), wig=wig.copy(), scal=scal.copy())
        _, st = ref.step()
        assert st == 0
        sim.step()
        assert state_err(sim.get_state(), ref.w, P) < 1e-12
    sim.close()


def test_sod_blast_3d_fp32_bulk_tracks_fp64():
    wl = inputs.c3_sod_blast(N=8, n=3)
    w0 = inputs.project(wl, inputs.sod_blast_ic(wl))
    a = dgx.Simulation(wl, precision=dgx.DG_FP64)
    b = dgx.Simulation(wl, precision=dgx.DG_FP32_BULK)
    a.set_state(w0)
    b.set_state(w0)
    for _ in range(6):
        a.step()
        b.step()
    wa, wb = a.get_state(), b.get_state()
    # the stated FP32-bulk tolerance, 1e-5 relative L1 in density (measured 5.8e-8 after 30 steps,
    # no sensor or wiggle-source switch flipped between the precisions)
    assert rel_l1(wb, wa, 0) < 1e-5
    a.close()
    b.close()


@pytest.mark.parametrize("n,N", [(1, (6, 5, 4)), (3, (5, 4, 3))])
def test_limited_cfl_steps_fp32_bulk(n, N):
    """Three CFL steps with AV and the limiter in FP32-bulk, the time step chosen by each side: the
    3-D FP32 plans of degrees 1 and 3 run the lane-group step prologue (sensor, wiggle source and
    the CFL maxima), whose dt must agree with the oracle's to FP32 rounding (relative 1e-5), and the
    states to the FP32-bulk tolerance."""
    wl = inputs.Workload("lim", 3, n, N, (0, 0, 0), (1.0, 1.0, 1.0), gamma=1.4, av_on=1, positivity_on=1,
                         cfl=0.3)
    w, _ = troubled_state(wl, seed=11 + n)
    P = problem(wl)
    ref = oracle.Sim(P, w)
    sim = dgx.Simulation(wl, precision=dgx.DG_FP32_BULK)
    sim.set_state(w)
    for _ in range(3):
        dt_ref, st = ref.step()
        assert st == 0
        sim.step()
        dt_gpu = sim.get_aux()[2][0]
        assert abs(dt_gpu - dt_ref) <= 1e-5 * dt_ref
    assert rel_l1(sim.get_state(), ref.w, 0) < 1e-5
    sim.close()
