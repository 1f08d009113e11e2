"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerances:
  * one right-hand side: the error of each field is measured against the size of the terms that are
    summed, |u_f| (max c_s + max|v|) / h_min (helpers.rhs_scale): near equilibrium those terms cancel
    to a far smaller result, and rounding errors scale with the terms, not with the result.
    FP64: 1e-13 of that scale (a few hundred unit roundoffs of 1.1e-16); FP32-bulk: 1e-5 (~170 FP32
    unit roundoffs of 6e-8).
  * whole SSP-RK steps: FP64 L-infinity per field relative to the field's physical scale
    (helpers.state_scale: rho_max, rho_max lambda for momentum, e_max, 1 for alpha) 1e-11;
    FP32-bulk relative L1 in density 1e-5.
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


def _wl(dim, n, N, hi, bc=(0, 0, 0), nu=0.0, av=0, gamma=1.4, cfl=0.3):
    N = tuple(N) + (1,) * (3 - len(N))
    hi = tuple(hi) + (1.0,) * (3 - len(hi))
    return inputs.Workload(f"t{dim}{n}", dim, n, N, (0.0, 0.0, 0.0), hi, bc=tuple(bc) + (0,) * (3 - len(bc)),
                           gamma=gamma, nu=nu, kappa=nu, av_on=av, cfl=cfl)


RHS_CASES = [
    # dim, n, cells, box, bc, nu, av  -- sizes span several tiles and leave ragged tails
    (2, 0, (37, 21), (1.0, 1.0), (0, 0), 0.0, 0),
    (2, 1, (19, 11), (1.0, 0.7), (0, 0), 0.0, 0),
    (2, 2, (17, 9), (1.3, 1.0), (0, 0), 1e-3, 1),
    (2, 3, (11, 13), (1.0, 2.0), (0, 0), 1e-3, 1),
    (2, 3, (10, 7), (1.0, 1.0), (1, 1), 0.0, 1),
    (2, 4, (9, 7), (1.0, 1.0), (1, 0), 0.0, 1),
    (2, 5, (6, 5), (1.0, 1.0), (0, 1), 2e-3, 1),
    # several tiles of the 2-D lane-group kernel (8 x 8 cells at degree 3, 16 x 8 at degree 1), ragged
    (2, 3, (37, 21), (1.0, 1.5), (0, 1), 1e-3, 1),
    (2, 1, (45, 19), (1.2, 1.0), (1, 0), 0.0, 1),
    (3, 0, (9, 5, 6), (1.0, 1.0, 1.0), (0, 0, 0), 0.0, 0),
    (3, 1, (7, 5, 3), (1.0, 0.8, 0.6), (0, 0, 0), 1e-3, 1),
    (3, 2, (5, 5, 3), (1.0, 1.0, 1.0), (0, 0, 1), 0.0, 1),
    (3, 3, (5, 3, 3), (1.0, 1.0, 1.0), (0, 0, 0), 1e-3, 1),
    (3, 3, (3, 4, 5), (1.0, 1.0, 1.0), (1, 1, 1), 0.0, 1),
    (3, 4, (3, 3, 2), (1.0, 1.0, 1.0), (0, 0, 0), 1e-3, 1),
    (3, 5, (3, 2, 2), (1.0, 1.0, 1.0), (0, 1, 0), 0.0, 1),
]


@pytest.mark.parametrize("dim,n,N,box,bc,nu,av", RHS_CASES)
@pytest.mark.parametrize("prec", [dgx.DG_FP64, dgx.DG_FP32_BULK])
def test_rhs_parity(dim, n, N, box, bc, nu, av, prec):
    wl = _wl(dim, n, N, box, bc, nu, av)
    w = inputs.random_modal_state(wl, seed=100 + 10 * dim + n)
    wig = np.random.default_rng(n).uniform(0.0, 0.5, wl.ncell) if av else None
    ref, st = oracle.rhs(problem(wl), w, wig)
    assert st == 0
    sim = dgx.Simulation(wl, precision=prec)
    sim.set_state(w)
    if av:
        sim.set_aux(wig=wig)
    out = sim.rhs()
    err = rhs_err(out, ref, problem(wl), w)
    assert err < (FP64_RHS_TOL if prec == dgx.DG_FP64 else FP32_RHS_TOL), err
    sim.close()


DEGENERATE_CASES = [
    # one cell along an axis: the cell is its own periodic neighbour, or both its faces are outflow
    # boundaries; a single periodic cell
    (2, 3, (1, 5), (1.0, 0.7), (1, 0)),
    (2, 2, (7, 1), (1.0, 0.7), (0, 0)),
    (2, 3, (1, 1), (1.0, 0.7), (0, 0)),
    (2, 1, (1, 4), (1.0, 0.7), (1, 0)),
    (3, 2, (1, 2, 3), (1.0, 0.7, 0.9), (0, 0, 0)),
    (3, 1, (2, 1, 1), (1.0, 0.7, 0.9), (0, 1, 0)),
]


@pytest.mark.parametrize("dim,n,N,box,bc", DEGENERATE_CASES)
@pytest.mark.parametrize("prec", [dgx.DG_FP64, dgx.DG_FP32_BULK])
def test_rhs_parity_degenerate_grids(dim, n, N, box, bc, prec):
    wl = _wl(dim, n, N, box, bc, 1e-3, 1)
    w = inputs.random_modal_state(wl, seed=7 + n)
    ref, st = oracle.rhs(problem(wl), w)
    assert st == 0
    sim = dgx.Simulation(wl, precision=prec)
    sim.set_state(w)
    out = sim.rhs()
    err = rhs_err(out, ref, problem(wl), w)
    assert err < (FP64_RHS_TOL if prec == dgx.DG_FP64 else FP32_RHS_TOL), err
    # a whole step
    o = oracle.Sim(problem(wl), w)
    _, st = o.step()
    assert st == 0
    sim.step()
    if prec == dgx.DG_FP64:
        assert state_err(sim.get_state(), o.w, problem(wl)) < 1e-11
    else:
        assert rel_l1(sim.get_state(), o.w, 0) < 1e-5
    sim.close()


def _run_both(wl, w0, nsteps, prec, dt=0.0, rk=0):
    P = problem(wl, rk_stages=rk)
    ref = oracle.Sim(P, w0)
    sim = dgx.Simulation(wl, precision=prec, rk_stages=rk)
    sim.set_state(w0)
    for _ in range(nsteps):
        _, st = ref.step(dt)
        assert st == 0
        sim.step(dt)
    out = sim.get_state()
    return sim, ref, out


def test_density_wave_20_steps_fp64_and_fp32():
    """2-D Euler density wave, 32^2, degree 2, SSP-RK3, 20 CFL-0.3 steps (the plain-method workload)."""
    wl = inputs.c1_density_wave(N=32, n=2)
    w0 = inputs.project(wl, inputs.density_wave_ic(wl, 0.0))
    sim, ref, out = _run_both(wl, w0, 20, dgx.DG_FP64)
    assert state_err(out, ref.w, ref.prob) < FP64_STEP_TOL
    S, wig, scal = sim.get_aux()
    assert abs(scal[2] - ref.t) < 1e-14 * ref.t and scal[1] == 20
    sim.close()
    sim, ref, out32 = _run_both(wl, w0, 20, dgx.DG_FP32_BULK)
    assert rel_l1(out32, ref.w, 0) < FP32_L1_TOL
    # same accuracy against the exact solution
    P = problem(wl)
    e64 = oracle.l1_error(P, out, inputs.density_wave_ic(wl, ref.t))
    e32 = oracle.l1_error(P, out32, inputs.density_wave_ic(wl, ref.t))
    assert abs(e32 / e64 - 1.0) < 0.01, (e32, e64)
    sim.close()


@pytest.mark.parametrize("prec", [dgx.DG_FP64, dgx.DG_FP32_BULK])
def test_shear_layer_ns_av_steps(prec):
    """2-D compressible NS shear layer with artificial viscosity, degree 3, SSP(5,4), several steps;
    checks the state, the sensor history and the time-step bookkeeping."""
    wl = inputs.c2_shear_layer(N=16, n=3)
    w0 = inputs.project(wl, inputs.shear_layer_ic(wl))
    sim, ref, out = _run_both(wl, w0, 6, prec)
    if prec == dgx.DG_FP64:
        assert state_err(out, ref.w, ref.prob) < FP64_STEP_TOL
        S, wig, scal = sim.get_aux()
        assert np.abs(S - ref.S_prev).max() < 1e-12
        assert np.abs(wig - ref.wig).max() <= 1e-10 * max(1.0, np.abs(ref.wig).max())
        assert abs(scal[0] - ref.scal[0]) < 1e-15 * ref.scal[0]
    else:
        assert rel_l1(out, ref.w, 0) < FP32_L1_TOL
    sim.close()


@pytest.mark.parametrize("prec", [dgx.DG_FP64, dgx.DG_FP32_BULK])
def test_3d_ns_av_steps(prec):
    wl = _wl(3, 2, (6, 5, 4), (1.0, 1.0, 1.0), (0, 0, 0), 2e-3, 1, gamma=1.4, cfl=0.4)
    w0 = inputs.random_modal_state(wl, seed=11, amp=0.03)
    sim, ref, out = _run_both(wl, w0, 3, prec)
    if prec == dgx.DG_FP64:
        assert state_err(out, ref.w, ref.prob) < FP64_STEP_TOL
    else:
        assert rel_l1(out, ref.w, 0) < FP32_L1_TOL
    sim.close()


@pytest.mark.parametrize("rk,n", [(1, 0), (2, 1), (3, 2), (5, 3), (5, 2)])
def test_every_rk_scheme(rk, n):
    wl = _wl(2, n, (9, 8), (1.0, 1.0), (0, 0), 1e-3, 1)
    w0 = inputs.random_modal_state(wl, seed=3, amp=0.03)
    sim, ref, out = _run_both(wl, w0, 3, dgx.DG_FP64, rk=rk)
    assert state_err(out, ref.w, ref.prob) < FP64_STEP_TOL
    sim.close()


def test_sod_tube_outflow_steps():
    g = 1.4
    wl = inputs.Workload("sod", 2, 2, (48, 3, 1), (0, 0, 0), (1.0, 3.0 / 48, 1.0), bc=(1, 0, 0), gamma=g, av_on=1,
                         cfl=0.3)
    w0 = inputs.project(wl, inputs.sod_tube_ic(wl))
    sim, ref, out = _run_both(wl, w0, 10, dgx.DG_FP64)
    assert state_err(out, ref.w, ref.prob) < FP64_STEP_TOL
    sim.close()


def test_sod_tube_per_step_parity():
    """Shock workload, step by step: the oracle restarts every step from the GPU's state and sensor history
    (S_prev, wiggle source, dt, step count), so each whole step -- sensor, CFL dt, all stages -- is compared
    on identical input."""
    g = 1.4
    wl = inputs.Workload("sod", 2, 3, (40, 2, 1), (0, 0, 0), (1.0, 2.0 / 40, 1.0), bc=(1, 0, 0), gamma=g, av_on=1,
                         cfl=0.3)
    w0 = inputs.project(wl, inputs.sod_tube_ic(wl))
    P = problem(wl)
    sim = dgx.Simulation(wl)
    sim.set_state(w0)
    for _ in range(12):
        wg = sim.get_state()
        S, wig, scal = sim.get_aux()
        ref = oracle.Sim(P, wg, S_prev=S.copy(), wig=wig.copy(), scal=scal.copy())
        _, st = ref.step()
        assert st == 0
        sim.step()
        out = sim.get_state()
        assert state_err(out, ref.w, P) < 1e-13
        S2, wig2, scal2 = sim.get_aux()
        assert np.abs(wig2 - ref.wig).max() <= 1e-9 * max(1.0, np.abs(ref.wig).max())
        assert scal2[0] == pytest.approx(ref.scal[0], rel=1e-15)
    sim.close()


def test_max_dt_and_conserved_sums():
    wl = inputs.c2_shear_layer(N=24, n=3)
    w0 = inputs.project(wl, inputs.shear_layer_ic(wl))
    P = problem(wl)
    for prec, tol in ((dgx.DG_FP64, 1e-14), (dgx.DG_FP32_BULK, 1e-6)):
        sim = dgx.Simulation(wl, precision=prec)
        sim.set_state(w0)
        dt_ref, st = oracle.max_dt(P, w0)
        assert abs(sim.max_dt() / dt_ref - 1) < tol
        tot = sim.conserved_sums()
        ref = w0[:4, :, 0].sum(1) * np.prod(wl.h)
        assert np.allclose(tot, ref, rtol=1e-14, atol=1e-14 * np.abs(ref).max())
        sim.close()


def test_graph_replay_equals_step_loop_bitwise():
    wl = inputs.c2_shear_layer(N=16, n=3)
    w0 = inputs.project(wl, inputs.shear_layer_ic(wl))
    for prec in (dgx.DG_FP64, dgx.DG_FP32_BULK):
        a = dgx.Simulation(wl, precision=prec)
        b = dgx.Simulation(wl, precision=prec)
        a.set_state(w0)
        b.set_state(w0)
        for _ in range(5):
            a.step()
        b.steps(5)
        assert np.array_equal(a.get_state(), b.get_state())
        assert np.array_equal(a.get_aux()[1], b.get_aux()[1])
        a.close()
        b.close()


def test_conservation_over_steps_periodic():
    wl = inputs.c2_shear_layer(N=16, n=3)
    w0 = inputs.project(wl, inputs.shear_layer_ic(wl))
    for prec, tol in ((dgx.DG_FP64, 1e-13), (dgx.DG_FP32_BULK, 1e-7)):
        sim = dgx.Simulation(wl, precision=prec)
        sim.set_state(w0)
        m0 = sim.conserved_sums()
        sim.steps(8)
        sim.sync()
        m1 = sim.conserved_sums()
        assert np.all(np.abs(m1 - m0) <= tol * np.abs(m0).max()), (m1 - m0)
        sim.close()


def test_nonphysical_state_reported_not_faulted():
    wl = _wl(2, 2, (8, 8), (1.0, 1.0))
    w = inputs.random_modal_state(wl, seed=1)
    w[0, 5, 0] = -0.5  # negative cell-mean density
    sim = dgx.Simulation(wl)
    sim.set_state(w)
    with pytest.raises(dgx.DGError) as e:
        sim.rhs()
    assert e.value.code == dgx.DG_ENONPHYS
    # the handle stays usable
    sim.set_state(inputs.random_modal_state(wl, seed=2))
    sim.rhs()
    sim.close()


def test_device_pointer_entry_points_with_torch():
    torch = pytest.importorskip("torch")
    wl = inputs.c2_shear_layer(N=8, n=3)
    w0 = inputs.project(wl, inputs.shear_layer_ic(wl))
    sim = dgx.Simulation(wl)
    sim.set_stream(torch.cuda.current_stream().cuda_stream)
    wd = torch.from_numpy(w0).cuda()
    dgx.dg_set_state_device(sim.h, wd.data_ptr())
    rd = torch.empty_like(wd)
    dgx.dg_rhs_device(sim.h, rd.data_ptr())
    back = torch.empty_like(wd)
    dgx.dg_get_state_device(sim.h, back.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(back, wd)
    ref, _ = oracle.rhs(problem(wl), w0, np.zeros(wl.ncell))
    assert rhs_err(rd.cpu().numpy(), ref, problem(wl), w0) < FP64_RHS_TOL
    sim.close()


@pytest.mark.parametrize("prec", [dgx.DG_FP64, dgx.DG_FP32_BULK])
def test_full_size_shear_layer_rhs_and_one_step(prec):
    """The benchmarked workload at full size: 256x256 cells, degree 3, NS + AV, in the launch
    configuration of the benchmark (same kernels, same tiles)."""
    wl = inputs.c2_shear_layer()
    w0 = inputs.project(wl, inputs.shear_layer_ic(wl))
    P = problem(wl)
    wig = np.random.default_rng(5).uniform(0, 0.3, wl.ncell)
    ref, st = oracle.rhs(P, w0, wig)
    assert st == 0
    sim = dgx.Simulation(wl, precision=prec)
    sim.set_state(w0)
    sim.set_aux(wig=wig)
    out = sim.rhs()
    assert rhs_err(out, ref, P, w0) < (FP64_RHS_TOL if prec == dgx.DG_FP64 else FP32_RHS_TOL)
    sim.set_aux(wig=np.zeros(wl.ncell))
    sim.step()
    o = oracle.Sim(P, w0)
    o.step()
    out = sim.get_state()
    if prec == dgx.DG_FP64:
        assert state_err(out, o.w, P) < FP64_STEP_TOL
    else:
        assert rel_l1(out, o.w, 0) < FP32_L1_TOL
    sim.close()


# The 3-D FP32-bulk kernel of degrees 1 and 3 marches along z through chunks of planes (DGX_ZCHUNK
# sets the chunk length; small grids otherwise get one-plane chunks): multi-plane chunks with a
# remainder, ragged column tiles in x and y, periodic and outflow boundaries, one plane along z.
ZMARCH_CASES = [
    # n, cells, box, bc, nu, av, chunk
    (3, (9, 6, 13), (1.0, 0.8, 1.3), (0, 0, 0), 1e-3, 1, 0),
    (3, (9, 6, 13), (1.0, 0.8, 1.3), (0, 0, 0), 1e-3, 1, 5),
    (3, (5, 7, 8), (1.0, 1.0, 1.0), (1, 0, 1), 0.0, 1, 3),
    (3, (6, 5, 9), (1.0, 1.0, 1.0), (0, 1, 0), 2e-3, 0, 4),
    (3, (5, 3, 1), (1.0, 1.0, 0.5), (0, 0, 0), 1e-3, 1, 0),
    (3, (3, 2, 2), (1.0, 1.0, 1.0), (0, 0, 1), 0.0, 1, 2),
    (1, (17, 9, 11), (1.0, 0.9, 1.1), (0, 0, 0), 1e-3, 1, 4),
    (1, (10, 12, 7), (1.0, 1.0, 1.0), (1, 1, 1), 0.0, 1, 3),
]


@pytest.mark.parametrize("n,N,box,bc,nu,av,chunk", ZMARCH_CASES)
def test_zmarch_rhs_and_step_parity(n, N, box, bc, nu, av, chunk, monkeypatch):
    if chunk:
        monkeypatch.setenv("DGX_ZCHUNK", str(chunk))
    wl = _wl(3, n, N, box, bc, nu, av)
    P = problem(wl)
    w = inputs.random_modal_state(wl, seed=300 + n + chunk)
    wig = np.random.default_rng(n + chunk).uniform(0.0, 0.5, wl.ncell) if av else None
    ref, st = oracle.rhs(P, w, wig)
    assert st == 0
    sim = dgx.Simulation(wl, precision=dgx.DG_FP32_BULK)
    sim.set_state(w)
    if av:
        sim.set_aux(wig=wig)
    assert rhs_err(sim.rhs(), ref, P, w) < FP32_RHS_TOL
    sim.close()
    # three whole steps (fused first stage: sensor, wiggle source and CFL speeds; dt reduction in the
    # second) against the oracle
    o = oracle.Sim(P, w)
    sim = dgx.Simulation(wl, precision=dgx.DG_FP32_BULK)
    sim.set_state(w)
    for _ in range(3):
        _, st = o.step()
        assert st == 0
        sim.step()
    assert rel_l1(sim.get_state(), o.w, 0) < FP32_L1_TOL
    S, wg, scal = sim.get_aux()
    assert abs(scal[0] / o.scal[0] - 1) < 1e-5
    if av:
        assert np.abs(wg - o.wig).max() <= 1e-3 * max(1.0, np.abs(o.wig).max())
    sim.close()
