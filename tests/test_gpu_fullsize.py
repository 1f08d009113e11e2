"""Parity at the workloads' full sizes, in the launch configuration bench.py uses (persistent stage
kernel, the handle's default tiles and grid), element by element where the oracle can compute the
whole output and on sampled outputs otherwise.

* density wave 32^2, degree 2, 20 SSP-RK3 steps: the state against the oracle, and the metric's
  "same L1 error": the FP32-bulk L1 error against the exact solution equals the FP64 one within 1%;
* Sod plane + blast 64^3, degree 3 (AV, limiter, outflow): the whole right-hand side in FP64 and
  FP32-bulk, and one whole FP64 step;
* driven turbulence box 128^3, degree 3: from rest every flux cancels and the right-hand side is the
  driving source alone; sampled cells against an independent numpy Gauss assembly of rho s with the
  oracle's driving field, and the properties that hold at every cell (no mass, energy or alpha
  source at rest);
* the 64-member ensemble: batched against the same members stepped alone, and its smallest smooth
  and smallest shock-tube members against the oracle.
Tolerances as in test_gpu_parity (flux-term scale for right-hand sides, physical scales for states).
"""
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


def test_density_wave_32_full_run_and_same_l1_error():
    wl = inputs.c1_density_wave(N=32, n=2)
    P = problem(wl)
    w0 = inputs.project(wl, inputs.density_wave_ic(wl, 0.0))
    ref = oracle.Sim(P, w0)
    sims = {p: dgx.Simulation(wl, precision=p) for p in (dgx.DG_FP64, dgx.DG_FP32_BULK)}
    for s in sims.values():
        s.set_state(w0)
    for _ in range(20):
        dt, st = ref.step()
        assert st == 0
        for s in sims.values():
            s.step()
    T = ref.t
    out64, out32 = sims[dgx.DG_FP64].get_state(), sims[dgx.DG_FP32_BULK].get_state()
    assert state_err(out64, ref.w, P) < 1e-11
    assert rel_l1(out32, ref.w, 0) < 1e-5
    assert abs(sims[dgx.DG_FP64].get_aux()[2][2] - T) < 1e-13
    ex = inputs.density_wave_ic(wl, T)
    e64 = oracle.l1_error(P, out64, ex)
    e32 = oracle.l1_error(P, out32, ex)
    assert e64 > 0 and abs(e32 / e64 - 1) < 0.01, (e32, e64)
    for s in sims.values():
        s.close()


@pytest.fixture(scope="module")
def sod_blast_64():
    wl = inputs.c3_sod_blast(N=64, n=3)
    P = problem(wl)
    w = inputs.project(wl, inputs.sod_blast_ic(wl))
    oracle.positivity(P, w)  # the projected jumps are non-physical at some points before limiting
    return wl, P, w


@pytest.mark.parametrize("prec", [dgx.DG_FP64, dgx.DG_FP32_BULK])
def test_sod_blast_64_full_rhs(sod_blast_64, prec):
    wl, P, w = sod_blast_64
    ref, st = oracle.rhs(P, w)
    assert st == 0
    sim = dgx.Simulation(wl, precision=prec)
    sim.set_state(w)
    out = sim.rhs()
    assert rhs_err(out, ref, P, w) < (1e-13 if prec == dgx.DG_FP64 else 1e-5)
    sim.close()


def test_sod_blast_64_full_step(sod_blast_64):
    wl, P, w = sod_blast_64
    ref = oracle.Sim(P, w)
    _, st = ref.step()
    assert st == 0
    sim = dgx.Simulation(wl)
    sim.set_state(w)
    sim.step()
    assert state_err(sim.get_state(), ref.w, P) < 1e-11
    assert abs(sim.get_aux()[2][0] / ref.scal[0] - 1) < 1e-13
    sim.close()


@pytest.mark.parametrize("prec", [dgx.DG_FP64, dgx.DG_FP32_BULK])
def test_turbulence_box_128_full_rhs_at_rest(prec):
    wl = inputs.c4_turbulence_box(N=128, n=3)
    P = problem(wl)
    w = inputs.rest_state(wl)
    fst = oracle.forcing_state()
    oracle.forcing_update(P, fst, 0.05)
    sim = dgx.Simulation(wl, precision=prec)
    sim.set_state(w)
    sim.set_forcing(fst)
    out = sim.rhs()
    d = 3
    flux = (1.0 / wl.gamma) * 2.0 / min(P.h)  # flux-term size: pressure p = 1/gamma over h/2
    tol = (1e-13 if prec == dgx.DG_FP64 else 1e-5) * flux
    # at rest: the HLLC mass flux of equal states is exactly zero and so are all alpha sources;
    # the energy gets no driving work (s.(rho v) = 0), only the heat flux of rounding-level
    # gradients of the uniform state
    assert not np.any(out[0]) and not np.any(out[d + 2])
    assert np.abs(out[d + 1]).max() < tol
    # sampled cells: momentum = 2^-d sum_j G_j phi_l(xi_j) rho s(x_j) (+ flux terms that cancel to
    # rounding of the flux size p 2/h)
    rng = np.random.default_rng(128)
    cells = rng.choice(P.ncell, 200, replace=False)
    q = wl.n + 1
    xg, wg = np.polynomial.legendre.leggauss(q)
    idx = np.stack(np.meshgrid(*([np.arange(q)] * d), indexing="ij")[::-1], -1).reshape(-1, d)
    xi, G = xg[idx], np.prod(wg[idx], 1)
    phi = np.ones((len(xi), len(idx)))
    for a in range(d):
        Pt = np.stack([math.sqrt(2 * l + 1) * np.polynomial.legendre.legval(xi[:, a], [0] * l + [1])
                       for l in range(q)], 1)
        phi *= Pt[:, idx[:, a]]
    h = np.array(P.h)
    xc = P.cell_centres()[cells]
    X = (xc[:, None, :] + 0.5 * h * xi[None]).reshape(-1, d)
    s = oracle.forcing_eval(P, fst, X)[:, :d].reshape(len(cells), len(xi), d)
    expect = np.einsum("kja,j,jl->akl", s, G, phi) / 2.0 ** d  # rho = 1
    got = out[1:d + 1][:, cells, :]
    assert np.abs(got - expect).max() < tol
    assert np.abs(expect).max() > 10 * tol  # the source is what is being compared
    sim.close()


def test_ensemble_full_manifest_batched_and_oracle():
    members = inputs.c5_manifest(count=64)
    a = [dgx.Simulation(m.wl, precision=dgx.DG_FP32_BULK) for m in members]
    b = [dgx.Simulation(m.wl, precision=dgx.DG_FP32_BULK) for m in members]
    w0s = [inputs.member_state(m) for m in members]
    for sa, sb, w0 in zip(a, b, w0s):
        sa.set_state(w0)
        sb.set_state(w0)
    batch = dgx.dg_batch_create([s.h for s in b])
    for s in a:
        for _ in range(3):
            s.step()
    dgx.dg_batch_step(batch, 3)
    dgx.dg_batch_sync(batch)
    for sa, sb, m in zip(a, b, members):
        assert state_err(sb.get_state(), sa.get_state(), problem(m.wl)) < 2e-5
    # the smallest smooth and the smallest shock-tube member against the oracle (FP32-bulk vs FP64,
    # the stated 1e-5 relative L1 in density; measured 1.7e-7 on the shock tube after 50 steps with no
    # artificial-viscosity switch decision flipped)
    for kind, tol in (("wave", 1e-5), ("sod", 1e-5)):
        k = min((i for i in range(len(members)) if members[i].kind == kind), key=lambda i: members[i].wl.dofs)
        ref = oracle.Sim(problem(members[k].wl), w0s[k])
        for _ in range(3):
            _, st = ref.step()
            assert st == 0
        assert rel_l1(b[k].get_state(), ref.w, 0) < tol
    dgx.dg_batch_destroy(batch)
    for s in a + b:
        s.close()
