"""The five workloads at their stated step counts against the oracle (element by element), FP64 and
FP32-bulk, with the stated tolerances: FP64 within 1e-11 relative L-infinity (per-field physical
scale, helpers.state_err), FP32-bulk within 1e-5 relative L1 in density.

* shear layer: 256^2 cells, degree 3, NS + AV, SSP(5,4), 500 steps;
* Sod plane + blast: degree 3, AV + positivity limiter, outflow, 200 steps on 16^3 cells (the
  oracle's cost of 64^3 x 200 steps is beyond a test; the 64^3 grid itself is compared for a whole
  right-hand side and a whole step in test_gpu_fullsize);
* driven turbulence box: degree 3, NS + AV + driving, started at rms Mach 0.3, 100 steps on 16^3
  cells, and the shell-summed velocity power spectrum of the GPU runs against the oracle's
  (32^3 cells with DGX_LONG=1: about ten minutes of oracle time on 16 host cores);
* ensemble: 50 steps of the whole 64-member batch against the same members stepped alone, and its
  smallest smooth and smallest shock-tube members against the oracle.
Every run also reports its measured errors (pytest -s).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2208_11131_gb300 import build as B
from paper_2208_11131_gb300 import dgx, inputs

from .helpers import problem, rel_l1, state_err

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    dgx.lib()


def _run_both(wl, w0, steps, fst=None):
    """the oracle and the two GPU precisions from the same state, `steps` CFL steps each"""
    P = problem(wl)
    ref = oracle.Sim(P, w0)
    sims = {p: dgx.Simulation(wl, precision=p) for p in (dgx.DG_FP64, dgx.DG_FP32_BULK)}
    for s in sims.values():
        s.set_state(w0)
    for _ in range(steps):
        _, st = ref.step()
        assert st == 0
    for s in sims.values():
        for _ in range(steps):
            s.step()
    out = {p: s.get_state() for p, s in sims.items()}
    times = {p: s.get_aux()[2][2] for p, s in sims.items()}
    for s in sims.values():
        s.close()
    return P, ref, out[dgx.DG_FP64], out[dgx.DG_FP32_BULK], times


def _check(name, P, ref, o64, o32, times):
    e64 = state_err(o64, ref.w, P)
    e32 = rel_l1(o32, ref.w, 0)
    print(f"\n{name}: fp64 rel Linf {e64:.3e}  fp32-bulk rel L1(rho) {e32:.3e}  t {ref.t:.6g} "
          f"(gpu fp64 {times[dgx.DG_FP64]:.6g})")
    assert e64 < FP64_TOL, (name, e64)
    assert e32 < FP32_TOL, (name, e32)
    assert abs(times[dgx.DG_FP64] / ref.t - 1) < 1e-12


def test_shear_layer_256_500_steps():
    wl = inputs.c2_shear_layer(N=256, n=3)
    w0 = inputs.project(wl, inputs.shear_layer_ic(wl))
    _check("shear layer 256^2 x 500", *_run_both(wl, w0, 500))


def test_sod_blast_16_200_steps():
    wl = inputs.c3_sod_blast(N=16, n=3)
    w0 = inputs.project(wl, inputs.sod_blast_ic(wl))
    _check("sod plane + blast 16^3 x 200", *_run_both(wl, w0, 200))


def velocity_spectrum(wl, w):
    """shell sums of |FFT(v)|^2 over integer |k| of the cell-mean velocity (rho v)_0 / rho_0"""
    N = wl.N[0]
    v = (w[1:4, :, 0] / w[0, :, 0]).reshape(3, N, N, N)
    vk = np.fft.fftn(v, axes=(1, 2, 3)) / N ** 3
    f = np.fft.fftfreq(N, 1.0 / N)
    kk = np.sqrt(f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2)
    shell = np.rint(kk).astype(int)
    power = (np.abs(vk) ** 2).sum(0)
    return np.bincount(shell.ravel(), weights=power.ravel())


@pytest.mark.parametrize("N", [16, pytest.param(32, marks=pytest.mark.skipif(
    not os.environ.get("DGX_LONG"), reason="DGX_LONG=1: ten minutes of oracle time"))])
def test_turbulence_box_100_steps_and_spectrum(N):
    wl = inputs.c4_turbulence_box(N=N, n=3)
    w0 = inputs.turbulence_ic_state(wl)
    P, ref, o64, o32, times = _run_both(wl, w0, 100)
    _check(f"driven turbulence box {N}^3 x 100", P, ref, o64, o32, times)
    Er, E64, E32 = (velocity_spectrum(wl, w) for w in (ref.w, o64, o32))
    tot = Er.sum()
    assert Er[1:4].sum() > 0.5 * tot  # the energy sits in the driven and initial shells
    # a relative state error e moves the power of a shell by at most about 2 e times the total (the
    # cross term of the difference field with the velocity, Cauchy-Schwarz); in the energetic shells
    # (over 1% of the total) also relative to the shell itself.  e: the stated 1e-11 (FP64) and 1e-5
    # (FP32-bulk); nearly empty shells can differ more relative to themselves
    big = Er > 0.01 * tot
    for name, E, e in (("fp64", E64, FP64_TOL), ("fp32-bulk", E32, FP32_TOL)):
        d_tot = np.abs(E - Er).max() / tot
        d_big = (np.abs(E - Er)[big] / Er[big]).max()
        print(f"spectrum {N}^3 {name}: max shell difference / total {d_tot:.3e}, "
              f"/ shell (energetic shells) {d_big:.3e}")
        assert d_tot < 2 * e and d_big < 2 * e, (name, d_tot, d_big)


def test_ensemble_50_steps():
    members = inputs.c5_manifest(count=64)
    w0s = [inputs.member_state(m) for m in members]
    a = [dgx.Simulation(m.wl, precision=dgx.DG_FP32_BULK) for m in members]
    b = [dgx.Simulation(m.wl, precision=dgx.DG_FP32_BULK) for m in members]
    for sa, sb, w0 in zip(a, b, w0s):
        sa.set_state(w0)
        sb.set_state(w0)
    batch = dgx.dg_batch_create([s.h for s in b])
    for s in a:
        s.steps(50)
    dgx.dg_batch_step(batch, 50)
    dgx.dg_batch_sync(batch)
    worst = 0.0
    for sa, sb, m in zip(a, b, members):
        sa.sync()
        # batched and stand-alone members are separate compilations of one kernel body (FMA
        # contraction may differ): FP32-bulk rounding over 50 steps, at the FP32-bulk tolerance
        e = rel_l1(sb.get_state(), sa.get_state(), 0)
        worst = max(worst, e)
        assert e < FP32_TOL, (m.wl.name, e)
    for kind in ("wave", "sod"):
        k = min((i for i in range(len(members)) if members[i].kind == kind), key=lambda i: members[i].wl.dofs)
        ref = oracle.Sim(problem(members[k].wl), w0s[k])
        for _ in range(50):
            _, st = ref.step()
            assert st == 0
        e = rel_l1(b[k].get_state(), ref.w, 0)
        print(f"\nensemble member {k} ({kind}, {members[k].wl.N[0]}^2, n={members[k].wl.n}) x 50: "
              f"fp32-bulk rel L1(rho) vs oracle {e:.3e}; batched vs alone worst {worst:.3e}")
        assert e < FP32_TOL
    dgx.dg_batch_destroy(batch)
    for s in a + b:
        s.close()
