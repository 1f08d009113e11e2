"""The total-degree basis (Sec. 2.3) on the GPU against the oracle's native total-degree path:
right-hand side (2-D/3-D, n = 1..5, NS, AV, tracer; FP64 and FP32-bulk), whole steps with the
limiter, order n+1 convergence, the caller-visible mode count, device-pointer transfers, and
batched members.  Tolerances as in test_gpu_parity."""
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


def _wl(dim, n, N, hi, nu=0.0, av=0, tr=0, lim=0, bc=(0, 0, 0)):
    N = tuple(N) + (1,) * (3 - len(N))
    hi = tuple(hi) + (1.0,) * (3 - len(hi))
    return inputs.Workload(f"td{dim}{n}", dim, n, N, (0.0, 0.0, 0.0), hi, bc=bc, gamma=1.4, nu=nu, kappa=nu,
                           av_on=av, positivity_on=lim, cfl=0.3, tracer_on=tr, eta=2e-3 if tr else 0.0, basis=1)


CASES = [
    (2, 1, (9, 7), (1.0, 1.3), 0.0, 0, 0),
    (2, 2, (11, 6), (1.0, 2.0), 1e-3, 1, 0),
    (2, 3, (13, 10), (1.0, 2.0), 1e-3, 1, 1),
    (2, 5, (6, 5), (1.0, 1.0), 0.0, 1, 0),
    (3, 2, (4, 4, 3), (1.0, 1.0, 1.0), 1e-3, 1, 0),
    (3, 3, (4, 3, 3), (1.0, 1.0, 0.7), 0.0, 1, 1),
    (3, 4, (3, 2, 2), (1.0, 1.0, 1.0), 1e-3, 0, 0),
]


@pytest.mark.parametrize("prec", [dgx.DG_FP64, dgx.DG_FP32_BULK])
@pytest.mark.parametrize("dim,n,N,hi,nu,av,tr", CASES)
def test_total_degree_rhs_parity(dim, n, N, hi, nu, av, tr, prec):
    wl = _wl(dim, n, N, hi, nu, av, tr)
    P = problem(wl)
    w = inputs.random_modal_state(wl, seed=40 + n)
    ref, st = oracle.rhs(P, w)
    assert st == 0
    sim = dgx.Simulation(wl, precision=prec)
    assert sim.M == P.M == len(inputs.mode_exponents(dim, n, 1))
    sim.set_state(w)
    out = sim.rhs()
    assert out.shape == w.shape
    assert rhs_err(out, ref, P, w) < (1e-13 if prec == dgx.DG_FP64 else 1e-5)
    assert np.array_equal(sim.get_state(), w)
    sim.close()


@pytest.mark.parametrize("prec", [dgx.DG_FP64, dgx.DG_FP32_BULK])
def test_total_degree_shock_tube_steps_with_limiter(prec):
    wl = _wl(2, 3, (24, 2), (1.0, 2.0 / 24), 0.0, 1, 0, lim=1, bc=(1, 0, 0))
    P = problem(wl)
    w0 = inputs.project(wl, inputs.sod_tube_ic(wl))
    ref = oracle.Sim(P, w0)
    sim = dgx.Simulation(wl, precision=prec)
    sim.set_state(w0)
    for _ in range(5):
        _, st = ref.step()
        assert st == 0
        sim.step()
    out = sim.get_state()
    if prec == dgx.DG_FP64:
        assert state_err(out, ref.w, P) < 1e-11
    else:
        assert rel_l1(out, ref.w, 0) < 1e-5  # the stated FP32-bulk tolerance (measured 1.9e-7 at 20 steps)
    sim.close()


def test_total_degree_density_wave_order():
    errs = []
    for N in (16, 32):
        wl = inputs.c1_density_wave(N=N, n=3).with_(basis=1)
        P = problem(wl)
        sim = dgx.Simulation(wl)
        sim.set_state(inputs.project(wl, inputs.density_wave_ic(wl, 0.0)))
        t = 0.0
        while t < 0.1 - 1e-14:
            dt = min(sim.max_dt(), 0.1 - t)
            sim.step(dt)
            t += dt
        errs.append(oracle.l1_error(P, sim.get_state(), inputs.density_wave_ic(wl, 0.1)))
        sim.close()
    assert 4 - 0.4 < math.log2(errs[0] / errs[1]) < 4 + 0.6, errs


def test_total_degree_device_transfers():
    torch = pytest.importorskip("torch")
    wl = _wl(3, 2, (5, 4, 3), (1.0, 1.0, 1.0), 1e-3, 1)
    w = inputs.random_modal_state(wl, seed=3)
    sim = dgx.Simulation(wl)
    dw = torch.from_numpy(w).cuda()
    dgx.dg_set_state_device(sim.h, dw.data_ptr())
    back = torch.zeros_like(dw)
    dgx.dg_get_state_device(sim.h, back.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(back, dw)
    rd = torch.zeros_like(dw)
    dgx.dg_rhs_device(sim.h, rd.data_ptr())
    torch.cuda.synchronize()
    ref, _ = oracle.rhs(problem(wl), w)
    assert rhs_err(rd.cpu().numpy(), ref, problem(wl), w) < 1e-13
    sim.close()


def test_total_degree_batched_members():
    members = [_wl(2, n, (16, 12), (1.0, 1.0), 1e-3 * (n % 2), 1) for n in (2, 3, 3, 4)]
    a = [dgx.Simulation(wl) for wl in members]
    b = [dgx.Simulation(wl) for wl in members]
    for k, (sa, sb, wl) in enumerate(zip(a, b, members)):
        w0 = inputs.random_modal_state(wl, seed=60 + k)
        sa.set_state(w0)
        sb.set_state(w0)
    batch = dgx.dg_batch_create([s.h for s in b])
    for s in a:
        for _ in range(3):
            s.step()
    dgx.dg_batch_step(batch, 3)
    dgx.dg_batch_sync(batch)
    for sa, sb, wl in zip(a, b, members):
        assert state_err(sb.get_state(), sa.get_state(), problem(wl)) < 1e-13
    dgx.dg_batch_destroy(batch)
    for s in a + b:
        s.close()


# 3-D FP32-bulk at degrees 1 and 3 (no tracer) stores only the total-degree modes (packed storage:
# (n+1)(n+2)(n+3)/6 of (n+1)^3 values per cell and field); the stage, prologue and limiter kernels
# read and write that layout directly.
PACKED = [
    (3, (9, 6, 7), 1e-3, 1, 0),
    (3, (5, 4, 9), 0.0, 1, 1),
    (1, (10, 9, 6), 1e-3, 1, 0),
    (3, (6, 5, 4), 0.0, 0, 0),
]


@pytest.mark.parametrize("n,N,nu,av,lim", PACKED)
def test_packed_total_degree_rhs_and_steps(n, N, nu, av, lim, monkeypatch):
    monkeypatch.setenv("DGX_ZCHUNK", "3")  # multi-plane chunks of the z-marching kernel
    wl = _wl(3, n, N, (1.0, 0.9, 1.1), nu, av, 0, lim, bc=(1, 0, 0) if lim else (0, 0, 0))
    P = problem(wl)
    if lim:
        w = inputs.project(wl, inputs.sod_tube_ic(wl))
    else:
        w = inputs.random_modal_state(wl, seed=80 + n)
    ref, st = oracle.rhs(P, w)
    assert st == 0
    sim = dgx.Simulation(wl, precision=dgx.DG_FP32_BULK)
    assert sim.M == P.M == len(inputs.mode_exponents(3, n, 1))
    sim.set_state(w)
    assert np.array_equal(sim.get_state(), w)
    assert rhs_err(sim.rhs(), ref, P, w) < 1e-5
    o = oracle.Sim(P, w)
    for _ in range(4):
        _, st = o.step()
        assert st == 0
        sim.step()
    assert rel_l1(sim.get_state(), o.w, 0) < 1e-5
    assert abs(sim.max_dt() / oracle.max_dt(P, o.w)[0] - 1) < 1e-5
    wg = sim.get_state()  # the sums read the cell means at the packed stride
    assert np.allclose(sim.conserved_sums(), [np.sum(wg[f, :, 0]) * np.prod(P.h) for f in range(5)], rtol=1e-12,
                       atol=1e-14)
    sim.close()


def test_packed_total_degree_state_is_the_basis_size():
    """device memory of a 3-D degree-3 FP32-bulk handle: total-degree storage holds 20 of the 64
    tensor modes per cell and field"""
    torch = pytest.importorskip("torch")
    wl = _wl(3, 3, (32, 32, 32), (1.0, 1.0, 1.0), 1e-3, 1)
    used = {}
    for basis in (0, 1):
        torch.cuda.synchronize()
        f0, _ = torch.cuda.mem_get_info()
        sim = dgx.Simulation(wl.with_(basis=basis), precision=dgx.DG_FP32_BULK)
        torch.cuda.synchronize()
        f1, _ = torch.cuda.mem_get_info()
        used[basis] = f0 - f1
        sim.close()
    state = 6 * 32 ** 3 * (8 + 8 + 4 + 4 + 3 * 4)  # bytes per state value: u^n, u^n+1, FP32 copies, 3 deltas
    assert used[0] >= 64 * state
    assert used[1] < 0.34 * used[0]  # 20/64 = 0.3125 plus the per-handle scalars


def test_packed_total_degree_device_transfers_and_batch_refusal():
    torch = pytest.importorskip("torch")
    wl = _wl(3, 3, (5, 4, 3), (1.0, 1.0, 1.0), 1e-3, 1)
    w = inputs.random_modal_state(wl, seed=5)
    sim = dgx.Simulation(wl, precision=dgx.DG_FP32_BULK)
    dw = torch.from_numpy(w).cuda()
    dgx.dg_set_state_device(sim.h, dw.data_ptr())
    back = torch.zeros_like(dw)
    dgx.dg_get_state_device(sim.h, back.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(back, dw)
    with pytest.raises(dgx.DGError) as e:
        dgx.dg_batch_create([sim.h])
    assert e.value.code == dgx.DG_EUNSUPPORTED
    sim.close()
