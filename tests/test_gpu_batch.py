"""Batched ensembles (one persistent stage kernel per group over all members' tiles, per-member
device dt, graph replay) against the same members stepped one by one, FP64 and FP32-bulk,
including the graph path and an odd leftover step.

The batched and the single-simulation stage kernels are separate compilations of one body, so the
compiler may contract a different set of multiply-adds into FMAs: the two agree to rounding, not
bit for bit.  The first step's dt depends only on the common initial state and a maximum, so it is
equal exactly."""
import numpy as np
import pytest

import oracle
from paper_2208_11131_gb300 import build as B
from paper_2208_11131_gb300 import dgx, inputs

from .helpers import problem, state_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    dgx.lib()


def small_members():
    specs = [(16, 1, "wave", 0, 0.0), (24, 2, "sod", 0, 1e-3), (16, 3, "wave", 0, 1e-3), (20, 3, "sod", 1, 0.0),
             (12, 2, "wave", 0, 0.0), (16, 5, "sod", 1, 1e-3), (8, 4, "wave", 0, 0.0), (16, 1, "sod", 1, 0.0)]
    out = []
    for i, (N, n, kind, axis, nu) in enumerate(specs):
        bc = (0, 0, 0) if kind == "wave" else ((1, 0, 0) if axis == 0 else (0, 1, 0))
        g = 5.0 / 3.0 if kind == "wave" else 1.4
        # shock-tube members run with the positivity limiter (Sec. 4.2), as in the ensemble workload
        wl = inputs.Workload(f"m{i}", 2, n, (N, N, 1), (0, 0, 0), (1.0, 1.0, 1.0), bc=bc, gamma=g, nu=nu, kappa=nu,
                             av_on=1, cfl=0.3, positivity_on=1 if kind == "sod" else 0)
        out.append(inputs.Member(wl, kind, axis))
    return out


@pytest.mark.parametrize("prec,tol", [(dgx.DG_FP64, 1e-13), (dgx.DG_FP32_BULK, 2e-5)])
def test_batch_equals_members_stepped_alone(prec, tol):
    members = small_members()
    a = [dgx.Simulation(m.wl, precision=prec) for m in members]
    b = [dgx.Simulation(m.wl, precision=prec) for m in members]
    for sa, sb, m in zip(a, b, members):
        w0 = inputs.member_state(m)
        sa.set_state(w0)
        sb.set_state(w0)
    batch = dgx.dg_batch_create([s.h for s in b])

    def advance(k):
        for s in a:
            for _ in range(k):
                s.step()
        dgx.dg_batch_step(batch, k)
        dgx.dg_batch_sync(batch)

    def compare(exact_dt):
        for sa, sb, m in zip(a, b, members):
            P = problem(m.wl)
            wa = sa.get_state()
            assert state_err(sb.get_state(), wa, P) < tol
            Sa, ga, ca = sa.get_aux()
            Sb, gb, cb = sb.get_aux()
            assert ca[1] == cb[1]  # step counter
            if exact_dt:
                assert ca[0] == cb[0]
            assert abs(ca[0] - cb[0]) <= 50 * tol * ca[0] and abs(ca[2] - cb[2]) <= 50 * tol * ca[2]

    advance(1)  # one step outside the graph
    compare(True)
    advance(4)  # one graph of two steps, replayed twice
    compare(False)
    advance(3)  # from the odd parity: one step, then the graph once
    compare(False)
    dgx.dg_batch_destroy(batch)
    for s in a + b:
        s.close()


def test_batch_members_match_oracle():
    members = small_members()[:4]
    sims = [dgx.Simulation(m.wl) for m in members]
    refs = []
    for s, m in zip(sims, members):
        w0 = inputs.member_state(m)
        s.set_state(w0)
        refs.append(oracle.Sim(problem(m.wl), w0))
    batch = dgx.dg_batch_create([s.h for s in sims])
    dgx.dg_batch_step(batch, 4)
    dgx.dg_batch_sync(batch)
    for s, r, m in zip(sims, refs, members):
        for _ in range(4):
            _, st = r.step()
            assert st == 0
        assert state_err(s.get_state(), r.w, problem(m.wl)) < 1e-11
    dgx.dg_batch_destroy(batch)
    for s in sims:
        s.close()


def test_batch_with_limiter_members_matches_oracle():
    """limiter members form groups of their own (separate step prologue per member, limiter after
    every batched stage) next to the folded-prologue groups of the other members"""
    members = [m for m in small_members() if m.kind == "sod"][:2] + [small_members()[0]]
    assert any(m.wl.positivity_on for m in members) and not all(m.wl.positivity_on for m in members)
    sims = [dgx.Simulation(m.wl) for m in members]
    refs = []
    for s, m in zip(sims, members):
        w0 = inputs.member_state(m)
        s.set_state(w0)
        refs.append(oracle.Sim(problem(m.wl), w0))
    batch = dgx.dg_batch_create([s.h for s in sims])
    dgx.dg_batch_step(batch, 5)
    dgx.dg_batch_sync(batch)
    for s, r, m in zip(sims, refs, members):
        for _ in range(5):
            _, st = r.step()
            assert st == 0
        assert state_err(s.get_state(), r.w, problem(m.wl)) < 1e-11
    dgx.dg_batch_destroy(batch)
    for s in sims:
        s.close()


def test_batch_rejects_forced_members():
    wl = inputs.c4_turbulence_box(N=4, n=1)
    s = dgx.Simulation(wl)
    with pytest.raises(dgx.DGError) as e:
        dgx.dg_batch_create([s.h])
    assert e.value.code == dgx.DG_EUNSUPPORTED
    s.close()
