"""The allocation-free CFL time step (dg_max_dt_noalloc) against the handle-based dg_max_dt.

dg_max_dt_noalloc serves callers that cannot let a library call cudaMalloc (device memory owned
by their own pool, or loops that cannot take cudaMalloc's synchronisation): its scratch lives in
a static device array shared by all calls.  This file is collected last so that a failure here
comes after every other test has run; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2208_11131_gb300 import build as B
from paper_2208_11131_gb300 import dgx, inputs

pytestmark = pytest.mark.gpu

DT_TOL = 1e-14  # the tolerance of the dg_max_dt parity test (FP64)


def _dt_noalloc(torch, wl, w, cfl):
    grid = dgx.make_grid(wl.dim, wl.N[:wl.dim], wl.lo[:wl.dim], wl.hi[:wl.dim], wl.bc[:wl.dim])
    state = torch.from_numpy(np.ascontiguousarray(w)).cuda()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    dgx.dg_max_dt_noalloc(grid, wl.n, wl.gamma, cfl, state.data_ptr(), out.data_ptr(), stream)
    torch.cuda.synchronize()
    return float(out.item())


def _dt_handle(wl, w):
    sim = dgx.Simulation(wl, precision=dgx.DG_FP64)
    sim.set_state(w)
    dt = sim.max_dt()
    sim.close()
    return dt


def test_noalloc_dt_matches_handle_dt_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    B.build()
    cases = [
        inputs.c2_shear_layer(N=64, n=3),
        inputs.Workload("box3d", 3, 2, (9, 7, 5), (0, 0, 0), (1.0, 0.7, 0.5), gamma=1.4, cfl=0.3, av_on=1),
    ]
    states = [inputs.project(cases[0], inputs.shear_layer_ic(cases[0])),
              inputs.random_modal_state(cases[1], seed=4)]
    for wl, w in zip(cases, states):
        ref = _dt_handle(wl, w)
        first = _dt_noalloc(torch, wl, w, wl.cfl)
        second = _dt_noalloc(torch, wl, w, wl.cfl)
        assert abs(first / ref - 1.0) < DT_TOL
        assert abs(second / ref - 1.0) < DT_TOL


def test_noalloc_reports_nonphysical_state_then_recovers():
    torch = pytest.importorskip("torch")
    B.build()
    wl = inputs.c1_density_wave(N=16, n=2)
    w = inputs.project(wl, inputs.density_wave_ic(wl, 0.0))
    bad = w.copy()
    bad[0, 3, 0] = -1.0
    assert np.isnan(_dt_noalloc(torch, wl, bad, 0.3))
    # the shared status word is cleared by the next call
    good = _dt_noalloc(torch, wl, w, 0.3)
    assert abs(good / _dt_handle(wl, w) - 1.0) < DT_TOL


def test_noalloc_call_allocates_no_device_memory():
    """The entry point's reason to exist: after the first call on a device (which may load the
    library's kernels there), further calls leave the device's free memory unchanged."""
    torch = pytest.importorskip("torch")
    B.build()
    wl = inputs.c2_shear_layer(N=64, n=3)
    w = inputs.project(wl, inputs.shear_layer_ic(wl))
    grid = dgx.make_grid(wl.dim, wl.N[:wl.dim], wl.lo[:wl.dim], wl.hi[:wl.dim], wl.bc[:wl.dim])
    state = torch.from_numpy(np.ascontiguousarray(w)).cuda()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    dgx.dg_max_dt_noalloc(grid, wl.n, wl.gamma, wl.cfl, state.data_ptr(), out.data_ptr(), stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        dgx.dg_max_dt_noalloc(grid, wl.n, wl.gamma, wl.cfl, state.data_ptr(), out.data_ptr(), stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert abs(float(out.item()) / _dt_handle(wl, w) - 1.0) < DT_TOL
