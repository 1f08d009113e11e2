"""Failure paths of the library, injected on the host (no device fault is ever provoked).

DGX_FAULT=alloc:K makes the K-th device allocation of a handle's buffer set-up fail as if
cudaMalloc had run out of memory, without calling it: dg_create must return DG_ENOMEM, release
every buffer it had already taken, and leave the library usable."""
import os

import numpy as np
import pytest

from paper_2208_11131_gb300 import build as B
from paper_2208_11131_gb300 import dgx, inputs

pytestmark = pytest.mark.gpu


def test_injected_allocation_failure_gives_enomem_and_leaks_nothing():
    torch = pytest.importorskip("torch")
    B.build()
    wl = inputs.c2_shear_layer(N=32, n=3)
    w = inputs.project(wl, inputs.shear_layer_ic(wl))
    dgx.Simulation(wl, precision=dgx.DG_FP32_BULK).close()  # kernels loaded, set-up done
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    # dg_create allocates the FP64 buffers (11 allocations); dg_set_params (FP32-bulk, AV)
    # reallocates everything (13): k <= 11 fails inside dg_create, k = 12 inside dg_set_params
    for k in (1, 2, 5, 9, 12):
        os.environ["DGX_FAULT"] = f"alloc:{k}"
        try:
            with pytest.raises(dgx.DGError) as ei:
                dgx.Simulation(wl, precision=dgx.DG_FP32_BULK)
            assert ei.value.code == dgx.DG_ENOMEM, (k, ei.value)
        finally:
            del os.environ["DGX_FAULT"]
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (k, free0 - free1)
    # the library works normally afterwards
    sim = dgx.Simulation(wl, precision=dgx.DG_FP64)
    sim.set_state(w)
    sim.step()
    assert np.isfinite(sim.get_state()).all()
    sim.close()


def test_nonfinite_state_is_reported_as_nonphysical():
    """A NaN in the state handed to the library (a host-side fault of the caller) is caught at the
    Gauss points of the next step and reported through the status word, not by a trap."""
    B.build()
    wl = inputs.c1_density_wave(N=8, n=2)
    w = inputs.project(wl, inputs.density_wave_ic(wl, 0.0))
    w[2, 5, 1] = np.nan
    sim = dgx.Simulation(wl, precision=dgx.DG_FP64)
    sim.set_state(w)
    sim.step()
    with pytest.raises(dgx.DGError) as ei:
        sim.sync()
    assert ei.value.code == dgx.DG_ENONPHYS
    # the status word was cleared: a good state steps cleanly on the same handle
    sim.set_state(inputs.project(wl, inputs.density_wave_ic(wl, 0.0)))
    sim.step()
    sim.sync()
    sim.close()
