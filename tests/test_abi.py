"""The C-ABI library loads and exports every entry point that include/dgx.h declares (CPU only:
no compute call needs a GPU here)."""
import ctypes
import os
import re

import pytest

from paper_2208_11131_gb300 import build as B
from paper_2208_11131_gb300 import dgx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return dgx.lib()


def declared():
    txt = open(os.path.join(ROOT, "include", "dgx.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary_calls():
    names = declared()
    for required in ("dg_create", "dg_set_state", "dg_rhs", "dg_step", "dg_get_state", "dg_max_dt"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert names
    for n in names:
        assert hasattr(L, n), n
    assert sorted(dgx.EXPORTS) == names


def test_default_params_are_the_papers(L):
    p = dgx.dg_default_params()
    assert (p.av_scale, p.f_v, p.f_tau, p.f_w, p.s_onset, p.cfl) == (1.0, 2.5, 0.5, 0.2, 1e-4, 0.5)
    assert p.precision == dgx.DG_FP64 and p.rk_stages == 0 and p.av_on == 0


def test_invalid_arguments_rejected_before_any_device_call(L):
    h = ctypes.c_void_p()
    g = dgx.make_grid(4, (4, 4, 4), (0, 0, 0), (1, 1, 1))
    assert L.dg_create(ctypes.byref(g), 2, 1.4, 0.0, 0.0, ctypes.byref(h)) == dgx.DG_EINVAL
    g = dgx.make_grid(2, (4, 0), (0, 0), (1, 1))
    assert L.dg_create(ctypes.byref(g), 2, 1.4, 0.0, 0.0, ctypes.byref(h)) == dgx.DG_EINVAL
    g = dgx.make_grid(2, (4, 4), (0, 0), (1, 1))
    assert L.dg_create(ctypes.byref(g), 9, 1.4, 0.0, 0.0, ctypes.byref(h)) == dgx.DG_EINVAL
    assert L.dg_create(ctypes.byref(g), 2, 1.0, 0.0, 0.0, ctypes.byref(h)) == dgx.DG_EINVAL
    assert L.dg_create(ctypes.byref(g), 2, 1.4, -1.0, 0.0, ctypes.byref(h)) == dgx.DG_EINVAL
    assert L.dg_step(None, 0.0) == dgx.DG_EINVAL
    assert L.dg_default_params(None) == dgx.DG_EINVAL
    assert L.dg_status_string(dgx.DG_ENONPHYS) == b"non-physical state"


def test_noalloc_rejects_grids_beyond_its_static_scratch_before_any_device_call(L):
    """dg_max_dt_noalloc keeps one slot per time-step tile in a fixed 2^18-slot device array; a grid
    that needs more tiles is refused on the host before any CUDA call (the pointers are never
    touched).  3-D FP64 degree-5 time-step tiles are 2 x 2 x 1 cells, so 130 x 128 x 64 cells need
    65 * 64 * 64 = 266,240 tiles."""
    g = dgx.make_grid(3, (130, 128, 64), (0, 0, 0), (1, 1, 1))
    fake = ctypes.c_void_p(0x1000)
    code = L.dg_max_dt_noalloc(ctypes.byref(g), 5, 1.4, 0.3, fake, fake, None)
    assert code == dgx.DG_EUNSUPPORTED
    # one tile fewer than the limit along z passes the size check (it then needs a device, so only
    # the size rule is checked here: 65 * 64 * 63 tiles are within 2^18)
    assert 65 * 64 * 63 <= 1 << 18 < 65 * 64 * 64
