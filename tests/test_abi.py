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
