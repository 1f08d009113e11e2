"""Host logic of the tile autotuner (CPU only): the tile tables of the 2-D FP32 unit are read and
written back exactly, candidate tiles are the current tile and its neighbours, and a variant header
reaches the stage-kernel instantiations (checked on the preprocessed unit; no GPU)."""
import os
import re
import subprocess

import pytest

from paper_2208_11131_gb300 import autotune as T
from paper_2208_11131_gb300 import build as B


def test_tables_read_and_written_back_exactly():
    text = open(T.TU).read()
    t = T.read_tables(text)
    for name in T.TABLES:
        assert sorted(t[name]) == [0, 1, 2, 3, 4, 5]
        assert all(len(e) == 6 and e[2] == 1 for e in t[name].values())
    # the tracer table's prologue entries are those of the plain table (the prologue tiles are shared)
    assert all(t["DGX_TILES_TR"][n][3:] == t["DGX_TILES"][n][3:] for n in range(6))
    assert T.write_tables(text, t) == text
    t2 = T.with_tile(t, "DGX_TILES", 3, (4, 9))
    assert t2["DGX_TILES"][3] == (4, 9, 1) + t["DGX_TILES"][3][3:] and t["DGX_TILES"][3] != t2["DGX_TILES"][3]
    assert T.read_tables(T.write_tables(text, t2)) == t2


def test_candidates():
    c = T.candidates(6, 8)
    assert c[0] == (6, 8) and len(c) == len(set(c)) == 25
    assert all(4 <= a <= 8 and 6 <= b <= 10 for a, b in c)
    c = T.candidates(16, 2, reach=1)
    assert c[0] == (16, 2) and set(c) == {(a, b) for a in (15, 16) for b in (2, 3)}


def test_variant_header_reaches_the_instantiations(tmp_path):
    t = T.with_tile(T.read_tables(open(T.TU).read()), "DGX_TILES", 3, (4, 9))
    t = T.with_tile(t, "DGX_TILES_TR", 5, (3, 4))
    h = tmp_path / "tiles.h"
    h.write_text(T.header(t))
    out = subprocess.run([B._nvcc()] + B.ARCH + B.FLAGS + ["--pre-include", str(h), "-E", T.TU],
                         capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("nvcc preprocessing unavailable: " + out.stderr[-200:])
    pp = re.sub(r"\s+", "", out.stdout)
    assert "run_stage_2d_f32_any<2,3,float,4,9,1,false>" in pp
    assert "run_stage_2d_f32_any<2,5,float,3,4,1,true>" in pp
    assert "run_stage_2d_f32_any<2,3,float,6,8,1,false>" not in pp
