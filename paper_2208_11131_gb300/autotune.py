"""Per-degree tile autotuner of the 2-D FP32-bulk stage kernel.

The stage kernel works on tiles of TX x TY cells plus their face-neighbour halo; the tile fixes the
halo overhead, the shared memory per CTA and so the CTAs resident per SM, and the balance of the
per-thread phases.  For every requested degree this tool

1. takes the current tile of that degree (the tables of csrc/dgx_inst_2d_f32.cu: DGX_TILES for the
   plain plans, DGX_TILES_TR for the plans with a passive tracer) and candidate tiles around it;
2. compiles one variant of the 2-D FP32 translation unit per candidate, the two tables defined in a
   pre-included header with that degree's stage tile replaced, and links it with the library's other
   objects (the in-tree build), all variants in parallel; a candidate whose tile does not fit in
   shared memory fails to compile and is skipped, one that fits fewer CTAs per SM times slower;
3. times each variant in a process of its own on the shear layer of that degree (about 4 M conserved
   DOFs; whole FP32-bulk steps timed with CUDA events on the launching stream, L2 flushed before
   every step), and reports the fastest; ``--write`` puts the winners into the tables.

    python -m paper_2208_11131_gb300.autotune --degrees 3 5 [--tracer] [--tiles 6x8,4x8] [--write]

Single simulations of degrees 1 and 3 without a tracer run the 2-D lane-group kernel, whose tile is
fixed by its lane mapping; the table tiles of those degrees serve the batched kernel.  The tool times
single simulations, so it skips the plain table at degrees 1 and 3.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import subprocess
import sys
import tempfile

from . import build as B

TU = os.path.join(B.CSRC, "dgx_inst_2d_f32.cu")
TABLES = ("DGX_TILES", "DGX_TILES_TR")
# shear-layer cells per axis that give about 4 M conserved DOFs at each degree
CELLS = {0: 1024, 1: 512, 2: 384, 3: 256, 4: 200, 5: 160}
# degrees whose single-simulation plans without a tracer run the lane-group kernel (not the tiled one)
LANE_GROUP_DEGREES = (1, 3)
_ENTRY = re.compile(r"X\(\s*(\d+)\s*,\s*(\d+)\s*,\s*(\d+)\s*,\s*(\d+)\s*,\s*(\d+)\s*,\s*(\d+)\s*,\s*(\d+)\s*\)")


def _block(text: str, name: str):
    """(start, end) of the entries of `#define name(X) ...` (the macro's continued lines)"""
    m = re.search(r"#define %s\(X\) \\\n" % name, text)
    if not m:
        raise ValueError(f"no table {name}")
    end = m.end()
    while True:
        nl = text.index("\n", end)
        line = text[end:nl]
        end = nl + 1
        if not line.rstrip().endswith("\\"):
            return m.end(), nl


def read_tables(text: str) -> dict:
    """{table name: {degree: (stage TX, TY, TZ, prologue TX, TY, TZ)}}"""
    out = {}
    for name in TABLES:
        a, b = _block(text, name)
        out[name] = {int(g[0]): tuple(int(x) for x in g[1:]) for g in _ENTRY.findall(text[a:b])}
    return out


def table_body(entries: dict) -> str:
    """the macro body of a table, three entries per line"""
    items = [f"X({n}, {', '.join(str(v) for v in entries[n])})" for n in sorted(entries)]
    lines = [" ".join(items[i:i + 3]) for i in range(0, len(items), 3)]
    return " \\\n".join("    " + l for l in lines)


def write_tables(text: str, tables: dict) -> str:
    for name in TABLES:
        a, b = _block(text, name)
        text = text[:a] + table_body(tables[name]) + text[b:]
    return text


def header(tables: dict) -> str:
    """a header defining both tables (pre-included by a variant build)"""
    out = []
    for name in TABLES:
        items = "".join(f"X({n},{','.join(str(v) for v in tables[name][n])})" for n in sorted(tables[name]))
        out.append(f"#define {name}(X) {items}\n")
    return "".join(out)


def candidates(tx: int, ty: int, reach: int = 2) -> list:
    """the tile (tx, ty) first, then every tile within `reach` cells of it along each axis (2..16
    cells per axis), nearest first"""
    out = [(tx, ty)]
    near = sorted(((a, b) for a in range(max(2, tx - reach), min(16, tx + reach) + 1)
                   for b in range(max(2, ty - reach), min(16, ty + reach) + 1)),
                  key=lambda t: (abs(t[0] - tx) + abs(t[1] - ty), t))
    out += [t for t in near if t not in out]
    return out


def with_tile(tables: dict, name: str, degree: int, tile) -> dict:
    t = {k: dict(v) for k, v in tables.items()}
    e = t[name][degree]
    t[name][degree] = (tile[0], tile[1], 1) + e[3:]
    return t


def build_variants(variants: dict, workdir: str, jobs: int | None = None) -> dict:
    """{tag: tables} -> {tag: path of the variant library}, compile failures left out; at most `jobs`
    compilations at a time (default: the host's cores)"""
    lib = B.build()  # the in-tree objects of the other translation units
    common = [os.path.join(B.BUILD, f[:-3] + ".o") for f in sorted(os.listdir(B.CSRC))
              if f.endswith(".cu") and f != os.path.basename(TU)]
    assert os.path.exists(lib) and all(os.path.exists(o) for o in common)
    nvcc = B._nvcc()
    jobs = max(1, jobs or os.cpu_count() or 1)
    pending = list(variants.items())
    running, done = {}, {}
    while pending or running:
        while pending and len(running) < jobs:
            tag, tables = pending.pop(0)
            h = os.path.join(workdir, f"tiles_{tag}.h")
            with open(h, "w") as f:
                f.write(header(tables))
            obj = os.path.join(workdir, f"v_{tag}.o")
            cmd = [nvcc] + B.ARCH + B.FLAGS + ["--use_fast_math", "--pre-include", h, "-c", TU, "-o", obj]
            log = open(obj + ".log", "w")
            running[tag] = (subprocess.Popen(cmd, stdout=log, stderr=subprocess.STDOUT), obj, log)
        tag = next(iter(running))  # wait for the oldest compilation
        p, obj, log = running.pop(tag)
        rc = p.wait()
        log.close()
        done[tag] = obj if rc == 0 else None
    libs = {}
    for tag in variants:
        if done.get(tag) is None:
            continue
        so = os.path.join(workdir, f"lib_{tag}.so")
        subprocess.run([nvcc] + B.ARCH + ["-shared", "-o", so] + common + [done[tag], "-lcudart"], check=True)
        libs[tag] = so
    return libs


def time_library(path: str, degree: int, tracer: bool, steps: int, warmup: int) -> float:
    """ms per whole FP32-bulk step of the degree's shear layer with the library at `path` (call in a
    process of its own: a process loads one library)"""
    import numpy as np
    import torch

    from . import dgx, inputs

    dgx.lib(path)
    wl = inputs.c2_shear_layer(N=CELLS[degree], n=degree)
    w0 = inputs.project(wl, inputs.shear_layer_ic(wl))
    if tracer:  # a dye: rho c = rho / 2 in the cell means
        wl = wl.with_(tracer_on=1, eta=1e-5)
        rc = np.zeros_like(w0[0])
        rc[:, 0] = 0.5 * w0[0, :, 0]
        w0 = np.ascontiguousarray(np.concatenate([w0[:4], rc[None], w0[4:]]))
    sim = dgx.Simulation(wl, precision=dgx.DG_FP32_BULK)
    sim.set_stream(torch.cuda.current_stream().cuda_stream)
    sim.set_state(w0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        dgx.dg_step_timed(sim.h, 0.0, 7)
    ms = []
    for k in range(steps):
        flush.fill_(k & 0xFF)
        ms.append(sum(dgx.dg_step_timed(sim.h, 0.0, 7)))
    sim.close()
    return float(np.mean(ms))


def tune(degrees, tracer: bool, tiles=None, steps: int = 20, warmup: int = 5, reach: int = 2,
         workdir: str | None = None) -> dict:
    """time the candidates of every degree; returns {degree: {"current": tile, "best": tile,
    "ms": {tile: ms per step}}} with tiles as "TXxTY" strings"""
    name = TABLES[1] if tracer else TABLES[0]
    tables = read_tables(open(TU).read())
    if workdir is None:
        os.makedirs(os.path.join(B.BUILD, "tune"), exist_ok=True)
        workdir = tempfile.mkdtemp(prefix="run_", dir=os.path.join(B.BUILD, "tune"))
    plan = {}
    if not tracer:
        degrees = [n for n in degrees if n not in LANE_GROUP_DEGREES]
    for n in degrees:
        cur = tables[name][n][:2]
        cands = [tuple(int(v) for v in t.split("x")) for t in tiles] if tiles else candidates(*cur, reach)
        if cur not in cands:
            cands = [cur] + cands
        for t in cands:
            plan[f"n{n}_{t[0]}x{t[1]}"] = (n, t, with_tile(tables, name, n, t))
    libs = build_variants({tag: v[2] for tag, v in plan.items()}, workdir)
    report = {}
    for tag, (n, t, _) in plan.items():
        r = report.setdefault(n, {"current": "%dx%d" % tables[name][n][:2], "ms": {}})
        if tag not in libs:
            r["ms"]["%dx%d" % t] = None  # does not compile (shared memory)
            continue
        out = subprocess.run([sys.executable, "-m", "paper_2208_11131_gb300.autotune", "--time", libs[tag],
                              "--degree", str(n), "--steps", str(steps), "--warmup", str(warmup)] +
                             (["--tracer"] if tracer else []),
                             capture_output=True, text=True, cwd=B.ROOT)
        if out.returncode != 0:
            raise RuntimeError(f"timing {tag} failed:\n{out.stderr[-2000:]}")
        r["ms"]["%dx%d" % t] = json.loads(out.stdout.strip().splitlines()[-1])["ms"]
    for n, r in report.items():
        timed = {k: v for k, v in r["ms"].items() if v is not None}
        r["best"] = min(timed, key=timed.get)
    return report


def apply(report: dict, tracer: bool) -> None:
    """write the fastest tile of every tuned degree into the tables"""
    name = TABLES[1] if tracer else TABLES[0]
    text = open(TU).read()
    tables = read_tables(text)
    for n, r in report.items():
        tables = with_tile(tables, name, int(n), tuple(int(v) for v in r["best"].split("x")))
    with open(TU, "w") as f:
        f.write(write_tables(text, tables))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--degrees", type=int, nargs="*", default=[0, 1, 2, 3, 4, 5],
                    help="degrees to tune (the plain table skips 1 and 3, see above)")
    ap.add_argument("--tracer", action="store_true", help="tune the tiles of the plans with a passive tracer")
    ap.add_argument("--tiles", help="candidate tiles, e.g. 6x8,4x8 (default: the current tile and its neighbours)")
    ap.add_argument("--reach", type=int, default=2, help="neighbour candidates within this many cells per axis")
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--write", action="store_true", help="write the winners into csrc/dgx_inst_2d_f32.cu")
    ap.add_argument("--time", help=argparse.SUPPRESS)  # internal: time one variant library
    ap.add_argument("--degree", type=int, help=argparse.SUPPRESS)
    a = ap.parse_args(argv)
    if a.time:
        print(json.dumps({"ms": time_library(a.time, a.degree, a.tracer, a.steps, a.warmup)}), flush=True)
        return
    report = tune(a.degrees, a.tracer, a.tiles.split(",") if a.tiles else None, a.steps, a.warmup, a.reach)
    print(json.dumps({"table": TABLES[1] if a.tracer else TABLES[0], "degrees": report}), flush=True)
    if a.write:
        apply(report, a.tracer)


if __name__ == "__main__":
    main()
