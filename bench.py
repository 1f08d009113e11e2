#!/usr/bin/env python
"""Throughput of the DG hot path: DOF-updates/s of whole SSP-RK steps on one GB300.

Workload (default): the 3-D driven subsonic turbulence box of Sec. 7, 128^3 periodic cells, degree 3
(64 modes/cell), 5 conserved fields + alpha, gamma = 1.001, nu = kappa = 1e-4, artificial viscosity
on, Ornstein-Uhlenbeck driving on, SSP(5,4), CFL 0.5, FP32-bulk arithmetic with FP64 state
accumulation.  The timed state starts turbulent: a seeded solenoidal velocity field of the wave
vectors 1 <= |k| <= 3 scaled to rms Mach 0.3 (uniform density 1, pressure 1/gamma).  A "step" is one
whole Runge-Kutta step: the driving update and field, five fused right-hand-side/stage kernels (the
first also doing the step prologue: sensor, wiggle source, CFL speeds of u^n; the second starting
with the dt reduction).  DOF-updates per step = cells x modes x 5 conserved fields x 5 stages.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dgx|reference] [--precision fp32|fp64]
                  [--workload NAME]

Timing: W untimed steps, then K steps, each timed on the device with CUDA events recorded by the
library around its own launches (dg_step_timed), with an L2 flush (a 256 MiB device write) before
each timed step, outside the events (the step's working set exceeds L2 in any case).  Barrier +
synchronize on both sides, max over ranks.  N > 1 runs independent replicas (the path is sharded by
whole simulations; no collective on the data path), `value` is the sum of the units all ranks
processed over the slowest rank's time.  --impl reference times the FP64 CPU oracle on the host
cores (rank 0 only) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s per GB300 (FP32-bulk vs FP64, same L1 error) + % HBM roofline"
UNIT = "DOF-updates/s"
FLUSH_BYTES = 256 << 20
KERNEL_SRCS = [os.path.join(ROOT, "paper_2208_11131_gb300", "csrc", f)
               for f in ("dgx_internal.h", "dgx_kernels.cuh", "dgx_stage2.cuh", "dgx_stage3z.cuh", "dgx_stage2t.cuh", "dgx_limiter.cuh",
                         "dgx_inst.cuh", "dgx_inst_2d_f32.cu", "dgx_inst_3d_f32.cu", "dgx_inst_3d_packed_f32.cu", "dgx_inst_3d_f64.cu")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="dgx", choices=["dgx", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-extras", action="store_true", help="skip the fp64 side run, e2e and cpu baseline")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched 64-member ensemble measurement")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS),
                    help="workload of the main measurement (the extras run with the default one only)")
    return ap.parse_args()


# name -> (label, workload factory, initial modes, description of the initial state)
WORKLOADS = {
    "turbulence_box_128": ("driven_turbulence_3d_128cubed_deg3_av_ns_forcing_mach0.3",
                           lambda inputs: inputs.c4_turbulence_box(N=128, n=3),
                           lambda inputs, wl: inputs.turbulence_ic_state(wl),
                           "solenoidal random velocity, 1 <= |k| <= 3, rms Mach 0.3, rho = 1, p = 1/gamma"),
    "turbulence_box_64": ("driven_turbulence_3d_64cubed_deg3_av_ns_forcing_mach0.3",
                          lambda inputs: inputs.c4_turbulence_box(N=64, n=3),
                          lambda inputs, wl: inputs.turbulence_ic_state(wl),
                          "solenoidal random velocity, 1 <= |k| <= 3, rms Mach 0.3, rho = 1, p = 1/gamma"),
    "shear_layer_256": ("ns_shear_layer_2d_256x256_deg3_av",
                        lambda inputs: inputs.c2_shear_layer(N=256, n=3),
                        lambda inputs, wl: inputs.project(wl, inputs.shear_layer_ic(wl)),
                        "smooth Kelvin-Helmholtz shear layer of Sec. 6"),
    "sod_blast_64": ("sod_plane_blast_3d_64cubed_deg3_av_limiter",
                     lambda inputs: inputs.c3_sod_blast(N=64, n=3),
                     lambda inputs, wl: inputs.project(wl, inputs.sod_blast_ic(wl)),
                     "Sod plane (1, 1 | 0.125, 0.1) across a seeded plane + blast p = 100 in r < 0.1"),
}
DEFAULT_WORKLOAD = "turbulence_box_128"


def workload(name: str = DEFAULT_WORKLOAD):
    from paper_2208_11131_gb300 import inputs
    label, make, ic, _ = WORKLOADS[name]
    wl = make(inputs)
    return wl, (lambda: ic(inputs, wl)), label


def config_of(wl, extra=None, label=WORKLOADS[DEFAULT_WORKLOAD][0]):
    desc = {v[0]: v[3] for v in WORKLOADS.values()}.get(label)
    cfg = {"workload": label, "cells": list(wl.N[:wl.dim]), "degree": wl.n,
           "fields": wl.nfields, "conserved_dofs": wl.dofs, "rk_stages": 5, "nu": wl.nu, "kappa": wl.kappa,
           "gamma": wl.gamma, "cfl": wl.cfl, "av": bool(wl.av_on), "driving": bool(wl.forcing_on),
           "positivity_limiter": bool(wl.positivity_on), "initial_state": desc,
           "l2": "flushed before every timed step (256 MiB device write)"}
    if extra:
        cfg.update(extra)
    return cfg


def stage_bytes_per_value(fp32: bool):
    """Algorithmic bytes per state value (field x cell x mode) for the five stage launches of SSP(5,4)
    in delta form: every array a stage must read once and write once.
      FP32-bulk: 1: u_hi, d0' | 2: u_hi, d0, d1' | 3: u_hi, d1, d2' | 4: u_hi, d2, x, d0', x' |
                 5: u_hi, d0, x, u (FP64), u' (FP64), u_hi'   -> 4-byte words except u, u'
      FP64:      u and every delta array are 8-byte words; no u_hi copies."""
    if fp32:
        return [8, 12, 12, 20, 4 + 4 + 4 + 8 + 8 + 4]
    return [16, 24, 24, 40, 8 + 8 + 8 + 8]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-i", str(self.index), "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_sha() -> str:
    """sha256 over the stage kernel's sources and the FP32 tile tables (a traffic figure is only used for
    the kernel and tiles it was taken on)"""
    h = hashlib.sha256()
    for f in KERNEL_SRCS:
        h.update(code_only(open(f).read()).encode())
    return h.hexdigest()


def code_only(src: str) -> str:
    """C++ source without comments and with whitespace runs collapsed (edits of comments alone do
    not change the kernel)"""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def counted_for(key: str, field: str):
    """a per-launch figure (`field`) of a committed ncu summary, if the kernel source is unchanged"""
    try:
        tab = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        return None
    ent = tab.get(key)
    if not ent or ent.get("kernel_sha256") != kernel_sha():
        return None
    return ent.get(field)


def traffic_for(key: str):
    """DRAM bytes per stage launch from a committed ncu summary, if the kernel source is unchanged."""
    try:
        tab = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        return None
    ent = tab.get(key)
    if not ent:
        return None
    sha = kernel_sha()
    return ent["bytes_per_launch"] if ent.get("kernel_sha256") == sha else None


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch.distributed as dist
    dist.init_process_group("nccl" if os.environ.get("DGX_BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return dist.get_rank(), ws, int(os.environ.get("LOCAL_RANK", "0"))


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, ws):
    """the maximum of x over the ranks (a device tensor under NCCL, a host one under gloo)"""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(local_ms, units_per_rank, ws):
    """whole-job throughput of ws replicas: the units all ranks processed over the slowest rank's
    time; returns (that time in ms, units per second)"""
    total_ms = allreduce_max(local_ms, ws)
    return total_ms, units_per_rank * ws / (total_ms / 1e3)


def l1_error_of(wl, w, func):
    """L1 density error against a closed form with the n+2 point rule of the error norm (Sec. 5.1)"""
    import numpy as np
    from numpy.polynomial import legendre as L
    q = wl.n + 2
    x, g = L.leggauss(q)
    d = wl.dim
    idx = np.stack(np.meshgrid(*([np.arange(q)] * d), indexing="ij")[::-1], -1).reshape(-1, d)
    xi, G = x[idx], np.prod(g[idx], 1)
    midx = np.stack(np.meshgrid(*([np.arange(wl.n + 1)] * d), indexing="ij")[::-1], -1).reshape(-1, d)
    phi = np.ones((len(xi), len(midx)))
    for a in range(d):
        Pt = np.stack([np.sqrt(2 * l + 1) * L.legval(xi[:, a], [0] * l + [1]) for l in range(wl.n + 1)], 1)
        phi *= Pt[:, midx[:, a]]
    axes = [wl.lo[a] + (np.arange(wl.N[a]) + 0.5) * wl.h[a] for a in range(d)]
    xc = np.stack([m.reshape(-1) for m in np.meshgrid(*axes[::-1], indexing="ij")[::-1]], 1)
    X = (xc[:, None, :] + 0.5 * np.array(wl.h[:d]) * xi[None]).reshape(-1, d)
    ex = np.asarray(func(X))[0].reshape(wl.ncell, len(xi))
    num = w[0] @ phi.T
    return float(np.sum(np.abs(ex - num) * G[None, :]) / 2.0 ** d / wl.ncell)


def oracle_problem(wl):
    import oracle
    return oracle.Problem(dim=wl.dim, n=wl.n, N=tuple(wl.N[:wl.dim]), lo=tuple(wl.lo[:wl.dim]),
                          hi=tuple(wl.hi[:wl.dim]), bc=tuple(wl.bc[:wl.dim]), gamma=wl.gamma, nu=wl.nu,
                          kappa=wl.kappa, av_on=wl.av_on, positivity_on=wl.positivity_on, cfl=wl.cfl,
                          forcing_on=wl.forcing_on, force_amp=wl.force_amp, force_ts=wl.force_ts,
                          force_dt=wl.force_dt, force_seed=wl.force_seed)


# the oracle's bounded sample of each workload: the same physics on a grid it steps in about a second
SAMPLE_CELLS = {"turbulence_box_128": 16, "turbulence_box_64": 16, "shear_layer_256": 256, "sod_blast_64": 16}


def sample_workload(name: str, cells: int | None = None):
    """the workload `name` on the oracle's sample grid (same degree, physics and initial-state recipe)"""
    from paper_2208_11131_gb300 import inputs
    label, make, ic, _ = WORKLOADS[name]
    full = make(inputs)
    N = SAMPLE_CELLS[name] if cells is None else cells
    wl = full.with_(N=tuple([N] * full.dim + [1] * (3 - full.dim)))
    return wl, ic(inputs, wl)


def run_oracle_steps(wl, w0, nsteps: int, seconds: float | None = None):
    """time whole oracle steps; returns (seconds, steps done, threads)"""
    import oracle
    P = oracle_problem(wl)
    if wl.positivity_on:
        oracle.positivity(P, w0)
    sim = oracle.Sim(P, w0)
    t0 = time.perf_counter()
    done = 0
    while done < nsteps:
        _, st = sim.step()
        if st != 0:
            raise RuntimeError(f"oracle step status {st}")
        done += 1
        if seconds is not None and time.perf_counter() - t0 > seconds:
            break
    return time.perf_counter() - t0, done, oracle.num_threads()


def cpu_baseline(name: str):
    """the oracle as it stands on the host cores: all cores on the workload's sample grid for about
    12 s, and one core on an 8-cell-per-axis (3-D) or 64^2 (2-D) grid for about 8 s"""
    import oracle
    wl, w0 = sample_workload(name)
    secs, done, cores = run_oracle_steps(wl, w0, 1000, seconds=12.0)
    out = {"value": wl.dofs * 5 * done / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{'x'.join(str(c) for c in wl.N[:wl.dim])} cells of the same workload (same degree, "
                     f"physics and initial-state recipe), {done} whole FP64 SSP(5,4) steps; per-DOF cost "
                     f"of the oracle does not depend on the grid size"}
    wl1, w1 = sample_workload(name, 8 if wl.dim == 3 else 64)
    prev = oracle.num_threads()
    oracle.set_threads(1)
    try:
        secs1, done1, _ = run_oracle_steps(wl1, w1, 1000, seconds=8.0)
    finally:
        oracle.set_threads(prev)
    out["one_core"] = {"value": wl1.dofs * 5 * done1 / secs1, "unit": UNIT, "cores": 1,
                       "sample": f"{'x'.join(str(c) for c in wl1.N[:wl1.dim])} cells, {done1} steps"}
    return out


def reference_arm(args, rank, ws):
    if rank != 0:
        return
    name = getattr(args, "workload", DEFAULT_WORKLOAD)
    wl_full, _, label = workload(name)
    wl, w0 = sample_workload(name)
    run_oracle_steps(wl, w0.copy(), args.warmup)
    secs, done, cores = run_oracle_steps(wl, w0.copy(), args.steps)
    units = wl.dofs * 5 * done
    value = units / secs
    sample = (f"{'x'.join(str(c) for c in wl.N[:wl.dim])} cells of the same workload, {done} whole FP64 SSP(5,4) "
              f"steps per timed run (the full grid takes minutes per oracle step)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": done, "warmup": args.warmup, "ms_per_step": 1e3 * secs / done, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(wl_full, {"engine": "FP64 CPU oracle (C, OpenMP)"}, label=label),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def alu_peaks():
    """FP32 and FP64 FMA-chain throughput (TFLOP/s) of this GPU, from the probe library built next to
    libdgx.so; None where it is missing"""
    import ctypes
    path = os.path.join(ROOT, "paper_2208_11131_gb300", "libdgxpeak.so")
    try:
        L = ctypes.CDLL(path)
    except OSError:
        return None
    L.dgx_fma_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    out = {}
    for name, fp64, iters in (("fp32_tflops", 0, 1 << 16), ("fp64_tflops", 1, 1 << 12)):
        v = ctypes.c_double()
        if L.dgx_fma_peak(fp64, iters, 5, ctypes.byref(v)) == 0:
            out[name] = v.value
    out["how"] = "FMA chains (8 per thread) over every SM, best of 5 launches, CUDA events"
    return out


def step_working_set_bytes(nvals: int, fp32: bool) -> int:
    """bytes of the state arrays one SSP(5,4) step touches: u^n and u^{n+1} (FP64), in the bulk mode
    their FP32 copies, and the three delta registers (stage precision)"""
    return nvals * ((8 + 8 + 4 + 4 + 3 * 4) if fp32 else (8 + 8 + 3 * 8))


def link_bandwidth(torch, host_in, host_out) -> dict:
    """host<->device copy rate of one plain pinned copy of the state's size each way (CUDA events on the
    current stream): the bound of the end-to-end figure's transfers"""
    dev = torch.empty(host_in.shape, dtype=host_in.dtype, device="cuda")
    out = {}
    for name, dst, src in (("h2d_gbs", dev, host_in), ("d2h_gbs", host_out, dev)):
        dst.copy_(src, non_blocking=True)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dst.copy_(src, non_blocking=True)
        e1.record()
        e1.synchronize()
        out[name] = host_in.numel() * host_in.element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del dev
    return out


def stage_roofline(nvals: int, ncell: int, fp32: bool, stage_ms: float, peak_gbs: float) -> dict:
    """HBM roofline of the stage launches of one SSP(5,4) step: algorithmic bytes (every array a stage
    reads once and writes once, plus the per-cell wiggle source) over the summed stage-launch time"""
    nbytes = nvals * sum(stage_bytes_per_value(fp32)) + 5 * 8 * ncell
    achieved = nbytes / (stage_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s", "frac": achieved / peak_gbs,
            "algorithmic_bytes_per_launch": nbytes / 5, "avg_launch_ms": stage_ms / 5}


def l2_bytes(device: int):
    """the device's L2 size in bytes, or None where the runtime does not report it"""
    try:
        import torch
        return int(getattr(torch.cuda.get_device_properties(device), "L2_cache_size"))
    except Exception:
        return None


def l2_resident(working_set: int, device: int):
    """whether a step's working set fits in L2 (None if the L2 size is unknown)"""
    l2 = l2_bytes(device)
    return None if l2 is None else working_set <= l2


def rk_stages_for(n: int) -> int:
    """default SSP-RK stage count of degree n (the library's choice when rk_stages is 0)"""
    return {0: 1, 1: 2, 2: 3}.get(n, 5)


def ensemble_measurement(dgx, inputs, torch, stream, steps: int, warmup: int, log2_cells=(6, 10), label=None):
    """64 independent 2-D runs of mixed size (64..512 cells per axis), degree (1..5) and physics
    (density wave / Sod tube, Euler+AV / NS+AV), FP32-bulk: whole SSP-RK steps of all members, batched
    (one persistent stage kernel per (degree, physics) group over every member's tiles, per-member
    device dt, CUDA graph) against the same members stepped one after another on the same stream.
    Both are timed with CUDA events on that stream around `steps` whole steps."""
    members = inputs.c5_manifest(count=64, log2_cells=log2_cells)
    sims = []
    for m in members:
        s = dgx.Simulation(m.wl, precision=dgx.DG_FP32_BULK)
        s.set_stream(stream)
        s.set_state(inputs.member_state(m))
        sims.append(s)
    units = sum(m.wl.dofs * rk_stages_for(m.wl.n) for m in members)
    state_bytes = sum(m.wl.nfields * m.wl.ncell * m.wl.M * (8 + 4) for m in members)  # u^n (FP64) + u_hi (FP32)
    batch = dgx.dg_batch_create([s.h for s in sims])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn(warmup)
        torch.cuda.synchronize()
        ev0.record()
        fn(steps)
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / steps

    def batched(k):
        dgx.dg_batch_step(batch, k)

    def separate(k):
        for _ in range(k):
            for s in sims:
                dgx.dg_step(s.h, 0.0)

    ms_b = timed(batched)
    ms_s = timed(separate)
    dgx.dg_batch_sync(batch)
    dgx.dg_batch_destroy(batch)
    for s in sims:
        s.close()
    return {"workload": label or "ensemble_64_mixed_2d_deg1to5_fp32bulk", "members": len(members),
            "cells_per_axis": sorted({m.wl.N[0] for m in members}),
            "dof_updates_per_step": units, "state_bytes": state_bytes, "steps": steps, "warmup": warmup,
            "batched": {"ms_per_step": ms_b, "value": units / (ms_b / 1e3), "unit": UNIT},
            "one_by_one": {"ms_per_step": ms_s, "value": units / (ms_s / 1e3), "unit": UNIT},
            "speedup": ms_s / ms_b,
            "l2": "not flushed; the members' state alone exceeds L2"}


def n_launches(wl, stages: int = 5) -> int:
    """kernel launches the library makes per step for a workload: the driving update and field (when
    driving is on), the stage kernels (the first with the step prologue folded in, unless the limiter
    is on: then a prologue, a dt reduction and a limiter after every stage and on the state entering
    the step)"""
    n = stages + (2 if wl.forcing_on else 0)
    if wl.positivity_on:
        n += 2 + stages + 1
    return n


def timed_steps(dgx, wl, w0, steps, warm, stream, flush, prec=None):
    """(per-step launch times [steps][7] in ms, state after) of whole steps through dg_step_timed"""
    sim = dgx.Simulation(wl, precision=dgx.DG_FP32_BULK if prec is None else prec)
    sim.set_stream(stream)
    sim.set_state(w0)
    for _ in range(warm):
        dgx.dg_step_timed(sim.h, 0.0, 7)
    per = []
    for k in range(steps):
        flush.fill_(k & 0xFF)
        per.append(dgx.dg_step_timed(sim.h, 0.0, 7))
    sim.sync()
    return per, sim


def path_line(wl, per, label, fp32=True, peak=None):
    """ms per step, value and the stage-launch HBM roofline of a measured path"""
    import numpy as np
    ms = float(np.mean([sum(x) for x in per]))
    stage_ms = float(np.mean([sum(x[2:]) for x in per]))
    out = {"workload": label, "ms_per_step": ms, "value": wl.dofs * 5 / (ms / 1e3), "unit": UNIT,
           "steps": len(per), "launch_ms_mean": [float(np.mean([x[i] for x in per])) for i in range(7)]}
    if peak:
        nvals = wl.nfields * wl.ncell * wl.M
        out["roofline"] = stage_roofline(nvals, wl.ncell, fp32, stage_ms, peak)
        out["working_set_bytes"] = step_working_set_bytes(nvals, fp32)
    return out


def side_workloads(dgx, inputs, oracle_l1, torch, stream, flush, peak):
    """throughput of the other paths at their own sizes (FP32-bulk, L2 flushed before each timed
    step): the 2-D NS shear layer (Sec. 6) and the same with a passive dye (Sec. 3.4), the 64^3 Sod
    plane + blast with the positivity limiter (Sec. 4.2; the limiter launches are inside the stage
    slots), and the metric's same-L1-error check on the 32^2 density wave."""
    import numpy as np
    out = {}
    for name, steps, warm in (("shear_layer_256", 20, 5), ("sod_blast_64", 6, 2)):
        wl, ic, label = workload(name)
        per, sim = timed_steps(dgx, wl, ic(), steps, warm, stream, flush)
        sim.close()
        out[name] = path_line(wl, per, label, True, peak)

    wl = inputs.c2_shear_layer(N=256, n=3).with_(tracer_on=1, eta=1e-5)
    w = inputs.project(wl.with_(tracer_on=0), inputs.shear_layer_ic(wl.with_(tracer_on=0)))
    # dye: concentration 1 in the lower-density layer (|y - 1| > 0.5) and 0 elsewhere, smoothed
    c = inputs.project(wl.with_(tracer_on=0, av_on=0), lambda X: np.stack(
        [0.5 * (np.tanh((np.abs(X[:, 1] - 1.0) - 0.5) / 0.05) + 1.0)] * 4))[0]
    rc = np.zeros_like(c)
    rc[:, 0] = w[0, :, 0] * c[:, 0]  # rho c from the cell means (a dye of the layers)
    w0 = np.ascontiguousarray(np.concatenate([w[:4], rc[None], w[4:]]))
    per, sim = timed_steps(dgx, wl, w0, 10, 3, stream, flush)
    sim.close()
    out["tracer"] = path_line(wl, per, "ns_shear_layer_2d_256x256_deg3_av_with_dye", True, peak)

    wl = inputs.c1_density_wave(N=32, n=2)
    w0 = inputs.project(wl, inputs.density_wave_ic(wl, 0.0))
    errs = {}
    for name, prec in (("fp64", dgx.DG_FP64), ("fp32", dgx.DG_FP32_BULK)):
        sim = dgx.Simulation(wl, precision=prec)
        sim.set_state(w0)
        for _ in range(20):
            sim.step()
        T = sim.get_aux()[2][2]
        errs[name] = oracle_l1(wl, sim.get_state(), inputs.density_wave_ic(wl, T))
        sim.close()
    out["same_l1_c1"] = {"workload": "density_wave_2d_32x32_deg2_20_steps", "l1_rho_fp64": errs["fp64"],
                         "l1_rho_fp32": errs["fp32"], "rel_diff": abs(errs["fp32"] / errs["fp64"] - 1)}
    return out


def dgx_arm(args, rank, ws, local):
    import numpy as np
    import torch

    from paper_2208_11131_gb300 import build as B
    from paper_2208_11131_gb300 import dgx, inputs

    torch.cuda.set_device(local)
    B.build()
    dgx.lib()
    wl, ic, label = workload(args.workload)
    w0 = ic()
    default = args.workload == DEFAULT_WORKLOAD
    fp32 = args.precision == "fp32"
    prec = dgx.DG_FP32_BULK if fp32 else dgx.DG_FP64
    stream = torch.cuda.current_stream().cuda_stream
    sim = dgx.Simulation(wl, precision=prec)
    sim.set_stream(stream)
    sim.set_state(w0)
    nl = 7
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        dgx.dg_step_timed(sim.h, 0.0, nl)
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    barrier(ws)
    clocks.start()
    time.sleep(0.25)
    per_launch = []
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        per_launch.append(dgx.dg_step_timed(sim.h, 0.0, nl))
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    barrier(ws)
    clk = clocks.stop()
    sim.sync()
    aux = sim.get_aux()
    state = sim.get_state()
    step_ms = [sum(x) for x in per_launch]
    total_ms, value = job_value(sum(step_ms), wl.dofs * 5 * args.steps, ws)
    stage_ms = sum(sum(x[2:]) for x in per_launch)
    launches = args.steps * 5
    bpv = stage_bytes_per_value(fp32)
    nvals = wl.nfields * wl.ncell * wl.M
    # per-cell wiggle source read by every stage (8 bytes per cell)
    stage_bytes = nvals * sum(bpv) + 5 * 8 * wl.ncell
    achieved = stage_bytes * args.steps / (stage_ms / 1e3) / 1e9
    peaks, peak_kind = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    key = f"stage_kernel|{label}|{'fp32' if fp32 else 'fp64'}"
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic_for(key), "peak_source": f"{peak_kind} hbm_gbs",
            "algorithmic_bytes_per_launch": stage_bytes / 5,
            "avg_launch_ms": stage_ms / launches,
            "share_of_step": stage_ms / sum(step_ms)}
    vel = state[1:1 + wl.dim, :, 0] / state[0, :, 0]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64", "data": "synthetic",
            "config": config_of(wl, label=label,
                                extra={"precision": "fp32-bulk (fp64 state and RK accumulation)" if fp32 else "fp64",
                                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                                       "working_set_bytes": step_working_set_bytes(nvals, fp32),
                                       "l2_bytes": l2_bytes(local),
                                       "l2_resident": l2_resident(step_working_set_bytes(nvals, fp32), local)}),
            "roofline": roof, "clocks": clk,
            "gpu_launches": args.steps * n_launches(wl),
            "launch_ms_mean": [float(np.mean([x[i] for x in per_launch])) for i in range(nl)],
            # host time of the timed loop: each step is one dg_step_timed call, which waits for the
            # step's last event, plus the L2 flush fill launched before it
            "wall_ms_per_step": 1e3 * t_wall / args.steps,
            "state_after_timed_steps": {"t": float(aux[2][2]), "steps_taken": int(aux[2][1]),
                                        "rms_cell_mean_speed": float(np.sqrt((vel ** 2).sum(0).mean()))}}

    if not args.no_extras and default:
        # end to end through the public C ABI with pinned host buffers: H2D state, one step, D2H state
        host_in = torch.from_numpy(w0).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        a_in, a_out = host_in.numpy(), host_out.numpy()
        e2e_steps = 3
        dgx.dg_set_state(sim.h, a_in)
        dgx.dg_step(sim.h, 0.0)
        dgx.dg_get_state(sim.h, a_out)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            dgx.dg_set_state(sim.h, a_in)
            dgx.dg_step(sim.h, 0.0)
            dgx.dg_get_state(sim.h, a_out)
        te = allreduce_max(time.perf_counter() - t0, ws)
        nbytes = a_in.nbytes
        line["e2e"] = {"value": wl.dofs * 5 * e2e_steps * ws / te, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                       "d2h_bytes_per_step": nbytes, "steps": e2e_steps,
                       "ms_per_step": 1e3 * te / e2e_steps, "link": link_bandwidth(torch, host_in, host_out)}
        del host_in, host_out, a_in, a_out
        # the other precision on the same workload, and the FP32-bulk vs FP64 difference
        other = dgx.Simulation(wl, precision=dgx.DG_FP64 if fp32 else dgx.DG_FP32_BULK)
        other.set_stream(stream)
        other.set_state(w0)
        ref = dgx.Simulation(wl, precision=prec)
        ref.set_stream(stream)
        ref.set_state(w0)
        ms_other = []
        nsteps_cmp = 6
        for k in range(nsteps_cmp):
            t = dgx.dg_step_timed(other.h, 0.0, nl)
            if k >= 2:
                ms_other.append(sum(t))
            ref.step()
        s_other, s_ref = other.get_state(), ref.get_state()
        a64, a32 = (s_other, s_ref) if fp32 else (s_ref, s_other)
        l1 = float(np.abs(a32[0] - a64[0]).sum() / np.abs(a64[0]).sum())
        other_ms = float(np.mean(ms_other))
        line["other_precision"] = {"dtype": "f64" if fp32 else "f32", "ms_per_step": other_ms,
                                   "value": wl.dofs * 5 / (other_ms / 1e3), "unit": UNIT,
                                   "steps": nsteps_cmp - 2}
        if fp32:
            # the FP64 path is bound by the FP64 arithmetic rate: executed FP64 flops per stage launch
            # (ncu: 2 x DFMA + DMUL + DADD thread instructions of the same kernel on this workload, per
            # cell, scaled to the grid) over the measured stage-launch time, against the FP64 FMA peak
            per_cell = counted_for(f"stage_kernel|{label}|fp64", "fp64_flops_per_cell")
            st64 = float(np.mean([sum(x[2:]) for x in [dgx.dg_step_timed(other.h, 0.0, nl) for _ in range(2)]]))
            pk = (alu_peaks() or {}).get("fp64_tflops")
            if per_cell and pk:
                ach = per_cell * wl.ncell * 5 / (st64 / 1e3) / 1e12
                line["other_precision"]["alu_roofline"] = {
                    "bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                    "peak_source": "measured FP64 FMA chains (bench alu_peaks)",
                    "flops_per_cell_per_launch": per_cell}
        line[f"fp32_vs_fp64_rel_l1_rho_after_{nsteps_cmp}_steps"] = l1
        other.close()
        ref.close()
        line["alu_peaks"] = alu_peaks()
        if rank == 0 and ws == 1:
            line["cpu_baseline"] = cpu_baseline(args.workload)
    sim.close()
    if not args.no_extras and default:
        # the paper's total-degree basis on the same box (Sec. 2.3): the headline's initial state
        # restricted to the modes l_x + l_y + l_z <= n, stored packed (20 of 64 modes per cell)
        wlt = wl.with_(basis=1)
        keep = [i for i, e in enumerate(inputs.mode_exponents(3, wl.n, 0)) if e.sum() <= wl.n]
        per, st = timed_steps(dgx, wlt, np.ascontiguousarray(w0[:, :, keep]), 6, 2, stream, flush)
        st.close()
        line["total_degree_basis"] = path_line(wlt, per, label + "_total_degree_basis", True, peak)
    if not args.no_ensemble and default:
        line["ensemble"] = ensemble_measurement(dgx, inputs, torch, stream, steps=20, warmup=3)
        # where batching pays: 64 members of 32^2 to 128^2 cells, each too small to fill the GPU alone
        line["ensemble_small"] = ensemble_measurement(dgx, inputs, torch, stream, steps=20, warmup=3,
                                                      log2_cells=(5, 8),
                                                      label="ensemble_64_small_2d_32to128_deg1to5_fp32bulk")
    if not args.no_extras and default and rank == 0:
        line["other_paths"] = side_workloads(dgx, inputs, l1_error_of, torch, stream, flush, peak)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, ws, local = dist_init()
    if args.impl == "reference":
        reference_arm(args, rank, ws)
    else:
        dgx_arm(args, rank, ws, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
