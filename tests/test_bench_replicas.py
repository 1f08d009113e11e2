"""The multi-process path of bench.py on CPU: two gloo ranks (one process each, as torchrun starts
them) run the replica logic the GPU runs use -- process-group set-up from the environment, the
barrier, the maximum of the ranks' times, the whole-job value (units of all ranks over the slowest
rank's time) -- and the oracle arm, which rank 0 alone runs and prints while the other rank returns
without work.  The oracle arm runs on a tiny shear layer so that the test takes seconds."""
import argparse
import contextlib
import io
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank), DGX_BENCH_BACKEND="gloo", OMP_NUM_THREADS="1")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_2208_11131_gb300 import inputs

    r, w, local = bench.dist_init()
    assert (r, w, local) == (rank, ws, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    local_ms = 10.0 * (rank + 1)  # rank 1 is the slow one
    total_ms, value = bench.job_value(local_ms, 1000, w)
    wl = inputs.c2_shear_layer(N=8, n=3)
    bench.workload = lambda name=None: (wl, lambda: inputs.project(wl, inputs.shear_layer_ic(wl)), "tiny")
    bench.sample_workload = lambda name, cells=None: (wl, inputs.project(wl, inputs.shear_layer_ic(wl)))
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.reference_arm(argparse.Namespace(warmup=1, steps=2, gpus=w), r, w)
    bench.barrier(w)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"total_ms": total_ms, "value": value, "stdout": buf.getvalue()}, f)


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    ws = 2
    mp.start_processes(_rank, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    for r in res:
        assert r["total_ms"] == 20.0  # the slowest rank's time on every rank
        assert r["value"] == pytest.approx(1000 * ws / 0.020)
    assert res[1]["stdout"] == ""  # rank 1: no work, no line
    lines = [l for l in res[0]["stdout"].splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == ws and line["steps"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0
