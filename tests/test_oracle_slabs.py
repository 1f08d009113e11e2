"""The oracle split into x-slabs over gloo ranks (CPU): every step of the decomposed run -- neighbour
layers exchanged before each stage's right-hand side, the time step from the maxima all-reduced over
the ranks -- is bitwise equal to the undecomposed oracle (the locality of Sec. 3.2 that the
multi-GPU exchange of Sec. 8.1-8.2 relies on)."""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    # name: (problem keyword arguments, initial state recipe, steps)
    "ns_av_3d_periodic": (dict(dim=3, n=2, N=(8, 4, 4), hi=(1.0, 0.5, 0.5), gamma=1.4, nu=2e-3, kappa=2e-3,
                               av_on=1, cfl=0.3), "random", 3),
    "sod_2d_outflow_limiter": (dict(dim=2, n=3, N=(16, 2), hi=(1.0, 0.125), bc=(1, 0), gamma=1.4, av_on=1,
                                    positivity_on=1, cfl=0.3), "sod", 4),
}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _setup(name):
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2208_11131_gb300 import inputs
    kw, recipe, steps = CASES[name]
    P = oracle.Problem(**kw)
    N = tuple(kw["N"]) + (1,) * (3 - kw["dim"])
    hi = tuple(kw["hi"]) + (1.0,) * (3 - kw["dim"])
    wl = inputs.Workload(name, kw["dim"], kw["n"], N, (0.0, 0.0, 0.0), hi, bc=tuple(kw.get("bc", (0, 0))) + (0,),
                         gamma=kw["gamma"], nu=kw.get("nu", 0.0), kappa=kw.get("kappa", 0.0), av_on=kw["av_on"],
                         positivity_on=kw.get("positivity_on", 0), cfl=kw["cfl"])
    w0 = inputs.random_modal_state(wl, seed=11) if recipe == "random" else inputs.project(wl, inputs.sod_tube_ic(wl))
    return P, w0, steps


def _rank(rank, ws, port, out_dir, name):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      OMP_NUM_THREADS="1")
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from oracle import slabs
    P, w0, steps = _setup(name)
    r = slabs.SlabRank(P, w0, rank, ws)
    dts = []
    for _ in range(steps):
        dt, st = r.step()
        assert st == 0
        dts.append(dt)
    np.save(os.path.join(out_dir, f"{name}_{ws}_{rank}.npy"), r.w)
    with open(os.path.join(out_dir, f"{name}_{ws}_{rank}.json"), "w") as f:
        json.dump({"dts": dts, "x0": r.x0, "x1": r.x1, "S": r.S_prev.tolist(), "wig": r.wig.tolist()}, f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name,ws", [("ns_av_3d_periodic", 2), ("sod_2d_outflow_limiter", 2),
                                     ("sod_2d_outflow_limiter", 3)])
def test_slab_decomposed_steps_equal_the_whole_domain_bitwise(tmp_path, name, ws):
    mp = pytest.importorskip("torch.multiprocessing")
    mp.start_processes(_rank, args=(ws, _free_port(), str(tmp_path), name), nprocs=ws, join=True,
                       start_method="spawn")
    sys.path.insert(0, ROOT)
    import oracle
    from oracle import slabs
    P, w0, steps = _setup(name)
    ref = oracle.Sim(P, w0)
    dts = []
    for _ in range(steps):
        dt, st = ref.step()
        assert st == 0
        dts.append(dt)
    for rank in range(ws):
        meta = json.load(open(tmp_path / f"{name}_{ws}_{rank}.json"))
        w = np.load(tmp_path / f"{name}_{ws}_{rank}.npy")
        assert meta["dts"] == dts  # the all-reduced CFL step is the whole domain's, bit for bit
        expect = slabs.take_slab(P, ref.w, meta["x0"], meta["x1"])
        assert np.array_equal(w, expect), np.abs(w - expect).max()
        if P.av_on:
            sl = slabs.take_slab(P, ref.S_prev[None, :, None], meta["x0"], meta["x1"]).ravel()
            assert np.array_equal(np.array(meta["S"]), sl)


def test_slab_ranges_cover_the_axis():
    sys.path.insert(0, ROOT)
    from oracle import slabs
    for N0 in (1, 5, 16, 17):
        for nr in (1, 2, 3, 4):
            if nr > N0:
                continue
            r = [slabs.slab_range(N0, nr, k) for k in range(nr)]
            assert r[0][0] == 0 and r[-1][1] == N0
            assert all(r[k][1] == r[k + 1][0] for k in range(nr - 1))
            assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1
