"""Slab decomposition of the FP64 oracle across processes: the CPU reference of the multi-GPU
data exchange of Sec. 8.1 (the domain is cut into slabs along x, one per rank) and Sec. 8.2 (the
surface states of the cells on a slab boundary are exchanged before the surface fluxes are
computed).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: only tests may import it.  It adds no
arithmetic of its own: every right-hand side, sensor, limiter and maximum is the oracle's C code;
this module only moves data between ranks (torch.distributed point-to-point messages and
all-reduce, gloo on CPU) and repeats the oracle's Runge-Kutta combination in the same operation
order, so that a decomposed step is bitwise equal to the undecomposed one.

Why it is exact (the "partial results" property of Sec. 3.2): the surface flux and the recovered
gradient of a face depend only on the two cells that share it, the volume terms, sensor, wiggle
source and limiter only on the cell itself, and the oracle lifts the face fluxes into a cell in a
fixed order.  So a rank computes the right-hand side of its slab on the slab extended by one layer
of neighbour cells on each side (received from the neighbouring ranks each stage) and keeps the
slab's part; the time step takes the maxima of the sound and flow speeds over all ranks
(all-reduce max), as Eq. timestep takes them over the whole domain.  What is exchanged here is the
neighbour layer's modes; the paper exchanges the traces and recovery partial sums computed from
them, which carry the same information for the face.

Limits: no driving source (its wave vectors depend on the box, not the slab); grids whose cell
coordinates are exact in binary (e.g. power-of-two cell counts on unit boxes), so that the
extended sub-grid has bitwise the same cell size.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import Problem, _p, lib, max_speeds, rhs, rk_stages, rk_table


def slab_range(N0: int, nranks: int, rank: int):
    """cells [x0, x1) along x of `rank`: contiguous slabs, the first N0 % nranks one cell longer"""
    base, extra = divmod(N0, nranks)
    x0 = rank * base + min(rank, extra)
    return x0, x0 + base + (1 if rank < extra else 0)


def _grid(prob: Problem):
    N = list(prob.N) + [1] * (3 - len(prob.N))
    return N[0], N[1], N[2]


def take_slab(prob: Problem, w: np.ndarray, x0: int, x1: int) -> np.ndarray:
    """the slab x0 <= x < x1 of a whole-domain state [F][cells][M] (cells x fastest)"""
    N0, N1, N2 = _grid(prob)
    F, _, M = w.shape
    return np.ascontiguousarray(w.reshape(F, N2, N1, N0, M)[:, :, :, x0:x1, :].reshape(F, -1, M))


def sub_problem(prob: Problem, xa: int, xb: int) -> Problem:
    """the problem restricted to cells xa <= x < xb, outflow along x (a sub-grid's x faces are either
    inner faces of the slab or faces the caller discards)"""
    N0, N1, N2 = _grid(prob)
    h = (prob.hi[0] - prob.lo[0]) / N0
    lo = list(prob.lo)
    hi = list(prob.hi)
    lo[0] = prob.lo[0] + xa * h
    hi[0] = prob.lo[0] + xb * h
    bc = list(prob.bc)
    bc[0] = 1
    N = list(prob.N)
    N[0] = xb - xa
    kw = dict(prob.__dict__)
    kw.update(N=tuple(N), lo=tuple(lo), hi=tuple(hi), bc=tuple(bc))
    return Problem(**kw)


class SlabRank:
    """one rank's slab of a decomposed oracle run (collectives over the default process group)"""

    def __init__(self, prob: Problem, w_full: np.ndarray, rank: int, nranks: int):
        import torch.distributed as dist

        assert not prob.forcing_on, "the driving source is not decomposed"
        self.dist = dist
        self.prob, self.rank, self.nranks = prob, rank, nranks
        self.N0, self.N1, self.N2 = _grid(prob)
        self.x0, self.x1 = slab_range(self.N0, nranks, rank)
        self.w = take_slab(prob, w_full, self.x0, self.x1)
        self.own = sub_problem(prob, self.x0, self.x1)
        periodic = prob.bc[0] == 0
        # neighbours across the slab's x faces (None at an outflow boundary of the domain)
        self.left = (rank - 1) % nranks if (self.x0 > 0 or periodic) else None
        self.right = (rank + 1) % nranks if (self.x1 < self.N0 or periodic) else None
        self.gl = 1 if self.left is not None else 0
        self.gr = 1 if self.right is not None else 0
        self.ext = sub_problem(prob, self.x0 - self.gl, self.x1 + self.gr)
        ncell = self.own.ncell
        self.S_prev = np.zeros(ncell)
        self.wig = np.zeros(ncell)
        self.scal = np.zeros(3)

    # -- data movement
    def _layer(self, u: np.ndarray, side: int) -> np.ndarray:
        F, _, M = u.shape
        v = u.reshape(F, self.N2, self.N1, self.x1 - self.x0, M)
        return np.ascontiguousarray(v[:, :, :, 0 if side == 0 else -1, :])

    def exchange(self, u: np.ndarray) -> np.ndarray:
        """the slab extended by the neighbours' boundary layers: [F][cells of the extended sub-grid][M]"""
        import torch

        dist = self.dist
        F, _, M = u.shape
        shape = (F, self.N2, self.N1, M)
        reqs = []
        got = {}
        # send the left layer to the left neighbour and the right layer to the right neighbour;
        # receive their facing layers (tags tell the two directions apart when both are one rank)
        if self.left is not None:
            reqs.append(dist.isend(torch.from_numpy(self._layer(u, 0)), self.left, tag=0))
            got["l"] = torch.empty(shape, dtype=torch.float64)
            reqs.append(dist.irecv(got["l"], self.left, tag=1))
        if self.right is not None:
            reqs.append(dist.isend(torch.from_numpy(self._layer(u, 1)), self.right, tag=1))
            got["r"] = torch.empty(shape, dtype=torch.float64)
            reqs.append(dist.irecv(got["r"], self.right, tag=0))
        for r in reqs:
            r.wait()
        v = u.reshape(F, self.N2, self.N1, self.x1 - self.x0, M)
        parts = []
        if "l" in got:
            parts.append(got["l"].numpy()[:, :, :, None, :])
        parts.append(v)
        if "r" in got:
            parts.append(got["r"].numpy()[:, :, :, None, :])
        return np.ascontiguousarray(np.concatenate(parts, axis=3).reshape(F, -1, M))

    def interior(self, u_ext: np.ndarray) -> np.ndarray:
        F, _, M = u_ext.shape
        nx = self.x1 - self.x0 + self.gl + self.gr
        v = u_ext.reshape(F, self.N2, self.N1, nx, M)
        return np.ascontiguousarray(v[:, :, :, self.gl:self.gl + self.x1 - self.x0, :].reshape(F, -1, M))

    def allreduce(self, vals, op):
        import torch

        t = torch.tensor(vals, dtype=torch.float64)
        self.dist.all_reduce(t, op=op)
        return t.tolist()

    # -- the operator and one step, in the oracle's order of operations
    def rhs(self, u: np.ndarray):
        u_ext = self.exchange(u)
        wig_ext = None
        if self.prob.av_on:
            wv = self.wig.reshape(self.N2, self.N1, self.x1 - self.x0)
            wig_ext = np.ascontiguousarray(np.pad(wv, ((0, 0), (0, 0), (self.gl, self.gr))).reshape(-1))
        L_ext, st = rhs(self.ext, u_ext, wig_ext)
        return self.interior(L_ext), st

    def step(self, dt: float = 0.0):
        """one SSP Runge-Kutta step of the slab; returns (dt, status or-ed over the ranks)"""
        import torch.distributed as dist

        P = self.prob
        status = 0
        if P.positivity_on:
            status |= lib().or_positivity(ctypes.byref(self.own.cfg()), _p(self.w))
        if P.av_on:
            status |= lib().or_wiggle(ctypes.byref(self.own.cfg()), _p(self.w), _p(self.S_prev), _p(self.wig),
                                      float(self.scal[0]), int(self.scal[1]))
        if not dt > 0.0:
            cm, vm, st = max_speeds(self.own, self.w)
            status |= st
            cm, vm = self.allreduce([cm, vm], dist.ReduceOp.MAX)
            hmin = min((P.hi[a] - P.lo[a]) / list(P.N)[a] for a in range(P.dim))
            dt = P.cfl * hmin / (2.0 * (P.n + 1) * (cm + vm))
        s = P.rk_stages if P.rk_stages > 0 else rk_stages(P.n)
        al, be = rk_table(s)
        U = [self.w.copy()]
        L = []
        for i in range(1, s + 1):
            Li, st = self.rhs(U[i - 1])
            status |= st
            L.append(Li)
            acc = np.zeros_like(self.w)
            for k in range(i):
                if al[i, k] != 0.0:
                    acc = acc + al[i, k] * U[k]
                if be[i, k] != 0.0:
                    acc = acc + (be[i, k] * dt) * L[k]
            if P.positivity_on:
                status |= lib().or_positivity(ctypes.byref(self.own.cfg()), _p(acc))
            U.append(acc)
        self.w = U[s]
        self.scal[0] = dt
        self.scal[1] += 1.0
        self.scal[2] += dt
        (st_all,) = self.allreduce([float(status)], dist.ReduceOp.MAX)
        return dt, int(st_all)
