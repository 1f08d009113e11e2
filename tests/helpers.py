"""Shared helpers of the test suite: oracle problems from workloads, error norms."""
import numpy as np

import oracle


def problem(wl, **kw) -> oracle.Problem:
    args = dict(dim=wl.dim, n=wl.n, N=tuple(wl.N[: wl.dim]), lo=tuple(wl.lo[: wl.dim]), hi=tuple(wl.hi[: wl.dim]),
                bc=tuple(wl.bc[: wl.dim]), gamma=wl.gamma, nu=wl.nu, kappa=wl.kappa, av_on=wl.av_on,
                positivity_on=wl.positivity_on, cfl=wl.cfl, forcing_on=wl.forcing_on, force_amp=wl.force_amp,
                force_ts=wl.force_ts, force_dt=wl.force_dt, force_seed=wl.force_seed, tracer_on=wl.tracer_on,
                eta=wl.eta, basis=wl.basis)
    args.update(kw)
    return oracle.Problem(**args)


def rel_linf(a, b):
    """max over fields of max|a-b| / max|b| (per field scale)."""
    errs = []
    for f in range(b.shape[0]):
        scale = np.abs(b[f]).max()
        if scale == 0:
            scale = 1.0
        errs.append(np.abs(a[f] - b[f]).max() / scale)
    return max(errs)


def rel_l1(a, b, field=0):
    return np.abs(a[field] - b[field]).sum() / np.abs(b[field]).sum()


def rhs_scale(prob, w, ref):
    """Per-field size of the flux terms whose divergence is the right-hand side (each volume and face
    term is of that size, and rounding errors scale with it, not with the possibly cancelled result):
    lambda = max c_s + max |v| over the Gauss points, then over h_min
      rho: max rho lambda;  momentum: max rho lambda^2 (covers rho v^2 and p);  energy: gamma max e lambda;
      tracer rho c: max rho c lambda;
      alpha: (1 + max|alpha|) lambda (source terms f_v |div v| and alpha P c_s / (f_tau h))."""
    cm, vm, _ = oracle.max_speeds(prob, w)
    lam = cm + vm
    h = min(prob.h)
    d = prob.dim
    rho = np.abs(w[0, :, 0]).max()
    sc = [rho * lam / h] + [rho * lam * lam / h] * d + [prob.gamma * np.abs(w[d + 1, :, 0]).max() * lam / h]
    nc = d + 2
    if getattr(prob, "tracer_on", 0):  # tracer rho c: flux c rho v, like the density
        sc.append(max(np.abs(w[d + 2, :, 0]).max(), 1e-300) * lam / h)
        nc += 1
    if ref.shape[0] > nc:
        sc.append((1.0 + np.abs(w[nc, :, 0]).max()) * lam / h)
    return np.maximum(np.array(sc), np.abs(ref).reshape(ref.shape[0], -1).max(1))


def rhs_err(out, ref, prob, w):
    """max over fields of max|out_f - ref_f| / rhs_scale_f"""
    sc = rhs_scale(prob, w, ref)
    return max(np.abs(out[f] - ref[f]).max() / sc[f] for f in range(ref.shape[0]))


def state_scale(prob, ref):
    """Per-field physical scale of a state: rho_max; momentum rho_max (max c_s + max|v|) (a field that is
    zero by symmetry has no scale of its own); e_max; alpha: 1, the cap alpha_max of Sec. 4.1."""
    cm, vm, _ = oracle.max_speeds(prob, ref)
    d = prob.dim
    rho = np.abs(ref[0]).max()
    sc = [rho] + [rho * (cm + vm)] * d + [np.abs(ref[d + 1]).max()]
    nc = d + 2
    if getattr(prob, "tracer_on", 0):
        sc.append(rho)  # rho c with c of order one
        nc += 1
    if ref.shape[0] > nc:
        sc.append(1.0)
    return np.array(sc)


def state_err(out, ref, prob):
    """max over fields of max|out_f - ref_f| / state_scale_f"""
    sc = state_scale(prob, ref)
    return max(np.abs(out[f] - ref[f]).max() / sc[f] for f in range(ref.shape[0]))
