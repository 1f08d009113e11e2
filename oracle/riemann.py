"""Exact Riemann solver of the 1-D Euler equations for an ideal gas.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Textbook construction (Toro, "Riemann Solvers and Numerical Methods for Fluid
Dynamics", ch. 4): the star-region pressure is the root of
f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the shock (Rankine-Hugoniot)
branch for p > p_K and the isentropic rarefaction branch otherwise; the
solution is self-similar in x/t and sampled wave by wave.  It pins the
oracle's shock-tube evolution (the 1-D shock tube embedded in 2-D).
"""
from __future__ import annotations

import math

import numpy as np


def _fK(p, rho, pK, cK, g):
    if p > pK:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        f = (p - pK) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - 0.5 * (p - pK) / (B + p))
    else:
        f = 2.0 * cK / (g - 1.0) * ((p / pK) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * cK) * (p / pK) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, gamma):
    """(p*, u*) of the Riemann problem with primitive states (rho, u, p)."""
    rL, uL, pL = left
    rR, uR, pR = right
    g = gamma
    cL = math.sqrt(g * pL / rL)
    cR = math.sqrt(g * pR / rR)
    if 2.0 * (cL + cR) / (g - 1.0) <= uR - uL:
        raise ValueError("vacuum is generated")
    # two-rarefaction guess
    z = (g - 1.0) / (2.0 * g)
    p = ((cL + cR - 0.5 * (g - 1.0) * (uR - uL)) / (cL / pL ** z + cR / pR ** z)) ** (1.0 / z)
    p = max(p, 1e-12)
    for _ in range(200):
        fL, dL = _fK(p, rL, pL, cL, g)
        fR, dR = _fK(p, rR, pR, cR, g)
        dp = (fL + fR + uR - uL) / (dL + dR)
        pn = max(p - dp, 1e-14)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _fK(p, rL, pL, cL, g)
    fR, _ = _fK(p, rR, pR, cR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    return p, u


def sample(left, right, gamma, s):
    """primitive (rho, u, p) at similarity coordinates s = (x - x0)/t (array)."""
    rL, uL, pL = left
    rR, uR, pR = right
    g = gamma
    ps, us = star_state(left, right, gamma)
    cL = math.sqrt(g * pL / rL)
    cR = math.sqrt(g * pR / rR)
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    rho = np.empty_like(s)
    u = np.empty_like(s)
    p = np.empty_like(s)
    gm = (g - 1.0) / (g + 1.0)
    for i, S in enumerate(s):
        if S <= us:  # left of the contact
            if ps > pL:  # left shock
                SL = uL - cL * math.sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g))
                if S <= SL:
                    rho[i], u[i], p[i] = rL, uL, pL
                else:
                    rho[i] = rL * (ps / pL + gm) / (gm * ps / pL + 1.0)
                    u[i], p[i] = us, ps
            else:  # left rarefaction
                SHL = uL - cL
                cs = cL * (ps / pL) ** ((g - 1.0) / (2.0 * g))
                STL = us - cs
                if S <= SHL:
                    rho[i], u[i], p[i] = rL, uL, pL
                elif S >= STL:
                    rho[i] = rL * (ps / pL) ** (1.0 / g)
                    u[i], p[i] = us, ps
                else:
                    c = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * (uL - S))
                    rho[i] = rL * (c / cL) ** (2.0 / (g - 1.0))
                    u[i] = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL + S)
                    p[i] = pL * (c / cL) ** (2.0 * g / (g - 1.0))
        else:  # right of the contact
            if ps > pR:  # right shock
                SR = uR + cR * math.sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g))
                if S >= SR:
                    rho[i], u[i], p[i] = rR, uR, pR
                else:
                    rho[i] = rR * (ps / pR + gm) / (gm * ps / pR + 1.0)
                    u[i], p[i] = us, ps
            else:  # right rarefaction
                SHR = uR + cR
                cs = cR * (ps / pR) ** ((g - 1.0) / (2.0 * g))
                STR = us + cs
                if S >= SHR:
                    rho[i], u[i], p[i] = rR, uR, pR
                elif S <= STR:
                    rho[i] = rR * (ps / pR) ** (1.0 / g)
                    u[i], p[i] = us, ps
                else:
                    c = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * (uR - S))
                    rho[i] = rR * (c / cR) ** (2.0 / (g - 1.0))
                    u[i] = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * uR + S)
                    p[i] = pR * (c / cR) ** (2.0 * g / (g - 1.0))
    return rho, u, p
