"""Exact Riemann solver for the 1D Euler equations (ideal gas).

TEST INFRASTRUCTURE ONLY: it verifies the oracle's Sod-tube runs and is not
part of the finite-volume method of arXiv 2302.09005.

Method: E. F. Toro, "Riemann Solvers and Numerical Methods for Fluid
Dynamics", 3rd ed., ch. 4.  The star pressure p* is the root of
    f(p) = f_L(p) + f_R(p) + (u_R - u_L),
where f_K is the shock (Rankine-Hugoniot) branch for p > p_K and the
rarefaction (isentrope + Riemann invariant) branch for p <= p_K; Newton's
method on f gives p*, and the similarity solution is sampled at x/t.
"""
from __future__ import annotations

import math

import numpy as np


def _f_branch(p, rho_k, p_k, c_k, g):
    """f_K(p) and its derivative (Toro ch. 4, pressure functions)."""
    if p > p_k:  # shock
        A = 2.0 / ((g + 1.0) * rho_k)
        B = (g - 1.0) / (g + 1.0) * p_k
        sq = math.sqrt(A / (p + B))
        f = (p - p_k) * sq
        df = sq * (1.0 - 0.5 * (p - p_k) / (B + p))
    else:  # rarefaction
        pr = p / p_k
        f = 2.0 * c_k / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho_k * c_k) * pr ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(rhoL, uL, pL, rhoR, uR, pR, gamma=1.4, tol=1e-14, max_iter=100):
    """Return (p*, u*, rho*_L, rho*_R) of the exact Riemann solution."""
    g = gamma
    cL = math.sqrt(g * pL / rhoL)
    cR = math.sqrt(g * pR / rhoR)
    du = uR - uL
    if 2.0 * (cL + cR) / (g - 1.0) <= du:
        raise ValueError("vacuum is generated; not handled")
    # two-rarefaction initial guess (Toro ch. 4, "TRRS" guess)
    z = (g - 1.0) / (2.0 * g)
    p = ((cL + cR - 0.5 * (g - 1.0) * du) / (cL / pL ** z + cR / pR ** z)) ** (1.0 / z)
    p = max(p, 1e-12)
    for _ in range(max_iter):
        fL, dfL = _f_branch(p, rhoL, pL, cL, g)
        fR, dfR = _f_branch(p, rhoR, pR, cR, g)
        p_new = p - (fL + fR + du) / (dfL + dfR)
        p_new = max(p_new, 1e-14)
        if abs(p_new - p) <= tol * 0.5 * (p_new + p):
            p = p_new
            break
        p = p_new
    fL, _ = _f_branch(p, rhoL, pL, cL, g)
    fR, _ = _f_branch(p, rhoR, pR, cR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    gm = (g - 1.0) / (g + 1.0)

    def rho_star(rho_k, p_k):
        if p > p_k:
            return rho_k * ((p / p_k + gm) / (gm * p / p_k + 1.0))
        return rho_k * (p / p_k) ** (1.0 / g)

    return p, u, rho_star(rhoL, pL), rho_star(rhoR, pR)


def sample(xi, rhoL, uL, pL, rhoR, uR, pR, gamma=1.4):
    """Primitive state (rho, u, p) of the exact solution at similarity
    coordinates xi = (x - x0) / t (numpy array)."""
    g = gamma
    ps, us, rsL, rsR = star_state(rhoL, uL, pL, rhoR, uR, pR, g)
    cL = math.sqrt(g * pL / rhoL)
    cR = math.sqrt(g * pR / rhoR)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for idx, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pL:  # left shock
                SL = uL - cL * math.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
                st = (rhoL, uL, pL) if s <= SL else (rsL, us, ps)
            else:  # left rarefaction
                cs = cL * (ps / pL) ** ((g - 1) / (2 * g))
                SH, ST = uL - cL, us - cs
                if s <= SH:
                    st = (rhoL, uL, pL)
                elif s >= ST:
                    st = (rsL, us, ps)
                else:
                    c = 2 / (g + 1) * (cL + (g - 1) / 2 * (uL - s))
                    uu = 2 / (g + 1) * (cL + (g - 1) / 2 * uL + s)
                    rr = rhoL * (c / cL) ** (2 / (g - 1))
                    st = (rr, uu, pL * (c / cL) ** (2 * g / (g - 1)))
        else:  # right of the contact
            if ps > pR:  # right shock
                SR = uR + cR * math.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
                st = (rhoR, uR, pR) if s >= SR else (rsR, us, ps)
            else:  # right rarefaction
                cs = cR * (ps / pR) ** ((g - 1) / (2 * g))
                SH, ST = uR + cR, us + cs
                if s >= SH:
                    st = (rhoR, uR, pR)
                elif s <= ST:
                    st = (rsR, us, ps)
                else:
                    c = 2 / (g + 1) * (cR - (g - 1) / 2 * (uR - s))
                    uu = 2 / (g + 1) * (-cR + (g - 1) / 2 * uR + s)
                    rr = rhoR * (c / cR) ** (2 / (g - 1))
                    st = (rr, uu, pR * (c / cR) ** (2 * g / (g - 1)))
        rho[idx], u[idx], p[idx] = st
    return rho, u, p
