"""Exact solution of the 1D Riemann problem for a polytropic gas (textbook Riemann theory: the star
pressure is the root of f_L(p) + f_R(p) + u_R - u_L = 0 with the shock/rarefaction branches of the
pressure functions; Toro, Riemann Solvers and Numerical Methods, ch. 4).  Written independently of the
oracle; used to pin the wave-speed bound and the shock-tube solution."""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def _fK(p, rho, pK, a, g):
    if p > pK:  # shock branch
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        return (p - pK) * math.sqrt(A / (p + B))
    return 2.0 * a / (g - 1.0) * ((p / pK) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star_state(rhoL, uL, pL, rhoR, uR, pR, g):
    """Returns (p*, u*); raises ValueError on vacuum generation."""
    aL = math.sqrt(g * pL / rhoL)
    aR = math.sqrt(g * pR / rhoR)
    if 2.0 * (aL + aR) / (g - 1.0) <= uR - uL:
        raise ValueError("vacuum")

    def F(p):
        return _fK(p, rhoL, pL, aL, g) + _fK(p, rhoR, pR, aR, g) + uR - uL

    lo = 1e-14 * min(pL, pR)
    hi = max(pL, pR)
    while F(hi) < 0.0:
        hi *= 4.0
    ps = brentq(F, lo, hi, xtol=1e-300, rtol=1e-15, maxiter=500)
    us = 0.5 * (uL + uR) + 0.5 * (_fK(ps, rhoR, pR, aR, g) - _fK(ps, rhoL, pL, aL, g))
    return ps, us


def max_wave_speed(rhoL, uL, pL, rhoR, uR, pR, g):
    """max( (leftmost wave speed)^-, (rightmost wave speed)^+ ) of the exact solution."""
    aL = math.sqrt(g * pL / rhoL)
    aR = math.sqrt(g * pR / rhoR)
    ps, _ = star_state(rhoL, uL, pL, rhoR, uR, pR, g)
    if ps > pL:
        sL = uL - aL * math.sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g))
    else:
        sL = uL - aL
    if ps > pR:
        sR = uR + aR * math.sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g))
    else:
        sR = uR + aR
    return max(max(-sL, 0.0), max(sR, 0.0)), ps


def sample(xi, rhoL, uL, pL, rhoR, uR, pR, g):
    """(rho, u, p) of the self-similar solution at xi = x / t (array)."""
    xi = np.asarray(xi, float)
    aL = math.sqrt(g * pL / rhoL)
    aR = math.sqrt(g * pR / rhoR)
    ps, us = star_state(rhoL, uL, pL, rhoR, uR, pR, g)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    gm = (g - 1.0) / (g + 1.0)
    for q, s in enumerate(xi):
        if s <= us:  # left of the contact
            if ps > pL:
                SL = uL - aL * math.sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g))
                if s <= SL:
                    rho[q], u[q], p[q] = rhoL, uL, pL
                else:
                    rho[q] = rhoL * (ps / pL + gm) / (gm * ps / pL + 1.0)
                    u[q], p[q] = us, ps
            else:
                asL = aL * (ps / pL) ** ((g - 1.0) / (2.0 * g))
                if s <= uL - aL:
                    rho[q], u[q], p[q] = rhoL, uL, pL
                elif s >= us - asL:
                    rho[q] = rhoL * (ps / pL) ** (1.0 / g)
                    u[q], p[q] = us, ps
                else:
                    c = 2.0 / (g + 1.0) + gm / aL * (uL - s)
                    rho[q] = rhoL * c ** (2.0 / (g - 1.0))
                    u[q] = 2.0 / (g + 1.0) * (aL + (g - 1.0) / 2.0 * uL + s)
                    p[q] = pL * c ** (2.0 * g / (g - 1.0))
        else:
            if ps > pR:
                SR = uR + aR * math.sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g))
                if s >= SR:
                    rho[q], u[q], p[q] = rhoR, uR, pR
                else:
                    rho[q] = rhoR * (ps / pR + gm) / (gm * ps / pR + 1.0)
                    u[q], p[q] = us, ps
            else:
                asR = aR * (ps / pR) ** ((g - 1.0) / (2.0 * g))
                if s >= uR + aR:
                    rho[q], u[q], p[q] = rhoR, uR, pR
                elif s <= us + asR:
                    rho[q] = rhoR * (ps / pR) ** (1.0 / g)
                    u[q], p[q] = us, ps
                else:
                    c = 2.0 / (g + 1.0) - gm / aR * (uR - s)
                    rho[q] = rhoR * c ** (2.0 / (g - 1.0))
                    u[q] = 2.0 / (g + 1.0) * (-aR + (g - 1.0) / 2.0 * uR + s)
                    p[q] = pR * c ** (2.0 * g / (g - 1.0))
    return rho, u, p
