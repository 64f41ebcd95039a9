"""Seeded synthetic initial data for the stage (input generators only: no stage arithmetic).

States are returned conserved, component-major: U[c][node] with c = (rho, m_1..m_d, E), float64.

* Sod shock tube (1D, gamma = 1.4): the textbook two-state problem, used as the 1D workload.
* Isentropic vortex (Sec. 6.2, test case (i)): the Yee-Sandham vortex.  The paper's printed formula
  puts e^{1-r^2} in the velocity and calls the temperature a density increment; radial equilibrium
  needs the velocity factor e^{(1-r^2)/2} and T = 1 + dT, rho = T^{1/(gamma-1)}, p = rho^gamma, which
  is what is implemented (the tests check dp/dr = rho v_theta^2 / r).
* Four-quadrant Riemann data and two-state Riemann data with states drawn from numpy's
  default_rng(seed): the 2D workloads.
"""
from __future__ import annotations

import math

import numpy as np


def prim_to_cons(rho, vel, p, gamma):
    """rho [n], vel [d][n], p [n] -> U [d+2][n]."""
    vel = np.atleast_2d(vel)
    d = vel.shape[0]
    U = np.empty((d + 2, rho.shape[0]))
    U[0] = rho
    U[1:d + 1] = rho * vel
    U[d + 1] = p / (gamma - 1.0) + 0.5 * rho * (vel ** 2).sum(0)
    return U


def cons_to_prim(U, gamma):
    d = U.shape[0] - 2
    rho = U[0]
    vel = U[1:d + 1] / rho
    p = (gamma - 1.0) * (U[d + 1] - 0.5 * rho * (vel ** 2).sum(0))
    return rho, vel, p


def sod(x, gamma=1.4, x_split=0.5, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1)):
    """1D shock tube: (rho, u, p) = left for x < x_split, right otherwise."""
    x = np.asarray(x).reshape(-1)
    L = x < x_split
    rho = np.where(L, left[0], right[0])
    u = np.where(L, left[1], right[1])
    p = np.where(L, left[2], right[2])
    return prim_to_cons(rho, u[None, :], p, gamma)


def vortex(x, y, t, gamma=1.4, beta=5.0, vinf=(1.0, 1.0), x0=(-1.0, -1.0)):
    """Isentropic vortex at time t (exact solution on the unbounded plane)."""
    xb = x - x0[0] - t * vinf[0]
    yb = y - x0[1] - t * vinf[1]
    r2 = xb * xb + yb * yb
    g = beta / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    u = vinf[0] - g * yb
    v = vinf[1] + g * xb
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return prim_to_cons(rho, np.stack([u, v]), p, gamma)


def four_quadrant_states(seed=0, rho_range=(0.1, 2.0), vel_range=(-1.0, 1.0), p_range=(0.1, 2.0)):
    """Four (rho, u, v, p) states drawn uniformly from default_rng(seed), quadrant order
    (x<xs,y<ys), (x>=xs,y<ys), (x<xs,y>=ys), (x>=xs,y>=ys)."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(*rho_range, 4)
    u = rng.uniform(*vel_range, 4)
    v = rng.uniform(*vel_range, 4)
    p = rng.uniform(*p_range, 4)
    return rho, u, v, p


def four_quadrant(x, y, gamma=1.4, seed=0, split=(0.5, 0.5)):
    rho_s, u_s, v_s, p_s = four_quadrant_states(seed)
    q = (x >= split[0]).astype(int) + 2 * (y >= split[1]).astype(int)
    return prim_to_cons(rho_s[q], np.stack([u_s[q], v_s[q]]), p_s[q], gamma)


def two_state_riemann(x, y, rng, gamma=1.4, center=(0.5, 0.5)):
    """Two states split by a line through `center` with a random normal angle; rho and p log-uniform
    in [0.1, 10], velocity uniform in the disk |u| <= 2 (drawn from the given Generator)."""
    ang = rng.uniform(0.0, 2.0 * math.pi)
    nrm = np.array([math.cos(ang), math.sin(ang)])
    rho = np.exp(rng.uniform(math.log(0.1), math.log(10.0), 2))
    p = np.exp(rng.uniform(math.log(0.1), math.log(10.0), 2))
    rad = 2.0 * np.sqrt(rng.uniform(0.0, 1.0, 2))
    th = rng.uniform(0.0, 2.0 * math.pi, 2)
    u = rad * np.cos(th)
    v = rad * np.sin(th)
    side = (((x - center[0]) * nrm[0] + (y - center[1]) * nrm[1]) >= 0).astype(int)
    return prim_to_cons(rho[side], np.stack([u[side], v[side]]), p[side], gamma)
