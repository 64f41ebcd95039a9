"""Strong-stability-preserving Runge-Kutta steps in Shu-Osher form for the oracle (TEST INFRASTRUCTURE
ONLY: used by tests/ and bench.py's CPU baselines; the CUDA library never imports it).

A Shu-Osher method with coefficients alpha[i][j], beta[i][j] (j < i, each row of alpha summing to one)
advances u_0 = u^n through stages
    u_i = sum_j alpha[i][j] * ( u_j + (beta[i][j] / alpha[i][j]) * dt * L(u_j) ),   i = 1..s,
u^{n+1} = u_s.  For the limited scheme "u + tau L(u)" is the limited forward-Euler stage FE_tau(u) of the
sweep (Sec. 6.2 builds its time stepping from such convex combinations of forward-Euler stages), so each
stage is a convex combination of previous stages and forward-Euler steps of them.  Terms with
beta[i][j] = 0 are the stage u_j itself.

SSPRK(5,4): the paper's experiments use the five-stage fourth-order SSP method (Sec. 6.2) but print no
coefficients; these are the published coefficients of the optimal method of Spiteri and Ruuth (SIAM J.
Numer. Anal. 40, 2002), SSP coefficient C = 1.508.  The tests pin them independently: the eight order
conditions of order four hold to rounding, every row of alpha sums to one, and C = min alpha/beta.  Its
stages u_3 enter u_4 and u_5 with the same step beta/alpha = 1/C (to the rounding of the printed
digits), so one forward-Euler evaluation of u_3 serves both.
"""
from __future__ import annotations

import numpy as np

SSPRK3_ALPHA = [[1.0], [0.75, 0.25], [1.0 / 3.0, 0.0, 2.0 / 3.0]]
SSPRK3_BETA = [[1.0], [0.0, 0.25], [0.0, 0.0, 2.0 / 3.0]]

SSPRK54_ALPHA = [[1.0],
                 [0.444370493651235, 0.555629506348765],
                 [0.620101851488403, 0.0, 0.379898148511597],
                 [0.178079954393132, 0.0, 0.0, 0.821920045606868],
                 [0.0, 0.0, 0.517231671970585, 0.096059710526147, 0.386708617503269]]
SSPRK54_BETA = [[0.391752226571890],
                [0.0, 0.368410593050371],
                [0.0, 0.0, 0.251891774271694],
                [0.0, 0.0, 0.0, 0.544974750228521],
                [0.0, 0.0, 0.0, 0.063692468666290, 0.226007483236906]]


def butcher(alpha, beta):
    """Butcher tableau (A [s][s], b [s], c [s]) of a Shu-Osher method: every stage written as
    u_i = u^n + dt sum_k A[i][k] L(u_k) by substituting the earlier stages."""
    s = len(alpha)
    R = np.zeros((s + 1, s + 1))
    for i in range(1, s + 1):
        for j in range(i):
            R[i] += alpha[i - 1][j] * R[j]
            R[i][j] += beta[i - 1][j]
    A, b = R[:s, :s], R[s, :s]
    return A, b, A.sum(1)


def ssp_coefficient(alpha, beta):
    """C = min over beta > 0 of alpha / beta: the method is SSP under dt <= C * dt_FE."""
    return min(alpha[i][j] / beta[i][j] for i in range(len(alpha)) for j in range(len(alpha[i]))
               if beta[i][j] != 0.0)


def shu_osher_step(U, dt, fe, alpha, beta, t=0.0):
    """One step from U: fe(u, tau, time) is the forward-Euler stage u + tau L(u) with boundary data at
    `time`; stage u_j lives at time t + c_j dt.  A stage's forward-Euler evaluations with the same step
    (to 1e-12 relative) are one evaluation.  Returns (U^{n+1}, list of fe results' extra outputs)."""
    _, _, c = butcher(alpha, beta)
    stages = [U]
    extras = []
    cache = {}  # (j, tau) -> FE_tau(u_j)
    for i in range(len(alpha)):
        acc = None
        for j, a in enumerate(alpha[i]):
            if a == 0.0:
                continue
            if beta[i][j] == 0.0:
                term = stages[j]
            else:
                tau = (beta[i][j] / a) * dt
                hit = next((v for (jj, tt), v in cache.items() if jj == j and abs(tt - tau) <= 1e-12 * tau), None)
                if hit is None:
                    hit, extra = fe(stages[j], tau, t + c[j] * dt)
                    cache[(j, tau)] = hit
                    extras.append(extra)
                term = hit
            acc = a * term if acc is None else acc + a * term
        stages.append(acc)
    return stages[-1], extras
