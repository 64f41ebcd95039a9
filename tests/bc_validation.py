"""The modified isentropic vortex of Sec. 6.4 (subsec. BCvalidation): the vortex of Sec. 6.2, test case
(i) (gamma = 5/3, beta = 5, [-5,5]^2, centre starting at (-1, -1)) advected at v_inf = (M, M) up to
t_F = 6 / M, when its centre sits on the top right corner (5, 5), with Q1 elements, the convex-limited
scheme and SSPRK(5,4).  Four ways to give the boundary its data:
  (a) Dirichlet entries with the exact solution at every stage time;
  (b) in/outflow entries (Sec. 4.1) with the exact solution as their data;
  (c) in/outflow entries with the far-field state (rho, v, p) = (1, v_inf, 1) as their data;
  (d) in/outflow entries with the state at the start of the step as their data.
The paper reports the L1 errors and rates in Table ErrorBoundaryConditions.

Reading: the paper calls M the speed of the vortex centre relative to the speed of sound in each
direction, and sets t_F = 6 / M so that the centre ends on the corner; the centre moves by 6 in x and y
only with v_inf = (M, M), which is what is taken (the far-field sound speed is sqrt(5/3), so M = 1 is
1 / sqrt(5/3) = 0.77 of the sound speed per direction).
Test infrastructure: shared by the oracle pin and the GPU test."""
from __future__ import annotations

import numpy as np

from paper_2402_04514_gb300 import assembly, workloads
from tests.helpers import consolidated_l1

GAMMA = 5.0 / 3.0
CFL = 0.5
STRATEGY_BC = {"a": "dirichlet", "b": "inoutflow", "c": "inoutflow", "d": "inoutflow"}

# Table ErrorBoundaryConditions (L1 errors at 2304 and 9216 DoFs and the rate between them)
PAPER = {
    "a": {1.0: (4.37e-03, 8.63e-04, 2.34), 1.5: (3.05e-03, 6.26e-04, 2.28), 2.0: (3.05e-03, 6.13e-04, 2.31),
          2.5: (2.79e-03, 5.68e-04, 2.29)},
    "b": {1.0: (4.05e-03, 8.36e-04, 2.27), 1.5: (2.98e-03, 6.19e-04, 2.27), 2.0: (2.41e-03, 5.15e-04, 2.22),
          2.5: (1.99e-03, 4.29e-04, 2.21)},
    "c": {1.0: (1.36e-02, 1.07e-02, 0.35), 1.5: (4.09e-03, 1.70e-03, 1.26), 2.0: (2.41e-03, 5.15e-04, 2.22),
          2.5: (1.99e-03, 4.29e-04, 2.21)},
    "d": {1.0: (6.12e-03, 3.99e-03, 0.61), 1.5: (3.02e-03, 6.58e-04, 2.20), 2.0: (2.41e-03, 5.08e-04, 2.24),
          2.5: (2.03e-03, 4.33e-04, 2.22)},
}


def problem(ne, strategy):
    sides = {s: STRATEGY_BC[strategy] for s in ("left", "right", "bottom", "top")}
    return assembly.assemble_2d(ne, ne, 1, box=(-5.0, 5.0, -5.0, 5.0), bc=sides)


def exact(x, y, t, M):
    return workloads.vortex(x, y, t, gamma=GAMMA, vinf=(M, M))


def far_field(P, M):
    nb = P.nb
    return workloads.prim_to_cons(np.ones(nb), np.stack([np.full(nb, M), np.full(nb, M)]), np.ones(nb), GAMMA)


def boundary_data(P, strategy, M, U_step_start):
    """bdata_fn(t) for the stages of one step: [m][nb] in the caller's boundary order."""
    if strategy in ("a", "b"):
        return lambda t: np.ascontiguousarray(exact(P.b_x[0], P.b_x[1], t, M))
    if strategy == "c":
        ff = np.ascontiguousarray(far_field(P, M))
        return lambda t: ff
    old = np.ascontiguousarray(U_step_start[:, P.b_node])
    return lambda t: old


def run_oracle(ne, strategy, M, openmp=True):
    """L1 error (Sec. 6.2's consolidated norm) at t_F = 6 / M of the oracle's limited Q1 scheme with
    SSPRK(5,4), dt = CFL * C * (the forward-Euler bound of Sec. 3.3) clipped to t_F."""
    from oracle import ssprk
    from oracle.oracle import Oracle

    P = problem(ne, strategy)
    O = Oracle(P, gamma=GAMMA, openmp=openmp)
    C = ssprk.ssp_coefficient(ssprk.SSPRK54_ALPHA, ssprk.SSPRK54_BETA)
    U = np.ascontiguousarray(exact(P.x[0], P.x[1], 0.0, M))
    t, tF = 0.0, 6.0 / M
    while t < tF - 1e-12:
        bd = boundary_data(P, strategy, M, U)
        dt = min(CFL * C * O.max_dt(U, 1.0, bdata=bd(t)), tF - t)
        U, flags = O.ssprk54_step(U, dt, bd, t)
        assert flags == 0
        t += dt
    return consolidated_l1(P, U, exact(P.x[0], P.x[1], tF, M))


def run_gpu(ne, strategy, M, torch):
    """The same run on the GPU (tests/gpu_rk.py: every forward-Euler stage in the library with its data at
    the stage's time).  Returns the L1 error at t_F."""
    from paper_2402_04514_gb300.gdg import Solver
    from tests.gpu_rk import ssprk54_solve

    P = problem(ne, strategy)
    tF = 6.0 / M
    ff = far_field(P, M)

    def bdata(t, U_start):
        if strategy in ("a", "b"):
            return exact(P.b_x[0], P.b_x[1], t, M)
        if strategy == "c":
            return ff
        return U_start[:, torch.from_numpy(P.b_node.astype(np.int64)).cuda()].contiguous()

    U = ssprk54_solve(Solver(P, gamma=GAMMA), exact(P.x[0], P.x[1], 0.0, M), bdata, tF, torch, CFL)
    return consolidated_l1(P, U, exact(P.x[0], P.x[1], tF, M))


if __name__ == "__main__":
    # The table of L1 errors and rates of every strategy and speed on 24^2 .. 192^2 elements (GPU):
    #   python -m tests.bc_validation
    import math
    import sys

    import torch

    levels = (24, 48, 96, 192)
    for strategy in "abcd":
        for M in (1.0, 1.5, 2.0, 2.5):
            errs = [run_gpu(ne, strategy, M, torch) for ne in levels]
            rates = [math.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]
            print(strategy, M, " ".join(f"{e:.3e}" for e in errs), "rates", " ".join(f"{r:.2f}" for r in rates),
                  "paper", PAPER[strategy][M], flush=True)
    sys.exit(0)
