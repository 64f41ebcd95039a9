"""SSPRK(5,4) through gdg_stage with boundary data at every stage time (test infrastructure).

The fused gdg_ssprk54_step takes one boundary-data array per step; the experiments of Sec. 6.2 and 6.4 give
time-dependent Dirichlet or in/outflow data, so their GPU runs step with gdg_stage: each forward-Euler
stage runs in the library with its data at the stage's time, and the Shu-Osher combinations are formed
from the stages' outputs (gdg_stage's U_out = alpha U_base + (1 - alpha) FE(U_in) covers every stage but
the last, whose base combines u2 and FE(u3) = (u4 - alpha40 u0) / alpha43).  dt = cfl * C * the
forward-Euler bound of Sec. 3.3 (C the SSP coefficient), the last step clipped to t_end."""
from __future__ import annotations

import numpy as np


def ssprk54_solve(S, U0, bdata_fn, t_end, torch, cfl=0.5):
    """S: a Solver; U0: numpy [m][n]; bdata_fn(t, U_step_start) -> numpy or device [m][nb] (or None without
    data entries).  Returns the state at t_end as numpy."""
    from oracle import ssprk

    A, B = ssprk.SSPRK54_ALPHA, ssprk.SSPRK54_BETA
    _, _, c = ssprk.butcher(A, B)
    C = ssprk.ssp_coefficient(A, B)

    def dev(a):
        if a is None or hasattr(a, "is_cuda"):
            return a
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    U = dev(U0)
    t = 0.0
    while t < t_end - 1e-12:
        bd = lambda time: dev(bdata_fn(time, U))
        dt = min(cfl * C * S.max_dt(U, 1.0, bdata=bd(t)), t_end - t)
        tau = lambda i: B[i][i] / A[i][i] * dt
        u1 = S.stage(U, tau(0), bdata=bd(t + c[0] * dt))
        u2 = S.stage(u1, tau(1), U_base=U, alpha=A[1][0], bdata=bd(t + c[1] * dt))
        u3 = S.stage(u2, tau(2), U_base=U, alpha=A[2][0], bdata=bd(t + c[2] * dt))
        u4 = S.stage(u3, tau(3), U_base=U, alpha=A[3][0], bdata=bd(t + c[3] * dt))
        base = (A[4][2] * u2 + (A[4][3] / A[3][3]) * (u4 - A[3][0] * U)) / (1.0 - A[4][4])
        U = S.stage(u4, tau(4), U_base=base, alpha=1.0 - A[4][4], bdata=bd(t + c[4] * dt))
        t += dt
    assert S.status() == 0
    return U.cpu().numpy()
