"""The boundary-condition validation of Sec. 6.4 (subsec. BCvalidation) on the GPU (tests/bc_validation.py):
one in/outflow case with exact data against the oracle stage by stage, and the convergence of strategies
(a) exact Dirichlet data and (b) in/outflow entries with exact data, on meshes the oracle cannot afford,
against the rates of Table ErrorBoundaryConditions at the paper's finest levels."""
import math

import numpy as np
import pytest

from tests import bc_validation as bv
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04514_gb300 import build

    build.build()
    return torch


@pytest.mark.parametrize("M", [1.0, 2.0])
def test_inoutflow_vortex_stages_match_the_oracle(torch_cuda, M):
    """Strategy (b) on 24^2 Q1 elements: every limited stage of three SSPRK(5,4) steps, from the GPU's own
    state and with the exact data at the stage's time, equals the oracle's stage within 1e-12 relative per
    component (subsonic outflow at M = 1, supersonic everywhere at M = 2)."""
    torch = torch_cuda
    from oracle import ssprk
    from oracle.oracle import Oracle
    from paper_2402_04514_gb300.gdg import Solver

    P = bv.problem(24, "b")
    S, O = Solver(P, gamma=bv.GAMMA), Oracle(P, gamma=bv.GAMMA)
    A, B = ssprk.SSPRK54_ALPHA, ssprk.SSPRK54_BETA
    _, _, c = ssprk.butcher(A, B)
    U = np.ascontiguousarray(bv.exact(P.x[0], P.x[1], 0.0, M))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    t = 0.0
    for _ in range(3):
        bd = lambda s: np.ascontiguousarray(bv.exact(P.b_x[0], P.b_x[1], s, M))
        dt = 0.5 * ssprk.ssp_coefficient(A, B) * O.max_dt(U, 1.0, bdata=bd(t))
        stages = [U]
        for k in range(5):  # the forward-Euler evaluation of each stage, GPU against the oracle
            j = k if k < 4 else 4
            tau = B[k][j] / A[k][j] * dt
            got = S.stage(dev(stages[j]), tau, bdata=dev(bd(t + c[j] * dt))).cpu().numpy()
            want, flags = O.stage(stages[j], tau, bdata=bd(t + c[j] * dt))
            assert flags == 0 and S.status() == 0
            assert rel_err(got, want) <= 1e-12
            if k < 4:
                stages.append(A[k][0] * U + (1.0 - A[k][0]) * want if k > 0 else want)
            else:
                fe3 = (stages[4] - A[3][0] * U) / A[3][3]
                U = A[4][2] * stages[2] + A[4][3] * fe3 + A[4][4] * want
        t += dt


@pytest.mark.parametrize("strategy", ["a", "b"])
def test_exact_data_converge_at_the_papers_rate(torch_cuda, strategy):
    """L1 rates of strategies (a) and (b) between 192^2 and 384^2 Q1 elements (147,456 and 589,824 DoFs) at
    the supersonic speeds M = 2 and 2.5 within 0.15 of the table's rates at 589,824 DoFs; the far-field
    strategy (c) at M = 1 stalls (its rate below 0.5; the table's 0.03)."""
    torch = torch_cuda
    want = {("a", 2.0): 2.07, ("a", 2.5): 2.07, ("b", 2.0): 2.03, ("b", 2.5): 2.02}
    for M in (2.0, 2.5):
        e1 = bv.run_gpu(192, strategy, M, torch)
        e2 = bv.run_gpu(384, strategy, M, torch)
        rate = math.log2(e1 / e2)
        assert abs(rate - want[(strategy, M)]) <= 0.15, (M, e1, e2, rate)
    if strategy == "b":
        e1 = bv.run_gpu(96, "c", 1.0, torch)
        e2 = bv.run_gpu(192, "c", 1.0, torch)
        assert math.log2(e1 / e2) < 0.5
