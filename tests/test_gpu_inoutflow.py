"""In- and outflow boundaries (Sec. 4.1) on the GPU against the oracle: stages of the first-order and
limited schemes, and fused steps, on a shock tube whose shock leaves the domain, a four-quadrant problem
with open sides, a supersonic stream (supersonic inflow, supersonic outflow and subsonic sides) and a 3D
octant problem with three open sides."""
import numpy as np
import pytest

from tests.helpers import inoutflow_case, rel_err

pytestmark = pytest.mark.gpu

STAGE_TOL = 1e-12
LONG_TOL = 1e-10
ILL_TOL = 3e-11  # per step on the supersonic stream: at least three times the oracle's own one-ulp move


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04514_gb300 import build

    build.build()
    return torch


def _case(name):
    return inoutflow_case(name)


NAMES = ["sod1d_open", "fq_q2_open_sides", "supersonic_stream", "oct_q1_3d_open"]


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("order", [0, 2])
def test_inoutflow_stage_parity(torch_cuda, name, order):
    torch = torch_cuda
    from oracle.oracle import Oracle
    from paper_2402_04514_gb300.gdg import Solver

    P, U, bd = _case(name)
    S, O = Solver(P, params=dict(order=order)), Oracle(P, params=dict(order=order))
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    bdd = torch.from_numpy(bd).cuda()
    tau_g = S.max_dt(Ud, 0.5, bdata=bdd)
    tau_o = O.max_dt(U, 0.5, bdata=bd)
    assert abs(tau_g - tau_o) <= 1e-13 * tau_o
    out = S.stage(Ud, tau_o, bdata=bdd)
    ref, flags = O.stage(U, tau_o, bdata=bd)
    assert rel_err(out.cpu().numpy(), ref) <= STAGE_TOL
    assert S.status() == flags == 0


@pytest.mark.parametrize("name", NAMES)
def test_inoutflow_fused_steps(torch_cuda, name):
    """20 fused SSP-RK3 steps with the in/outflow data: every step agrees within 3e-12 (three stages, each
    within the 1e-12 of a stage) with the oracle's step from the same state with the device's tau, and on
    the shock tube the 20-step trajectories agree within 1e-10.  The nearly uniform supersonic stream is
    the exception: there the entropy-viscosity ratio N = R/D of Sec. 5.2 is a ratio of quantities near
    their rounding level, and the oracle's own step moves by up to 6.6e-12 when its input changes by one
    ulp (test_oracle_bc.py::test_supersonic_stream_conditioning), so no implementation with another
    rounding order can be held to 3e-12 there; its bound is ILL_TOL, three times that sensitivity or more.
    Step 16 of the open-sided Q2 case holds a line search whose psi, evaluated with fused multiply-adds,
    sits below its rounding resolution near the root: it converges only because the iteration bisects
    whenever the bracket has not halved."""
    torch = torch_cuda
    from oracle.oracle import Oracle
    from paper_2402_04514_gb300.gdg import Solver

    P, U, bd = _case(name)
    S, O = Solver(P), Oracle(P)
    S.set_clock(0.0, float("inf"), 0.5)
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    bdd = torch.from_numpy(bd).cuda()
    work = (torch.empty_like(Ud), torch.empty_like(Ud))
    Uo = np.ascontiguousarray(U).copy()
    tol = ILL_TOL if name == "supersonic_stream" else 3 * STAGE_TOL
    for _ in range(20):
        before = Ud.cpu().numpy()
        S.step(Ud, work, bdata=bdd)
        tau = S.clock()[1]
        one, f = O.ssprk3_step(before, tau, lambda t: bd)
        assert f == 0
        assert rel_err(Ud.cpu().numpy(), one) <= tol
        Uo, _ = O.ssprk3_step(Uo, tau, lambda t: bd)
    if name == "sod1d_open":
        assert rel_err(Ud.cpu().numpy(), Uo) <= LONG_TOL
    assert S.status() == 0
