"""In- and outflow boundaries (Sec. 4.1) on the GPU against the oracle: stages of the first-order and
limited schemes, and fused steps, on a shock tube whose shock leaves the domain, a four-quadrant problem
with open sides, a supersonic stream (supersonic inflow, supersonic outflow and subsonic sides) and a 3D
octant problem with three open sides."""
import numpy as np
import pytest

from paper_2402_04514_gb300 import assembly, workloads
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu

STAGE_TOL = 1e-12
LONG_TOL = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04514_gb300 import build

    build.build()
    return torch


def _case(name):
    if name == "sod1d_open":
        P = assembly.assemble_1d(200, 1, bc=("inoutflow", "inoutflow"))
        U = workloads.sod(P.x[0])
        return P, U, np.ascontiguousarray(workloads.sod(P.b_x[0]))
    if name == "oct_q1_3d_open":
        from tests.helpers import octant_problem
        P, U = octant_problem((5, 4, 4), 1, seed=3, bc=dict(left="inoutflow", right="inoutflow", back="inoutflow"))
        return P, U, np.ascontiguousarray(U[:, P.b_node])
    if name == "fq_q2_open_sides":
        P = assembly.assemble_2d(13, 13, 2, bc=dict(left="inoutflow", right="inoutflow"))
        U = workloads.four_quadrant(P.x[0], P.x[1], seed=0)
        return P, U, np.ascontiguousarray(U[:, P.b_node])
    # supersonic stream (Mach ~2.6 along x) over a density bump
    sides = dict(left="inoutflow", right="inoutflow", bottom="inoutflow", top="inoutflow")
    P = assembly.assemble_2d(16, 16, 1, bc=sides)
    x, y = P.x
    rho = 1.0 + 0.5 * np.exp(-40 * ((x - 0.4) ** 2 + (y - 0.5) ** 2))
    U = workloads.prim_to_cons(rho, np.stack([np.full(P.n, 3.0), np.full(P.n, 0.5)]), np.full(P.n, 1.0), 1.4)
    bd = workloads.prim_to_cons(np.full(P.nb, 1.0), np.stack([np.full(P.nb, 3.0), np.full(P.nb, 0.5)]),
                                np.full(P.nb, 1.0), 1.4)
    return P, U, np.ascontiguousarray(bd)


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
    the shock tube the 20-step trajectories agree within 1e-10.  (On the nearly uniform supersonic stream the entropy-viscosity ratio N = R/D of Sec. 5.2 is
    ill-conditioned, so two trajectories drift apart faster; the per-step agreement is the test there.)
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
    for _ in range(20):
        before = Ud.cpu().numpy()
        S.step(Ud, work, bdata=bdd)
        tau = S.clock()[1]
        one, f = O.ssprk3_step(before, tau, lambda t: bd)
        assert f == 0
        assert rel_err(Ud.cpu().numpy(), one) <= 3 * STAGE_TOL
        Uo, _ = O.ssprk3_step(Uo, tau, lambda t: bd)
    if name == "sod1d_open":
        assert rel_err(Ud.cpu().numpy(), Uo) <= LONG_TOL
    assert S.status() == 0
