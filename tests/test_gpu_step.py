"""The fused SSP-RK3 step (gdg_ssprk3_step) against the oracle: the time step is chosen on the device
from the first stage's edge sweep (Sec. 3.3, eq. (MaxCFLdt)) and the three stages run in Shu-Osher form
(Sec. 6.2), the last one in place.  Also the device clock (t_end clipping, finished instances untouched)
and gdg_stage with U_out == U_base.  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

from paper_2402_04514_gb300 import assembly, workloads
from tests.helpers import four_quadrant_problem, octant_problem, periodic_vortex_problem, rel_err

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


CASES = {
    "sod1d_q1": lambda: (assembly.assemble_1d(200, 1), None),
    "oct_q1_3d": lambda: octant_problem((7, 6, 5), 1, seed=1),
    "vortex_q1_periodic": lambda: periodic_vortex_problem(17, 1),
    "fq_q2_slip": lambda: four_quadrant_problem(13, 2, seed=0),
    "fq_q1_slip": lambda: four_quadrant_problem(19, 1, seed=4),
    "fq_q3_slip": lambda: four_quadrant_problem(7, 3, seed=2),
}


def _setup(torch, name, cfl=0.5):
    from oracle.oracle import Oracle
    from paper_2402_04514_gb300.gdg import Solver

    P, U = CASES[name]()
    if U is None:
        U = workloads.sod(P.x[0])
    S, O = Solver(P), Oracle(P)
    S.set_clock(0.0, float("inf"), cfl)
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    work = (torch.empty_like(Ud), torch.empty_like(Ud))
    return P, U, S, O, Ud, work


@pytest.mark.parametrize("name", sorted(CASES))
def test_fused_step_matches_oracle(torch_cuda, name):
    """One fused step: its tau equals the oracle's max_dt (1e-13 relative) and its state equals the
    oracle's SSP-RK3 step taken with that tau (1e-12 relative per component)."""
    torch = torch_cuda
    P, U, S, O, Ud, work = _setup(torch, name)
    S.step(Ud, work)
    t, tau, steps = S.clock()
    tau_o = O.max_dt(U, 0.5)
    assert abs(tau - tau_o) <= 1e-13 * tau_o and t == tau and steps == 1
    ref, flags = O.ssprk3_step(U, tau)
    assert rel_err(Ud.cpu().numpy(), ref) <= STAGE_TOL
    assert S.status() == flags == 0


@pytest.mark.parametrize("name", ["sod1d_q1", "fq_q1_slip"])
def test_fused_hundred_steps(torch_cuda, name):
    """100 fused steps; the oracle steps with the tau the device chose (read from the clock)."""
    torch = torch_cuda
    P, U, S, O, Ud, work = _setup(torch, name)
    if name == "fq_q1_slip":
        from paper_2402_04514_gb300.gdg import Solver

        P, U = four_quadrant_problem(8, 1, seed=4)
        S, Ud = Solver(P), torch.from_numpy(np.ascontiguousarray(U)).cuda()
        from oracle.oracle import Oracle

        O = Oracle(P)
        work = (torch.empty_like(Ud), torch.empty_like(Ud))
    Uo = U.copy()
    t_prev = 0.0
    for _ in range(100):
        S.step(Ud, work)
        t, tau, _ = S.clock()
        assert t == t_prev + tau
        t_prev = t
        Uo, _ = O.ssprk3_step(Uo, tau)
    got = Ud.cpu().numpy()
    assert rel_err(got, Uo) <= LONG_TOL
    rho = got[0]
    eps = got[-1] - 0.5 * (got[1:-1] ** 2).sum(0) / rho
    assert (rho > 0).all() and (eps > 0).all()
    assert S.status() == 0


def test_clock_clips_to_t_end_and_finished_steps_are_no_ops(torch_cuda):
    """With t_end = 1.5 tau_0 the second step is clipped and lands on t_end exactly; a third step leaves
    the state and the clock untouched (it is not counted)."""
    torch = torch_cuda
    P, U, S, O, Ud, work = _setup(torch, "fq_q2_slip")
    tau0 = O.max_dt(U, 0.5)
    t_end = 1.5 * tau0
    S.set_clock(0.0, t_end, 0.5)
    S.step(Ud, work)
    t1, tau1, _ = S.clock()
    U1 = Ud.cpu().numpy()
    S.step(Ud, work)
    t2, tau2, n2 = S.clock()
    assert t2 == t_end and n2 == 2 and 0 < tau2 <= 0.5 * tau0 * (1 + 1e-12)
    ref, _ = O.ssprk3_step(U1, tau2)
    U2 = Ud.cpu().numpy()
    assert rel_err(U2, ref) <= STAGE_TOL
    work[0].fill_(float("nan"))
    S.step(Ud, work)
    t3, tau3, n3 = S.clock()
    assert t3 == t_end and tau3 == 0.0 and n3 == 2
    assert np.array_equal(Ud.cpu().numpy(), U2)
    assert S.status() == 0


def test_stage_in_place_on_its_base(torch_cuda):
    """gdg_stage with U_out == U_base gives the same state as with a separate output."""
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import Solver

    P, U = four_quadrant_problem(11, 2, seed=5)
    S = Solver(P)
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    tau = S.max_dt(Ud, 0.5)
    U1 = S.stage(Ud, tau)
    sep = S.stage(U1, tau, U_base=Ud, alpha=0.75)
    base = Ud.clone()
    S.stage(U1, tau, U_base=base, alpha=0.75, out=base)
    assert torch.equal(sep, base)


@pytest.mark.parametrize("name", ["fq_q2_slip", "fq_q1_slip", "sod1d_q1", "vortex_q1_periodic", "fq_q1_8"])
def test_ssprk54_step_matches_oracle(torch_cuda, name):
    """gdg_ssprk54_step against the oracle's SSPRK(5,4) step (oracle/ssprk.py) taken with the dt the device
    chose: dt = cfl * C * the forward-Euler bound (C = 1.508) to 1e-12, the state within 1e-12 relative
    after one step; after 30 steps within 1e-10 on the cases of the 100-step SSPRK3 test (the 100-step
    runs of both integrators on Q2, Q3 and 3D meshes follow below)."""
    torch = torch_cuda
    from oracle import ssprk

    long_run = name in ("sod1d_q1", "fq_q1_8")
    if name == "fq_q1_8":
        from oracle.oracle import Oracle
        from paper_2402_04514_gb300.gdg import Solver

        P, U = four_quadrant_problem(8, 1, seed=4)
        S, O = Solver(P), Oracle(P)
        S.set_clock(0.0, float("inf"), 0.5)
        Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
        work = (torch.empty_like(Ud), torch.empty_like(Ud))
    else:
        P, U, S, O, Ud, work = _setup(torch, name)
    work3 = (work[0], work[1], torch.empty_like(Ud))
    C = ssprk.ssp_coefficient(ssprk.SSPRK54_ALPHA, ssprk.SSPRK54_BETA)
    Uo = U.copy()
    for it in range(30 if long_run else 1):
        dt_o = 0.5 * C * O.max_dt(Uo, 1.0)
        S.step(Ud, work3)
        t, dt, steps = S.clock()
        assert abs(dt - dt_o) <= 1e-12 * dt_o and steps == it + 1
        Uo, flags = O.ssprk54_step(Uo, dt)
        assert flags == 0
        if it == 0:
            assert rel_err(Ud.cpu().numpy(), Uo) <= STAGE_TOL
    got = Ud.cpu().numpy()
    assert rel_err(got, Uo) <= (LONG_TOL if long_run else STAGE_TOL)
    rho = got[0]
    eps = got[-1] - 0.5 * (got[1:-1] ** 2).sum(0) / rho
    assert (rho > 0).all() and (eps > 0).all()
    assert S.status() == 0


@pytest.mark.parametrize("integrator", ["ssprk3", "ssprk54"])
@pytest.mark.parametrize("name", ["fq_q2_slip", "fq_q3_slip", "oct_q1_3d"])
def test_hundred_steps_q2_q3_3d(torch_cuda, name, integrator):
    """100 fused steps of the limited scheme on shocked data with Q2 (the degree of the 1024^2 bench
    workload, here 13^2 elements), Q3 (7^2) and 3D hexahedral Q1 (7 x 6 x 5), with either integrator; the
    oracle steps with the dt the device chose.  The whole trajectory stays within 1e-10 of the oracle's
    (per component, relative to max |U|); every state admissible; no flag raised."""
    torch = torch_cuda
    P, U, S, O, Ud, work = _setup(torch, name)
    if integrator == "ssprk54":
        work = (work[0], work[1], torch.empty_like(Ud))
    Uo = U.copy()
    worst = 0.0
    for it in range(100):
        S.step(Ud, work)
        _, dt, steps = S.clock()
        assert steps == it + 1
        if integrator == "ssprk3":
            Uo, flags = O.ssprk3_step(Uo, dt)
        else:
            Uo, flags = O.ssprk54_step(Uo, dt)
        assert flags == 0
        if it % 10 == 9:
            worst = max(worst, rel_err(Ud.cpu().numpy(), Uo))
    got = Ud.cpu().numpy()
    worst = max(worst, rel_err(got, Uo))
    assert worst <= LONG_TOL, worst
    rho = got[0]
    eps = got[-1] - 0.5 * (got[1:-1] ** 2).sum(0) / rho
    assert (rho > 0).all() and (eps > 0).all()
    assert S.status() == 0
