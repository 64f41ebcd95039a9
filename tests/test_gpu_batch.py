"""Batches (gdg_batch_*): instances of different sizes, data and end times advanced in shared launches
give, bit for bit, the states and clocks of the same instances stepped alone with gdg_ssprk3_step (which
test_gpu_step checks against the oracle); a member's result does not depend on who else is in the batch."""
import numpy as np
import pytest

from paper_2402_04514_gb300 import assembly, workloads
from tests.helpers import dirichlet_vortex_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04514_gb300 import build

    build.build()
    return torch


def _riemann_instance(N, k, seed):
    P = assembly.assemble_2d(N, N, k)
    rng = np.random.default_rng(seed)
    U = workloads.two_state_riemann(P.x[0], P.x[1], rng)
    return P, U


def _members(torch, specs):
    """specs: (N, degree, seed, f): the member's end time is f times its first time step (inf: none).
    Returns solvers, initial states (numpy) and t_end per member."""
    from paper_2402_04514_gb300.gdg import Solver

    out = []
    for N, k, seed, f in specs:
        P, U = _riemann_instance(N, k, seed)
        S = Solver(P)
        U = np.ascontiguousarray(U)
        t_end = np.inf if not np.isfinite(f) else f * S.max_dt(torch.from_numpy(U).cuda(), 0.5)
        out.append((S, U, t_end))
    return out


def _run_alone(torch, members, steps):
    res = []
    for S, U, t_end in members:
        S.set_clock(0.0, t_end, 0.5)
        Ud = torch.from_numpy(U.copy()).cuda()
        work = (torch.empty_like(Ud), torch.empty_like(Ud))
        for _ in range(steps):
            S.step(Ud, work)
        res.append((Ud.cpu().numpy(), S.clock()))
    return res


def _run_batch(torch, members, steps, order=None, stream=None, persistent=False):
    from paper_2402_04514_gb300.gdg import Batch

    order = order or list(range(len(members)))
    sel = [members[i] for i in order]
    states, works = [], []
    for S, U, t_end in sel:
        S.set_clock(0.0, t_end, 0.5)
        Ud = torch.from_numpy(U.copy()).cuda()
        states.append(Ud)
        works.append((torch.empty_like(Ud), torch.empty_like(Ud)))
    B = Batch([m[0] for m in sel], states, works)
    if persistent:
        B.set_persistent(True)
    torch.cuda.synchronize()
    for _ in range(steps):
        B.step(stream=stream)  # on a stream of its own the step is captured once and replayed as a graph
    torch.cuda.synchronize()
    res = {}
    for i, (S, _, _), Ud in zip(order, sel, states):
        res[i] = (Ud.cpu().numpy(), S.clock())
    B.close()
    return res


@pytest.mark.parametrize("degree", [1, 2])
def test_batch_equals_each_member_alone(torch_cuda, degree):
    """Members of ragged sizes (several blocks with a partial last one, and one smaller than a block),
    two of which reach their end time inside the run: same bits and clocks as alone, in two batch
    orders, and with the step replayed as a CUDA graph on a stream of its own."""
    torch = torch_cuda
    specs = [(13, degree, 1, np.inf), (3, degree, 2, np.inf), (21, degree, 3, 2.5), (8, degree, 4, np.inf),
             (17, degree, 5, 1.5), (4, degree, 6, np.inf), (11, degree, 7, np.inf)]
    members = _members(torch, specs)
    steps = 6
    alone = _run_alone(torch, members, steps)
    for order, stream in ((None, None), ([4, 0, 6, 2, 5, 1, 3], None), (None, torch.cuda.Stream())):
        got = _run_batch(torch, members, steps, order, stream)
        for i, (U_a, clk_a) in enumerate(alone):
            U_b, clk_b = got[i]
            assert np.array_equal(U_a, U_b), i
            assert clk_a == clk_b, (i, clk_a, clk_b)
    # the members with an end time inside the run stopped on it
    for i, (S, U, t_end) in enumerate(members):
        t, tau, steps_done = alone[i][1]
        if np.isfinite(t_end):  # the steps after t_end did nothing and were not counted
            assert t == t_end and tau == 0.0 and steps_done < steps
        else:
            assert steps_done == steps
    for S, _, _ in members:
        assert S.status() == 0


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_persistent_batch_equals_each_member_alone(torch_cuda, degree):
    """The persistent mode (one cooperative launch per stage, grid-wide barriers between the phases):
    members of ragged sizes, two of them reaching their end time inside the run, give the same bits and
    clocks as alone, in two batch orders and on a stream of its own."""
    torch = torch_cuda
    specs = [(13, degree, 1, np.inf), (3, degree, 2, np.inf), (21, degree, 3, 2.5), (8, degree, 4, np.inf),
             (17, degree, 5, 1.5), (4, degree, 6, np.inf)]
    members = _members(torch, specs)
    steps = 5
    alone = _run_alone(torch, members, steps)
    for order, stream in ((None, None), ([4, 0, 5, 2, 1, 3], torch.cuda.Stream())):
        got = _run_batch(torch, members, steps, order, stream, persistent=True)
        for i, (U_a, clk_a) in enumerate(alone):
            U_b, clk_b = got[i]
            assert np.array_equal(U_a, U_b), i
            assert clk_a == clk_b, (i, clk_a, clk_b)
    for S, _, _ in members:
        assert S.status() == 0


@pytest.mark.parametrize("degree", [1, 2])
def test_batch_of_3d_members(torch_cuda, degree):
    """Hexahedral members of ragged sizes (eight-octant data, slip walls), one reaching its end time inside
    the run: the same bits and clocks as alone."""
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import Solver
    from tests.helpers import octant_problem

    members = []
    for shape, seed, f in (((5, 4, 3), 1, np.inf), ((2, 2, 2), 2, np.inf), ((6, 3, 4), 3, 1.5)):
        P, U = octant_problem(shape, degree, seed=seed)
        S = Solver(P)
        U = np.ascontiguousarray(U)
        t_end = np.inf if not np.isfinite(f) else f * S.max_dt(torch.from_numpy(U).cuda(), 0.5)
        members.append((S, U, t_end))
    steps = 4
    alone = _run_alone(torch, members, steps)
    for persistent in (False, True):
        got = _run_batch(torch, members, steps, [2, 0, 1], persistent=persistent)
        for i, (U_a, clk_a) in enumerate(alone):
            U_b, clk_b = got[i]
            assert np.array_equal(U_a, U_b), (i, persistent)
            assert clk_a == clk_b, (i, clk_a, clk_b)
    assert alone[2][1][2] < steps  # the third member stopped at its end time
    for S, _, _ in members:
        assert S.status() == 0


def test_batch_with_dirichlet_members(torch_cuda):
    """Members with Dirichlet boundary data (time-independent here) next to slip-wall members."""
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import Batch, Solver

    P1, U1, bd1 = dirichlet_vortex_problem(9, 1)
    P2, U2 = _riemann_instance(10, 1, 11)
    S1, S2 = Solver(P1, gamma=5.0 / 3.0), Solver(P2)
    b1 = bd1(0.0)
    b1d = torch.from_numpy(np.ascontiguousarray(b1)).cuda()
    ref = []
    for S, U, bd in ((S1, U1, b1d), (S2, U2, None)):
        S.set_clock(0.0, np.inf, 0.4)
        Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
        work = (torch.empty_like(Ud), torch.empty_like(Ud))
        for _ in range(4):
            S.step(Ud, work, bdata=bd)
        ref.append(Ud.cpu().numpy())
    states, works = [], []
    for S, U in ((S1, U1), (S2, U2)):
        S.set_clock(0.0, np.inf, 0.4)
        Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
        states.append(Ud)
        works.append((torch.empty_like(Ud), torch.empty_like(Ud)))
    B = Batch([S1, S2], states, works, [b1d, None])
    for _ in range(4):
        B.step()
    for r, Ud in zip(ref, states):
        assert np.array_equal(r, Ud.cpu().numpy())


def test_batch_rejects_inconsistent_members(torch_cuda):
    """Members of different element types, a member listed twice, and aliased buffers are refused."""
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import Batch, GdgError, Solver

    (S1, U1, _), (S2, U2, _) = _members(torch, [(5, 1, 1, np.inf), (5, 2, 2, np.inf)])
    Ua = torch.from_numpy(U1).cuda()
    Ub = torch.from_numpy(U2).cuda()
    wa = (torch.empty_like(Ua), torch.empty_like(Ua))
    wb = (torch.empty_like(Ub), torch.empty_like(Ub))
    with pytest.raises(GdgError):
        Batch([S1, S2], [Ua, Ub], [wa, wb])
    with pytest.raises(GdgError):
        Batch([S1, S1], [Ua, Ua.clone()], [wa, (torch.empty_like(Ua), torch.empty_like(Ua))])
    with pytest.raises(GdgError):
        Batch([S1], [Ua], [(Ua, wa[1])])


@pytest.mark.parametrize("degree", [1, 2])
def test_batch_members_against_the_oracle(torch_cuda, degree):
    """Members of a batch of ragged sizes against the oracle directly: after each of five batch steps,
    every member equals the oracle's SSP-RK3 step from the member's previous state, taken with the dt the
    member's clock chose (three stages, each within the 1e-12 of a stage: 3e-12 relative per component),
    and each member's five-step trajectory stays within 1e-10 of the oracle's."""
    torch = torch_cuda
    from oracle.oracle import Oracle
    from paper_2402_04514_gb300.gdg import Batch, Solver
    from tests.helpers import rel_err

    specs = [(13, 1), (3, 2), (9, 3), (6, 4)]
    members = []
    for N, seed in specs:
        P, U = _riemann_instance(N, degree, seed)
        S = Solver(P)
        S.set_clock(0.0, np.inf, 0.5)
        Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
        members.append((S, Oracle(P), Ud, (torch.empty_like(Ud), torch.empty_like(Ud)), np.ascontiguousarray(U)))
    B = Batch([m[0] for m in members], [m[2] for m in members], [m[3] for m in members])
    traj = [m[4].copy() for m in members]
    for step in range(5):
        before = [m[2].cpu().numpy() for m in members]
        B.step()
        torch.cuda.synchronize()
        for k, (S, O, Ud, _, _) in enumerate(members):
            _, dt, steps = S.clock()
            assert steps == step + 1
            one, flags = O.ssprk3_step(before[k], dt)
            assert flags == 0
            got = Ud.cpu().numpy()
            assert rel_err(got, one) <= 3e-12, (k, step)
            traj[k], _ = O.ssprk3_step(traj[k], dt)
            assert rel_err(got, traj[k]) <= 1e-10, (k, step)
    for S, *_ in members:
        assert S.status() == 0
