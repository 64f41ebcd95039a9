"""Launch schedules and the autotuner (gdg_autotune, gdg_batch_autotune): a schedule changes the launch
shapes only, so every schedule gives the same bits; the autotuner restores the state, the clock and the
flags it started from and installs a schedule drawn from its candidates; invalid schedules are refused."""
import numpy as np
import pytest

from paper_2402_04514_gb300 import assembly, workloads

pytestmark = pytest.mark.gpu

SCHEDULES = [
    dict(prim_threads=128, edge_threads=512, tau_threads=128, low_threads=512, limit2_threads=128,
         final_threads=512, high_block_cap=64, lsfix_slots=1),
    dict(prim_threads=512, edge_threads=128, tau_threads=512, low_threads=128, limit2_threads=512,
         final_threads=128, high_block_cap=96, lsfix_slots=16),
    dict(high_block_cap=37, lsfix_slots=3),  # a cap that is not a multiple of 32 (ragged blocks)
    dict(high_block_cap=288),  # the largest element block (32 Q2 elements)
    dict(row_slices=0),  # every row kernel in node order
    dict(row_slices=(1 << 2) | (1 << 5), high_block_cap=1),  # k_low and k_final sliced; one element per block
]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04514_gb300 import build

    build.build()
    return torch


def _instance(N, k, seed):
    P = assembly.assemble_2d(N, N, k)
    return P, np.ascontiguousarray(workloads.two_state_riemann(P.x[0], P.x[1], np.random.default_rng(seed)))


def _steps(torch, S, U, n):
    S.set_clock(0.0, float("inf"), 0.5)
    Ud = torch.from_numpy(U.copy()).cuda()
    work = (torch.empty_like(Ud), torch.empty_like(Ud))
    for _ in range(n):
        S.step(Ud, work)
    return Ud.cpu().numpy()


@pytest.mark.parametrize("degree", [1, 2])
def test_every_schedule_gives_the_same_bits(torch_cuda, degree):
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import Solver

    P, U = _instance(21, degree, 3)
    S = Solver(P)
    ref = _steps(torch, S, U, 3)
    for sc in SCHEDULES:
        S.set_schedule(**sc)
        assert np.array_equal(_steps(torch, S, U, 3), ref), sc


def test_autotune_restores_state_and_clock(torch_cuda):
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import Solver

    P, U = _instance(40, 2, 5)
    S = Solver(P)
    S.set_clock(0.0, 0.05, 0.5)
    Ud = torch.from_numpy(U.copy()).cuda()
    work = (torch.empty_like(Ud), torch.empty_like(Ud))
    S.step(Ud, work)
    before, clk = Ud.cpu().numpy(), S.clock()
    sc = S.autotune(Ud, work, trials=1)
    assert np.array_equal(Ud.cpu().numpy(), before) and S.clock() == clk and S.status() == 0
    for f in ("prim_threads", "edge_threads", "tau_threads", "low_threads", "limit2_threads", "final_threads"):
        assert sc[f] in (128, 256, 512)
    assert sc["high_block_cap"] in (36, 72, 144, 288) and sc["lsfix_slots"] in (1, 4, 16)  # 4..32 Q2 elements
    assert sc["row_slices"] & ~((1 << 1) | (1 << 2) | (1 << 4) | (1 << 5) | (1 << 8)) == 0
    # the tuned schedule continues the same trajectory as the default one
    S.step(Ud, work)
    S2 = Solver(P)
    S2.set_clock(0.0, 0.05, 0.5)
    U2 = torch.from_numpy(U.copy()).cuda()
    w2 = (torch.empty_like(U2), torch.empty_like(U2))
    S2.step(U2, w2)
    S2.step(U2, w2)
    assert np.array_equal(Ud.cpu().numpy(), U2.cpu().numpy())


def test_batch_autotune_and_schedules(torch_cuda):
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import Batch, Solver

    members = [_instance(N, 1, seed) for N, seed in ((9, 1), (17, 2), (30, 3))]
    solvers = [Solver(P) for P, _ in members]
    alone = [_steps(torch, S, U, 3) for S, (_, U) in zip(solvers, members)]
    states, works = [], []
    for S, (_, U) in zip(solvers, members):
        S.set_clock(0.0, float("inf"), 0.5)
        Ud = torch.from_numpy(U.copy()).cuda()
        states.append(Ud)
        works.append((torch.empty_like(Ud), torch.empty_like(Ud)))
    B = Batch(solvers, states, works)
    B.autotune(trials=1)
    for Ud, (_, U) in zip(states, members):  # autotuning left the members where they were
        assert np.array_equal(Ud.cpu().numpy(), U)
    B.set_schedule(**SCHEDULES[1])
    for _ in range(3):
        B.step()
    for Ud, want in zip(states, alone):
        assert np.array_equal(Ud.cpu().numpy(), want)


def test_invalid_schedules_are_refused(torch_cuda):
    from paper_2402_04514_gb300.gdg import GdgError, Solver

    P, _ = _instance(5, 1, 1)
    S = Solver(P)
    for bad in (dict(low_threads=96), dict(high_block_cap=0), dict(high_block_cap=289), dict(lsfix_slots=0),
                dict(row_slices=1 << 3)):
        with pytest.raises(GdgError):
            S.set_schedule(**bad)
