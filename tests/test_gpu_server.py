"""The serving loop (gdg_server_*): requests submitted while others run are admitted into the running
batches, each result equals, bit for bit, the same request solved alone with gdg_ssprk3_step to its end
time, admission respects the HBM budget, and gdg_footprint is the device memory gdg_setup takes."""
import time

import numpy as np
import pytest

from paper_2402_04514_gb300 import assembly, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04514_gb300 import build

    build.build()
    return torch


def _request(N, k, seed, vortex=False):
    P = assembly.assemble_2d(N, N, k)
    if vortex:  # the isentropic vortex of Sec. 6.2 scaled to the unit square (slip walls, so only nearly steady)
        U = workloads.vortex(10.0 * P.x[0] - 5.0, 10.0 * P.x[1] - 5.0, 0.0, gamma=1.4)
    else:
        U = workloads.two_state_riemann(P.x[0], P.x[1], np.random.default_rng(seed))
    return P, np.ascontiguousarray(U)


def _alone(torch, P, U, t_end, cfl=0.5):
    from paper_2402_04514_gb300.gdg import Solver

    S = Solver(P)
    S.set_clock(0.0, t_end, cfl)
    Ud = torch.from_numpy(U.copy()).cuda()
    work = (torch.empty_like(Ud), torch.empty_like(Ud))
    for _ in range(100000):
        S.step(Ud, work)
        t, _, steps = S.clock()
        if t >= t_end:
            break
    return Ud.cpu().numpy(), steps


def test_results_match_alone_with_requests_arriving_mid_run(torch_cuda):
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import Server

    # three long requests first, then shorter ones that arrive while those run
    specs = [(32, 2, 1, False, 0.05), (28, 1, 2, False, 0.08), (20, 1, 3, True, 0.03), (9, 2, 4, True, 0.015),
             (5, 1, 5, False, 0.005), (15, 2, 6, False, 0.02), (24, 1, 7, False, 0.01)]
    reqs = [(_request(N, k, seed, vortex), t_end) for N, k, seed, vortex, t_end in specs]
    srv = Server()
    ids = []
    for i, ((P, U), t_end) in enumerate(reqs):
        ids.append(srv.submit(P, U, t_end))
        if i == 2:
            time.sleep(0.02)
    results = [srv.wait(r, timeout=300.0) for r in ids]
    srv.close()
    late_joined_running = any(info["t_start"] < results[j][1]["t_done"] for j in range(3)
                              for _, info in results[3:])
    assert late_joined_running  # continuous batching: a late request started before an early one ended
    for ((P, U), t_end), (got, info) in zip(reqs, results):
        want, steps = _alone(torch, P, U, t_end)
        assert info["status"] == 0 and info["flags"] == 0
        assert info["t_final"] == t_end and info["steps"] == steps
        assert np.array_equal(got, want)
        assert info["t_submit"] <= info["t_start"] <= info["t_done"]


def test_admission_waits_for_memory(torch_cuda):
    """With a budget for about two requests at a time, every request completes, the memory in use never
    exceeds the budget, and later requests start only after earlier ones freed their memory."""
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import Server, footprint

    reqs = [(_request(16, 2, seed), 0.01) for seed in range(6)]
    one = footprint(reqs[0][0][0]) + 3 * 4 * reqs[0][0][0].n * 8 + 4096
    srv = Server(hbm_budget=int(2.5 * one))
    ids = [srv.submit(P, U, t_end) for (P, U), t_end in reqs]
    peak = 0
    deadline = time.time() + 300
    while time.time() < deadline:
        st = srv.stats()
        peak = max(peak, st["bytes_in_use"])
        assert st["bytes_in_use"] <= st["budget"]
        if st["queued"] == 0 and st["active"] == 0:
            break
        time.sleep(0.002)
    results = [srv.wait(r, timeout=300.0) for r in ids]
    srv.close()
    assert all(info["status"] == 0 for _, info in results)
    starts = sorted(info["t_start"] for _, info in results)
    dones = sorted(info["t_done"] for _, info in results)
    assert starts[2] >= dones[0]  # the third admission waited for a completion
    assert peak <= int(2.5 * one)


def test_oversized_request_is_refused_and_footprint_is_exact(torch_cuda):
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import GdgError, Server, Solver, footprint

    P, U = _request(10, 2, 1)
    assert footprint(P) == Solver(P).info()["device_bytes"]
    srv = Server(hbm_budget=footprint(P) // 2)
    with pytest.raises(GdgError):
        srv.submit(P, U, 0.01)
    srv.close()


def test_served_requests_against_the_oracle(torch_cuda):
    """Requests served together (two Q2 and one Q1 two-state Riemann problems, submitted at once so that
    the Q2 ones share a batch) against the oracle directly: the oracle steps each request
    with its own time step of Sec. 3.3 (Cr = 0.5, the last step clipped to the end time) and the served
    result equals its trajectory within 1e-10 relative per component, with the same number of steps."""
    torch = torch_cuda
    from oracle.oracle import Oracle
    from paper_2402_04514_gb300.gdg import Server
    from tests.helpers import rel_err

    reqs = [(_request(7, 2, 21), 0.02), (_request(11, 1, 22), 0.03), (_request(5, 2, 23), 0.015)]
    srv = Server()
    ids = [srv.submit(P, U, t_end) for (P, U), t_end in reqs]
    results = [srv.wait(r, timeout=300.0) for r in ids]
    srv.close()
    for ((P, U), t_end), (got, info) in zip(reqs, results):
        O = Oracle(P)
        V, t, steps = U.copy(), 0.0, 0
        while t < t_end:
            tau = min(O.max_dt(V, 0.5), t_end - t)
            V, flags = O.ssprk3_step(V, tau)
            assert flags == 0
            t = t + tau if t + tau < t_end else t_end
            steps += 1
        assert info["status"] == 0 and info["flags"] == 0 and info["steps"] == steps
        assert rel_err(got, V) <= 1e-10
