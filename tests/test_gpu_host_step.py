"""gdg_ssprk3_step_host: the fused SSP-RK3 step (Sec. 6.2) of a state kept in host memory.  Page-locked
input is read by the first stage's primitive sweep over the host link, and page-locked output (with
page-locked input) is written by the last stage's sweeps; other buffers go through cudaMemcpyAsync.  Every
way the result must be bit for bit the device step's (the same kernels on the same values), and the device
step is compared with the oracle here once more and in test_gpu_step."""
import numpy as np
import pytest

from tests.helpers import dirichlet_vortex_problem, four_quadrant_problem, octant_problem, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04514_gb300 import build

    build.build()
    return torch


CASES = {  # (problem, state, Dirichlet data at time t or None, gamma)
    "fq_q2_slip": lambda: four_quadrant_problem(13, 2, seed=0) + (None, 1.4),
    "fq_q3_slip": lambda: four_quadrant_problem(7, 3, seed=2) + (None, 1.4),
    "oct_q1_3d": lambda: octant_problem((7, 6, 5), 1, seed=1) + (None, 1.4),
    "vortex_q2_dirichlet": lambda: dirichlet_vortex_problem(8, 2) + (5.0 / 3.0,),
}


def _pair(torch, name, params=None):
    """Two solvers on the same problem and clock: one for the device step, one for the host step."""
    from paper_2402_04514_gb300.gdg import Solver

    P, U, bfun, gamma = CASES[name]()
    bd = None if bfun is None else bfun(0.0)
    solvers = []
    for _ in range(2):
        S = Solver(P, gamma=gamma, params=params)
        S.set_clock(0.0, float("inf"), 0.5)
        solvers.append(S)
    return P, np.ascontiguousarray(U), bd, solvers, gamma


def _dev(torch, bd):
    return None if bd is None else torch.from_numpy(np.ascontiguousarray(bd)).cuda()


def _device_steps(torch, S, U0, bd, k):
    """The states after each of k device steps, and the first step's tau."""
    bd = _dev(torch, bd)
    Ud = torch.from_numpy(U0.copy()).cuda()
    work = (torch.empty_like(Ud), torch.empty_like(Ud))
    out = []
    for _ in range(k):
        S.step(Ud, work, bdata=bd)
        out.append(Ud.cpu().numpy().copy())
        if len(out) == 1:
            tau1 = S.clock()[1]
    return out, tau1


@pytest.mark.parametrize("name", sorted(CASES))
def test_pinned_host_step_equals_device_step(torch_cuda, name):
    """Three steps with page-locked host buffers (in and out alternating) equal the device steps bit for
    bit, clocks included; the first equals the oracle's step with the device's tau to 1e-12."""
    torch = torch_cuda
    from oracle.oracle import Oracle

    P, U0, bd, (Sd, Sh), gamma = _pair(torch, name)
    ref, tau1 = _device_steps(torch, Sd, U0, bd, 3)
    hin = torch.from_numpy(U0.copy()).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    U = torch.empty(U0.shape, dtype=torch.float64, device="cuda")
    work = (torch.empty_like(U), torch.empty_like(U))
    for k in range(3):
        hout.fill_(np.nan)
        Sh.step_host(hin, hout, U, work, bdata=_dev(torch, bd))
        torch.cuda.current_stream().synchronize()
        assert np.array_equal(hout.numpy(), ref[k]), k
        assert np.array_equal(U.cpu().numpy(), ref[k]), k
        hin, hout = hout, hin
    assert Sh.clock() == Sd.clock()
    assert Sh.status() == Sd.status() == 0
    O = Oracle(P, gamma=gamma)
    tau = O.max_dt(U0, 0.5, bdata=bd)
    assert abs(tau1 - tau) <= 1e-13 * tau
    first, _ = O.ssprk3_step(U0, tau, bdata_fn=None if bd is None else (lambda t: bd))
    assert rel_err(ref[0], first) <= 1e-12


def test_pageable_mixed_and_aliased_host_buffers(torch_cuda):
    """numpy (pageable) buffers take the copy path; page-locked input with pageable output, and pageable
    input with page-locked output, take it on one side; one page-locked buffer may be both input and
    output.  Every combination gives the device step's bits."""
    torch = torch_cuda
    P, U0, bd, (Sd, Sh), _ = _pair(torch, "fq_q2_slip")
    ref, _ = _device_steps(torch, Sd, U0, bd, 4)
    U = torch.empty(U0.shape, dtype=torch.float64, device="cuda")
    work = (torch.empty_like(U), torch.empty_like(U))
    sync = torch.cuda.current_stream().synchronize
    a, b = U0.copy(), np.full_like(U0, np.nan)
    Sh.step_host(a, b, U, work)
    sync()
    assert np.array_equal(b, ref[0]) and np.array_equal(a, U0)
    pin_in, page_out = torch.from_numpy(b.copy()).pin_memory(), np.full_like(U0, np.nan)
    Sh.step_host(pin_in, page_out, U, work)
    sync()
    assert np.array_equal(page_out, ref[1])
    pin_out = torch.full(U0.shape, np.nan, dtype=torch.float64).pin_memory()
    Sh.step_host(page_out, pin_out, U, work)
    sync()
    assert np.array_equal(pin_out.numpy(), ref[2])
    Sh.step_host(pin_out, pin_out, U, work)
    sync()
    assert np.array_equal(pin_out.numpy(), ref[3])


@pytest.mark.parametrize("order,passes", [(0, 2), (1, 2), (2, 1), (2, 0)])
def test_host_output_from_every_final_writer(torch_cuda, order, passes):
    """The last stage's output, and its host copy, come from the low-order sweep (order LOW, or no limiter
    pass), the element sweep (order HIGH) or sweep C (one pass): each gives the device step's bits."""
    torch = torch_cuda
    P, U0, bd, (Sd, Sh), _ = _pair(torch, "fq_q2_slip", params=dict(order=order, limiter_passes=passes))
    ref, _ = _device_steps(torch, Sd, U0, bd, 2)
    hin = torch.from_numpy(U0.copy()).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    U = torch.empty(U0.shape, dtype=torch.float64, device="cuda")
    work = (torch.empty_like(U), torch.empty_like(U))
    for k in range(2):
        hout.fill_(np.nan)
        Sh.step_host(hin, hout, U, work)
        torch.cuda.current_stream().synchronize()
        assert np.array_equal(hout.numpy(), ref[k]), k
        hin, hout = hout, hin


def test_mixed_precision_host_step(torch_cuda):
    """The mixed-precision instantiation of the primitive sweep reads host input the same way."""
    torch = torch_cuda
    P, U0, bd, (Sd, Sh), _ = _pair(torch, "fq_q2_slip", params=dict(precision=1))
    ref, _ = _device_steps(torch, Sd, U0, bd, 2)
    hin = torch.from_numpy(U0.copy()).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    U = torch.empty(U0.shape, dtype=torch.float64, device="cuda")
    work = (torch.empty_like(U), torch.empty_like(U))
    for k in range(2):
        Sh.step_host(hin, hout, U, work)
        torch.cuda.current_stream().synchronize()
        assert np.array_equal(hout.numpy(), ref[k]), k
        hin, hout = hout, hin


def test_finished_clock_copies_the_state_through(torch_cuda):
    """With t = t_end the step changes nothing: the host output and U both receive the input unchanged,
    and the clock does not move."""
    torch = torch_cuda
    P, U0, bd, (_, Sh), _ = _pair(torch, "fq_q2_slip")
    Sh.set_clock(1.0, 1.0, 0.5)
    hin = torch.from_numpy(U0.copy()).pin_memory()
    hout = torch.full_like(hin, np.nan).pin_memory()
    U = torch.full(U0.shape, np.nan, dtype=torch.float64, device="cuda")
    work = (torch.empty_like(U), torch.empty_like(U))
    Sh.step_host(hin, hout, U, work)
    torch.cuda.current_stream().synchronize()
    assert np.array_equal(hout.numpy(), U0) and np.array_equal(U.cpu().numpy(), U0)
    t, tau, steps = Sh.clock()
    assert t == 1.0 and steps == 0


def test_host_step_argument_checks(torch_cuda):
    """Aliased device buffers are refused before anything runs."""
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import GdgError

    P, U0, bd, (_, Sh), _ = _pair(torch, "fq_q2_slip")
    U = torch.empty(U0.shape, dtype=torch.float64, device="cuda")
    T = torch.empty_like(U)
    with pytest.raises(GdgError):
        Sh.step_host(U0, U0.copy(), U, (U, T))
