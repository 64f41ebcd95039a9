"""The mixed-precision path (GDG_PRECISION_MIXED, include/gdg.h) against the FP64 oracle and the FP64
path: its wave-speed bound never falls below the FP64 one and is symmetric bit for bit; one stage agrees
with the oracle to MIXED_STAGE_TOL; the invariants hold as in the FP64 path (conservation to FP64
rounding, rho > 0 and eps > 0, the local bounds enforced exactly); the accuracy on a smooth solution is
that of the FP64 path; batches of mixed members give the bits of the members alone."""
import numpy as np
import pytest

from paper_2402_04514_gb300 import assembly, workloads
from tests.helpers import (consolidated_l1, dirichlet_vortex_problem, four_quadrant_problem, octant_problem,
                           periodic_vortex_problem, rel_err)

pytestmark = pytest.mark.gpu

MIXED = dict(precision=1)
# One stage of the mixed path against the FP64 oracle, per component max |dU| / max |U|.  The difference
# comes from the raised wave-speed bound (by 2^-16 S, S <= 2 lambda + |u_L| + |u_R|, so d_ij^L by a
# relative 2e-5 to 2e-4) and from FP32 rounding (1e-7) of the other coefficients; both scale with tau d / m.
MIXED_STAGE_TOL = 2e-5
MARGIN_CLAIM = 2.0 ** -17  # the FP32 bound's error relative to S before the margin (gdg_internal.cuh)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04514_gb300 import build

    build.build()
    return torch


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _riemann_states(rng, n, gamma):
    """rho, p log-uniform over eight decades; normal velocities up to 30 sound speeds either way, with
    families that hit the formula's switches: equal states, two rarefactions, strong collisions, p~ near
    p_L or p_R, and nearly cancelling numerators."""
    rL, rR, pL, pR = np.exp(rng.uniform(np.log(1e-4), np.log(1e4), (4, n)))
    aL, aR = np.sqrt(gamma * pL / rL), np.sqrt(gamma * pR / rR)
    uL = rng.uniform(-30, 30, n) * aL
    uR = rng.uniform(-30, 30, n) * aR
    k = n // 6
    # equal states
    rR[:k], pR[:k], uR[:k], aR[:k] = rL[:k], pL[:k], uL[:k], aL[:k]
    # near-vacuum: the numerator a_L + a_R - (gamma - 1)/2 (u_R - u_L) close to zero
    s = slice(k, 2 * k)
    uR[s] = uL[s] + 2.0 * (aL[s] + aR[s]) / (gamma - 1.0) * (1.0 + rng.uniform(-1e-3, 1e-3, k))
    # mild jumps (p~ close to p_L and p_R)
    s = slice(2 * k, 3 * k)
    pR[s] = pL[s] * (1.0 + rng.uniform(-1e-3, 1e-3, k))
    rR[s] = rL[s] * (1.0 + rng.uniform(-1e-3, 1e-3, k))
    aR[s] = np.sqrt(gamma * pR[s] / rR[s])
    uR[s] = uL[s] + rng.uniform(-1e-3, 1e-3, k) * aL[s]
    return np.stack([rL, uL, pL, rR, uR, pR], 1)


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0, 1.3])
def test_wave_speed_bound_dominates_the_fp64_bound(torch_cuda, gamma):
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import wave_speed_check

    rng = np.random.default_rng(11)
    st = _riemann_states(rng, 600000, gamma)
    out = wave_speed_check(gamma, _dev(torch, st)).cpu().numpy()
    lam64, lmx, raw, S = out.T
    assert np.isfinite(out).all()
    assert (lmx >= lam64).all(), np.argmin(lmx - lam64)
    err = np.abs(raw - lam64) / S
    print(f"gamma {gamma}: max |lambda32 - lambda64| / S = {err.max():.3e} (2^{np.log2(err.max()):.1f}); "
          f"max (lambda_mx / lambda64 - 1) = {(lmx / np.maximum(lam64, 1e-300) - 1).max():.3e}")
    assert err.max() <= MARGIN_CLAIM
    # (L, R, n) -> (R, L, -n): the same bits (the FP64 formula contracts a_L p_L^-e + a_R p_R^-e into an
    # FMA and is symmetric only to an ulp; both paths evaluate d_ij^L once per edge)
    sw = st[:, [3, 4, 5, 0, 1, 2]].copy()
    sw[:, [1, 4]] *= -1.0
    out_sw = wave_speed_check(gamma, _dev(torch, sw)).cpu().numpy()
    assert np.array_equal(out_sw[:, 1], lmx)


CASES = [
    ("sod1d_q1", lambda: (assembly.assemble_1d(200, 1), None)),
    ("vortex_q1_periodic", lambda: periodic_vortex_problem(17, 1)),
    ("fq_q2_slip", lambda: four_quadrant_problem(13, 2, seed=0)),
    ("fq_q1_slip", lambda: four_quadrant_problem(19, 1, seed=4)),
    ("fq_q3_slip", lambda: four_quadrant_problem(7, 3, seed=2)),
    ("oct_q2_3d", lambda: octant_problem((4, 3, 3), 2, seed=2)),
]


def _problem(name):
    P, U = dict(CASES)[name]()
    if U is None:
        U = workloads.sod(P.x[0])
    return P, U


@pytest.mark.parametrize("name", [c[0] for c in CASES])
@pytest.mark.parametrize("order", [0, 1, 2])
def test_stage_against_the_oracle(torch_cuda, name, order):
    torch = torch_cuda
    from oracle.oracle import Oracle
    from paper_2402_04514_gb300.gdg import Solver

    P, U = _problem(name)
    S = Solver(P, params=dict(MIXED, order=order))
    O = Oracle(P, params=dict(order=order))
    Ud = _dev(torch, U)
    tau_o = O.max_dt(U, 0.5)
    tau_g = S.max_dt(Ud, 0.5)
    assert tau_o * (1 - 2e-4) <= tau_g <= tau_o  # a raised wave-speed bound gives a smaller step
    out = S.stage(Ud, tau_o, U_base=_dev(torch, U * 1.01), alpha=0.75)
    ref, flags = O.stage(U, tau_o, U_base=U * 1.01, alpha=0.75)
    torch.cuda.synchronize()
    e = rel_err(out.cpu().numpy(), ref)
    print(f"{name} order {order}: stage rel err {e:.3e}")
    assert e <= MIXED_STAGE_TOL
    assert S.status() == flags == 0
    _, _, tr = O.stage(U, tau_o, trace=True)
    S.stage(Ud, tau_o)
    dL = S.export("dL")
    assert (dL >= tr["dL"]).all()
    assert (dL <= tr["dL"] * (1 + 2.0 ** -11)).all()


@pytest.mark.parametrize("name,degree", [("fq_q2_slip", 2), ("fq_q1_slip", 1)])
def test_invariants_over_fused_steps(torch_cuda, name, degree):
    """Thirty fused SSP-RK3 steps of the limited scheme on shocked four-quadrant data with slip walls:
    the totals of rho and E stay constant to FP64 rounding (as in the FP64 path), every state is
    admissible, and a final stage lands inside the local bounds it exported."""
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import Solver

    P, U = four_quadrant_problem(24, degree, seed=3)
    drift = {}
    for prec in (0, 1):
        S = Solver(P, params=dict(precision=prec))
        S.set_clock(0.0, float("inf"), 0.5)
        Ud = _dev(torch, U)
        work = (torch.empty_like(Ud), torch.empty_like(Ud))
        tot0 = (P.mi * U).sum(1)
        worst = 0.0
        for _ in range(30):
            S.step(Ud, work)
            tot = (P.mi * Ud.cpu().numpy()).sum(1)
            worst = max(worst, max(abs(tot[c] - tot0[c]) / abs(tot0[c]) for c in (0, 3)))
        assert S.status() == 0
        drift[prec] = worst
        if prec == 1:
            got = Ud.cpu().numpy()
            rho = got[0]
            eps = got[-1] - 0.5 * (got[1:-1] ** 2).sum(0) / rho
            assert (rho > 0).all() and (eps > 0).all()
            tau = S.max_dt(Ud, 0.5)
            out = S.stage(Ud, tau).cpu().numpy()
            rmin, rmax, smin = S.export("rho_min"), S.export("rho_max"), S.export("s_min")
            rho = out[0]
            st = rho ** (-1.4) * (out[-1] - 0.5 * (out[1:-1] ** 2).sum(0) / rho)
            assert (rho >= rmin * (1 - 1e-13)).all() and (rho <= rmax * (1 + 1e-13)).all()
            assert (st >= smin * (1 - 1e-12)).all()
    print(f"{name}: relative drift of the rho and E totals over 30 steps: fp64 {drift[0]:.2e}, mixed {drift[1]:.2e}")
    assert drift[1] <= 1e-13


def test_accuracy_on_the_vortex_matches_fp64(torch_cuda):
    """The isentropic vortex (gamma = 5/3, exact Dirichlet data) on Q2 to t = 0.5: the L1 error of the
    mixed path is that of the FP64 path within 1%."""
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import Solver

    g = 5.0 / 3.0
    P, U0, bdata = dirichlet_vortex_problem(16, 2, gamma=g)
    errs = {}
    for prec in (0, 1):
        S = Solver(P, gamma=g, params=dict(precision=prec))
        Ud = _dev(torch, U0)
        bufs = (torch.empty_like(Ud), torch.empty_like(Ud))
        out = torch.empty_like(Ud)
        t, tF = 0.0, 0.5
        while t < tF - 1e-12:
            bd = _dev(torch, bdata(t))
            dt = min(S.max_dt(Ud, 0.5, bdata=bd), tF - t)
            S.ssprk3_step(Ud, dt, bufs, out, bdata_fn=lambda s: _dev(torch, bdata(s)), t=t)
            Ud, out = out, Ud
            t += dt
        assert S.status() == 0
        errs[prec] = consolidated_l1(P, Ud.cpu().numpy(), workloads.vortex(P.x[0], P.x[1], tF, gamma=g))
    print(f"vortex Q2 L1: fp64 {errs[0]:.6e} mixed {errs[1]:.6e}")
    assert abs(errs[1] / errs[0] - 1.0) <= 0.01


def test_batch_of_mixed_members_equals_alone(torch_cuda):
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import Batch, GdgError, Solver

    specs = [(13, 3), (5, 4), (21, 5)]
    members = [four_quadrant_problem(N, 2, seed=s) for N, s in specs]
    alone = []
    for P, U in members:
        S = Solver(P, params=MIXED)
        S.set_clock(0.0, float("inf"), 0.5)
        Ud = _dev(torch, U)
        work = (torch.empty_like(Ud), torch.empty_like(Ud))
        for _ in range(4):
            S.step(Ud, work)
        alone.append(Ud.cpu().numpy())
    solvers, states, works = [], [], []
    for P, U in members:
        S = Solver(P, params=MIXED)
        S.set_clock(0.0, float("inf"), 0.5)
        Ud = _dev(torch, U)
        solvers.append(S)
        states.append(Ud)
        works.append((torch.empty_like(Ud), torch.empty_like(Ud)))
    B = Batch(solvers, states, works)
    for _ in range(4):
        B.step()
    for a, Ud in zip(alone, states):
        assert np.array_equal(a, Ud.cpu().numpy())
    B.close()
    P, U = members[0]
    S64 = Solver(P)
    Ua = _dev(torch, U)
    with pytest.raises(GdgError):
        Batch([solvers[0], S64], [states[0], Ua], [works[0], (torch.empty_like(Ua), torch.empty_like(Ua))])


def test_open_and_dirichlet_boundaries(torch_cuda):
    """In/outflow (a supersonic stream with subsonic sides) and exact Dirichlet data (the Q3 vortex at
    gamma = 5/3): one limited stage of the mixed path against the oracle."""
    torch = torch_cuda
    from oracle.oracle import Oracle
    from paper_2402_04514_gb300.gdg import Solver

    sides = dict(left="inoutflow", right="inoutflow", bottom="inoutflow", top="inoutflow")
    P = assembly.assemble_2d(16, 16, 1, bc=sides)
    x, y = P.x
    rho = 1.0 + 0.5 * np.exp(-40 * ((x - 0.4) ** 2 + (y - 0.5) ** 2))
    U = workloads.prim_to_cons(rho, np.stack([np.full(P.n, 3.0), np.full(P.n, 0.5)]), np.full(P.n, 1.0), 1.4)
    bd = workloads.prim_to_cons(np.full(P.nb, 1.0), np.stack([np.full(P.nb, 3.0), np.full(P.nb, 0.5)]),
                                np.full(P.nb, 1.0), 1.4)
    Pv, Uv, bdv = dirichlet_vortex_problem(6, 3)
    for P, U, bd, g in ((P, U, bd, 1.4), (Pv, Uv, bdv(0.0), 5.0 / 3.0)):
        S, O = Solver(P, gamma=g, params=MIXED), Oracle(P, gamma=g)
        tau = O.max_dt(U, 0.5, bdata=bd)
        out = S.stage(_dev(torch, U), tau, bdata=_dev(torch, bd))
        ref, flags = O.stage(U, tau, bdata=bd)
        e = rel_err(out.cpu().numpy(), ref)
        print(f"boundaries: stage rel err {e:.3e}")
        assert e <= MIXED_STAGE_TOL and S.status() == flags == 0


def test_ssprk54_step(torch_cuda):
    """One fused SSPRK(5,4) step of the mixed path against the oracle's step with the dt the device chose
    (five stages, so five times the stage tolerance)."""
    torch = torch_cuda
    from oracle.oracle import Oracle
    from paper_2402_04514_gb300.gdg import Solver

    P, U = four_quadrant_problem(13, 2, seed=0)
    S, O = Solver(P, params=MIXED), Oracle(P)
    S.set_clock(0.0, float("inf"), 0.5)
    Ud = _dev(torch, U)
    work = (torch.empty_like(Ud), torch.empty_like(Ud), torch.empty_like(Ud))
    S.step(Ud, work)
    _, dt, steps = S.clock()
    ref, flags = O.ssprk54_step(U, dt)
    e = rel_err(Ud.cpu().numpy(), ref)
    print(f"ssprk54: step rel err {e:.3e}")
    assert steps == 1 and flags == 0 and S.status() == 0 and e <= 5 * MIXED_STAGE_TOL


def test_served_mixed_request_equals_alone(torch_cuda):
    """Requests of both precisions through the serving loop: each result equals, bit for bit, the same
    request solved alone with its own precision (the two precisions never share a batch)."""
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import Server, Solver

    reqs = [(four_quadrant_problem(9, 2, seed=s), prec, 0.01) for s, prec in ((1, 1), (2, 0), (3, 1))]
    srv = Server()
    ids = [srv.submit(P, U, t_end, params=dict(precision=prec)) for (P, U), prec, t_end in reqs]
    got = [srv.wait(r, timeout=300.0) for r in ids]
    srv.close()
    for ((P, U), prec, t_end), (res, info) in zip(reqs, got):
        S = Solver(P, params=dict(precision=prec))
        S.set_clock(0.0, t_end, 0.5)
        Ud = _dev(torch, U)
        work = (torch.empty_like(Ud), torch.empty_like(Ud))
        for _ in range(100000):
            S.step(Ud, work)
            if S.clock()[0] >= t_end:
                break
        assert info["status"] == 0 and np.array_equal(res, Ud.cpu().numpy())
