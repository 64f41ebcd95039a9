"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerance: per component, max |U_gpu - U_oracle| / max |U_oracle| <= 1e-12 after one stage and <= 1e-10
after 100 SSP-RK3 steps; invariant-domain checks (rho > 0, eps > 0, local bounds) hold exactly.
Sizes span several thread blocks with a ragged tail (blocks of 256 nodes, 153-160 nodes for the element sweep
under the default schedule)."""
import numpy as np
import pytest

from paper_2402_04514_gb300 import assembly, workloads
from tests.helpers import (dirichlet_vortex_problem, four_quadrant_problem, octant_problem, periodic_vortex_problem,
                           rel_err)

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


def _pair(P, gamma=1.4, params=None):
    from oracle.oracle import Oracle
    from paper_2402_04514_gb300.gdg import Solver

    return Solver(P, gamma=gamma, params=params), Oracle(P, gamma=gamma, params=dict(params or {}))


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [
    ("sod1d_q1", lambda: (assembly.assemble_1d(200, 1), None)),
    ("sod1d_q2_ragged", lambda: (assembly.assemble_1d(333, 2), None)),
    ("vortex_q1_periodic", lambda: periodic_vortex_problem(17, 1)),
    ("fq_q2_slip", lambda: four_quadrant_problem(13, 2, seed=0)),
    ("fq_q1_slip", lambda: four_quadrant_problem(19, 1, seed=4)),
    ("fq_q3_slip", lambda: four_quadrant_problem(7, 3, seed=2)),
    ("oct_q1_3d", lambda: octant_problem((7, 6, 5), 1, seed=1)),
    ("oct_q2_3d", lambda: octant_problem((4, 3, 3), 2, seed=2)),
]


def _problem(name):
    P, U = dict(CASES)[name]()
    if U is None:
        U = workloads.sod(P.x[0])
    return P, U


@pytest.mark.parametrize("name", [c[0] for c in CASES])
@pytest.mark.parametrize("order,passes", [(0, 2), (1, 2), (2, 0), (2, 1), (2, 2)])
def test_stage_parity(torch_cuda, name, order, passes):
    torch = torch_cuda
    P, U = _problem(name)
    prm = dict(order=order, limiter_passes=passes)
    S, O = _pair(P, params=prm)
    Ud = _dev(torch, U)
    tau_g = S.max_dt(Ud, 0.5)
    tau_o = O.max_dt(U, 0.5)
    assert abs(tau_g - tau_o) <= 1e-13 * tau_o
    for alpha, base in ((0.0, None), (0.75, U * 1.01)):
        out = S.stage(Ud, tau_o, U_base=None if base is None else _dev(torch, base), alpha=alpha)
        ref, flags = O.stage(U, tau_o, U_base=base, alpha=alpha)
        torch.cuda.synchronize()
        assert rel_err(out.cpu().numpy(), ref) <= STAGE_TOL
        assert S.status() == flags == 0


@pytest.mark.parametrize("name", ["fq_q2_slip", "fq_q1_slip", "vortex_q1_periodic"])
def test_intermediates_parity(torch_cuda, name):
    """d_ij^L, N_i, U^L, the bounds, A_ij, l (both passes) and U^(1) agree with the oracle's trace."""
    torch = torch_cuda
    P, U = _problem(name)
    S, O = _pair(P)
    tau = O.max_dt(U, 0.5)
    S.stage(_dev(torch, U), tau)
    _, _, tr = O.stage(U, tau, trace=True)
    assert rel_err(S.export("dL"), tr["dL"]) <= 1e-13
    if P.nb:
        assert rel_err(S.export("dB"), tr["dB"]) <= 1e-13
    # N_i = R_i / D_i loses relative accuracy where the stencil's states differ by little more than
    # rounding; it only ever multiplies those differences (through d^H), so what is bounded is
    # |dN_i| times the largest relative state difference over the stencil of i.
    rows = np.repeat(np.arange(P.n), np.diff(P.row_ptr))
    stencil = np.abs(P.cij).sum(0) > 0
    scale = np.abs(U).max(1, keepdims=True)
    var = np.zeros(P.n)
    np.maximum.at(var, rows[stencil], (np.abs(U[:, P.col_idx[stencil]] - U[:, rows[stencil]]) / scale).max(0))
    assert (np.abs(S.export("N") - tr["N"]) * var).max() <= 1e-12
    assert rel_err(S.export("UL"), tr["UL"]) <= STAGE_TOL
    for k in ("rho_min", "rho_max", "s_min"):
        assert rel_err(S.export(k), tr[k]) <= 1e-13
    assert rel_err(S.export("A"), tr["A"]) <= 1e-11
    if name == "fq_q2_slip":
        # this stage has line searches that need the bracketed iteration (the oracle iterates on 643 of
        # its 28392): the GPU runs them from its deferred queue, and they are checked with the rest below
        assert S.export("ls_deferred").sum() > 0
    l1 = S.export("l1")
    assert np.abs(l1 - tr["l1"]).max() <= 1e-12
    rem = l1 < 1.0  # where l1 = 1 the pass-2 coefficient multiplies a zero remainder
    assert np.abs(S.export("l2")[rem] - tr["l2"][rem]).max(initial=0.0) <= 1e-12
    assert rel_err(S.export("U1"), tr["U1"]) <= STAGE_TOL


@pytest.mark.parametrize("name", ["fq_q2_slip", "fq_q3_slip", "oct_q2_3d"])
def test_stage_parity_element_measure(torch_cuda, name):
    """A limited stage with the relaxation's mesh size from the element (relax_measure = 1): the bounds
    equal the oracle's within 1e-13 and the stage within 1e-12."""
    torch = torch_cuda
    P, U = _problem(name)
    S, O = _pair(P, params=dict(relax_measure=1))
    tau = O.max_dt(U, 0.5)
    out = S.stage(_dev(torch, U), tau)
    ref, flags, tr = O.stage(U, tau, trace=True)
    for k in ("rho_min", "rho_max", "s_min"):
        assert rel_err(S.export(k), tr[k]) <= 1e-13
    assert rel_err(out.cpu().numpy(), ref) <= STAGE_TOL
    assert S.status() == flags == 0


def test_dirichlet_q3_and_bounds_off(torch_cuda):
    torch = torch_cuda
    P, U, bdata = dirichlet_vortex_problem(6, 3)
    g = 5.0 / 3.0
    for prm in (dict(), dict(bounds_mode=1)):
        S, O = _pair(P, gamma=g, params=prm)
        bd = bdata(0.0)
        tau = O.max_dt(U, 0.5, bdata=bd)
        assert abs(S.max_dt(_dev(torch, U), 0.5, bdata=_dev(torch, bd)) - tau) <= 1e-13 * tau
        out = S.stage(_dev(torch, U), tau, bdata=_dev(torch, bd))
        ref, _ = O.stage(U, tau, bdata=bd)
        assert rel_err(out.cpu().numpy(), ref) <= STAGE_TOL


@pytest.mark.parametrize("name", ["sod1d_q1", "fq_q1_slip"])
def test_hundred_steps(torch_cuda, name):
    """100 SSP-RK3 steps of the limited scheme (tau from max_dt each step): <= 1e-10."""
    torch = torch_cuda
    P, U = _problem(name)
    if name == "fq_q1_slip":
        P, U = four_quadrant_problem(8, 1, seed=4)
    S, O = _pair(P)
    Ud = _dev(torch, U)
    bufs = (torch.empty_like(Ud), torch.empty_like(Ud))
    out = torch.empty_like(Ud)
    Uo = U.copy()
    for _ in range(100):
        tau = O.max_dt(Uo, 0.5)
        Uo, flags = O.ssprk3_step(Uo, tau)
        S.ssprk3_step(Ud, tau, bufs, out)
        Ud, out = out, Ud
    got = Ud.cpu().numpy()
    assert rel_err(got, Uo) <= LONG_TOL
    rho = got[0]
    eps = got[-1] - 0.5 * (got[1:-1] ** 2).sum(0) / rho
    assert (rho > 0).all() and (eps > 0).all()
    assert S.status() == 0


def test_edge_cases(torch_cuda):
    """One element; an empty mesh; a stage with tau = 0 (identity); a CFL violation is flagged."""
    torch = torch_cuda
    P = assembly.assemble_2d(1, 1, 2)
    U = workloads.four_quadrant(P.x[0], P.x[1], seed=1)
    S, O = _pair(P, params=dict(c_r=0.5))  # one element: h_i is O(1), c_r = 4 would make r_h^- < 0
    tau = O.max_dt(U, 0.5)
    out = S.stage(_dev(torch, U), tau)
    ref, _ = O.stage(U, tau)
    assert rel_err(out.cpu().numpy(), ref) <= STAGE_TOL
    out0 = S.stage(_dev(torch, U), 0.0)
    assert rel_err(out0.cpu().numpy(), U) <= 1e-15
    S.stage(_dev(torch, U), 3.0 * tau / 0.5)
    assert S.status(clear=True) & 2
    assert S.status() == 0
    from paper_2402_04514_gb300.assembly import Problem
    Pe = Problem(dim=2, degree=1, n=0, n_loc=4, row_ptr=np.zeros(1, np.int64), col_idx=np.zeros(0, np.int32),
                 cij=np.zeros((2, 0)), coloc=np.zeros(0, np.uint8), mi=np.zeros(0), MK=np.zeros((0, 4, 4)),
                 b_node=np.zeros(0, np.int32), b_c=np.zeros((2, 0)), b_type=np.zeros(0, np.int32),
                 b_part=np.zeros(0, np.int32), omega_measure=1.0, x=np.zeros((2, 0)))
    from paper_2402_04514_gb300.gdg import Solver
    Se = Solver(Pe)
    Ue = torch.zeros((4, 0), dtype=torch.float64, device="cuda")
    assert Se.max_dt(Ue, 0.5) == float("inf")
    Se.stage(Ue, 0.1)


def test_inadmissible_input_is_flagged(torch_cuda):
    torch = torch_cuda
    P, U = four_quadrant_problem(4, 1)
    U = U.copy()
    U[3, 7] = 0.5 * (U[1, 7] ** 2 + U[2, 7] ** 2) / U[0, 7] - 1e-3  # eps < 0
    S, _ = _pair(P)
    S.stage(_dev(torch, U), 1e-4)
    assert S.status() & 1


def _patch_problem(nx_full, k, ex0, ex1, ey0, ey1):
    h = 1.0 / nx_full
    return assembly.assemble_2d(ex1 - ex0, ey1 - ey0, k, box=(ex0 * h, ex1 * h, ey0 * h, ey1 * h))


def test_full_size_bench_configuration_sampled(torch_cuda):
    """The bench workload (Q2 on 1024^2 quads of [0,1]^2, 9.4M nodes, four-quadrant data, slip walls), one
    stage at full size in the bench's launch configuration.  Sampled elements are checked against the
    oracle run on a 15 x 15-element patch around each of them (the stage's dependency radius is below 6
    elements; interior c_ij, m_i, M_K and |Omega| are those of the full mesh); conservation of rho and E
    and the local bounds are checked everywhere."""
    torch = torch_cuda
    from oracle.oracle import Oracle
    from paper_2402_04514_gb300.gdg import Solver

    N, k = 1024, 2
    P = assembly.assemble_2d(N, N, k)
    U = workloads.four_quadrant(P.x[0], P.x[1], seed=0)
    S = Solver(P)
    Ud = _dev(torch, U)
    tau = S.max_dt(Ud, 0.5)
    out = S.stage(Ud, tau).cpu().numpy()
    assert S.status() == 0
    tot0, tot1 = (P.mi * U).sum(1), (P.mi * out).sum(1)
    for c in (0, 3):
        assert abs(tot1[c] - tot0[c]) <= 1e-12 * abs(tot0[c])
    rmin, rmax, smin = S.export("rho_min"), S.export("rho_max"), S.export("s_min")
    rho = out[0]
    st = rho ** (-1.4) * (out[3] - 0.5 * (out[1] ** 2 + out[2] ** 2) / rho)
    assert (rho >= rmin * (1 - 1e-13)).all() and (rho <= rmax * (1 + 1e-13)).all()
    assert (st >= smin * (1 - 1e-12)).all()
    rng = np.random.default_rng(7)
    samples = [(512, 512), (511, 511), (0, 0), (1023, 1023), (0, 700), (300, 1023)]
    samples += [tuple(rng.integers(0, N, 2)) for _ in range(4)]
    R = 7
    nl = (k + 1) ** 2
    for ex, ey in samples:
        ex0, ex1 = max(0, ex - R), min(N, ex + R + 1)
        ey0, ey1 = max(0, ey - R), min(N, ey + R + 1)
        Pp = _patch_problem(N, k, ex0, ex1, ey0, ey1)
        Pp.omega_measure = P.omega_measure
        Up = workloads.four_quadrant(Pp.x[0], Pp.x[1], seed=0)
        O = Oracle(Pp)
        ref, _ = O.stage(Up, tau)
        le = (ey - ey0) * (ex1 - ex0) + (ex - ex0)
        ge = ey * N + ex
        got = out[:, ge * nl:(ge + 1) * nl]
        want = ref[:, le * nl:(le + 1) * nl]
        scale = np.abs(U).max(1, keepdims=True)
        assert (np.abs(got - want) <= STAGE_TOL * scale).all(), (ex, ey)


def test_full_size_developed_state_sampled(torch_cuda):
    """The bench workload after 40 fused SSP-RK3 steps on the autotuned schedule (as bench.py runs it):
    the waves from the quadrant interfaces are several elements wide and the limiter is active there.  One
    more stage at full size; elements sampled on and next to the interfaces, and at random, are checked
    against the oracle on a 15 x 15-element patch of the GPU's own state around each of them (a dG node
    belongs to one element, so the patch state is the full state's element blocks)."""
    torch = torch_cuda
    from oracle.oracle import Oracle
    from paper_2402_04514_gb300.gdg import Solver

    N, k = 1024, 2
    nl = (k + 1) ** 2
    P = assembly.assemble_2d(N, N, k)
    Ud = _dev(torch, workloads.four_quadrant(P.x[0], P.x[1], seed=0))
    S = Solver(P)
    S.set_clock(0.0, float("inf"), 0.5)
    work = (torch.empty_like(Ud), torch.empty_like(Ud))
    for _ in range(3):
        S.step(Ud, work)
    S.autotune(Ud, work, trials=1)
    for _ in range(37):
        S.step(Ud, work)
    assert S.status() == 0
    U = Ud.cpu().numpy()
    tau = S.max_dt(Ud, 0.5)
    out = S.stage(Ud, tau).cpu().numpy()
    assert S.status() == 0
    l1 = S.export("l1")
    assert (l1 < 1.0).mean() > 1e-3  # the limiter is active
    tot0, tot1 = (P.mi * U).sum(1), (P.mi * out).sum(1)
    for c in (0, 3):
        assert abs(tot1[c] - tot0[c]) <= 1e-12 * abs(tot0[c])
    rng = np.random.default_rng(11)
    samples = [(512, 512), (511, 512), (513, 509), (510, 300), (514, 800), (200, 511), (850, 514), (509, 20)]
    samples += [tuple(rng.integers(0, N, 2)) for _ in range(3)]
    R = 7
    Ue = U.reshape(4, N * N, nl)
    limited = 0
    for ex, ey in samples:
        ex0, ex1 = max(0, ex - R), min(N, ex + R + 1)
        ey0, ey1 = max(0, ey - R), min(N, ey + R + 1)
        Pp = _patch_problem(N, k, ex0, ex1, ey0, ey1)
        Pp.omega_measure = P.omega_measure
        elems = (np.arange(ey0, ey1)[:, None] * N + np.arange(ex0, ex1)[None, :]).ravel()
        Up = np.ascontiguousarray(Ue[:, elems, :].reshape(4, -1))
        ref, _, tr = Oracle(Pp).stage(Up, tau, trace=True)
        le = (ey - ey0) * (ex1 - ex0) + (ex - ex0)
        ge = ey * N + ex
        got = out[:, ge * nl:(ge + 1) * nl]
        want = ref[:, le * nl:(le + 1) * nl]
        scale = np.abs(U).max(1, keepdims=True)
        assert (np.abs(got - want) <= STAGE_TOL * scale).all(), (ex, ey)
        rows = np.repeat(np.arange(Pp.n), np.diff(Pp.row_ptr))
        limited += int((tr["l1"][(rows // nl) == le] < 1.0).any())
    assert limited >= 3  # some samples sit where the limiter acts


@pytest.mark.parametrize("q", [1, 3, 5, 7, 12])
def test_fp64_helpers_against_cuda(torch_cuda, q):
    """The Newton-Raphson reciprocal and inverse root used in the sweep: the reciprocal is within 2 ulp
    of CUDA's 1.0 / x; the root is within 2 ulp of x^{-1/q} computed in extended precision (numpy's
    long double), as accurate as CUDA's pow(x, -1.0/q), whose rounded exponent costs it up to a few ulp
    when |log x| is large."""
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import math_selftest

    rng = np.random.default_rng(q)
    x = np.concatenate([np.exp(rng.uniform(np.log(1e-12), np.log(1e12), 200000)), [1.0, 2.0, 0.5, 3.0]])
    xd = torch.from_numpy(x).cuda()
    mine_r, ref_r = math_selftest(0, q, xd).cpu().numpy(), math_selftest(2, q, xd).cpu().numpy()
    mine_q, cuda_q = math_selftest(1, q, xd).cpu().numpy(), math_selftest(3, q, xd).cpu().numpy()
    assert (np.abs(mine_r - ref_r) <= 2 * np.spacing(np.abs(ref_r))).all()
    xl = x.astype(np.longdouble)
    exact = np.power(xl, -np.longdouble(1) / np.longdouble(q))
    ulp = np.spacing(np.abs(exact.astype(np.float64)))
    err_mine = np.abs(mine_q.astype(np.longdouble) - exact).astype(np.float64) / ulp
    err_cuda = np.abs(cuda_q.astype(np.longdouble) - exact).astype(np.float64) / ulp
    if np.finfo(np.longdouble).eps < 1e-18:  # a long double wider than double
        assert err_mine.max() <= max(2.0, err_cuda.max())
    else:
        assert (np.abs(mine_q - cuda_q) <= 8 * np.spacing(np.abs(cuda_q))).all()


def test_square_root_against_cuda(torch_cuda):
    """The square root of the wave-speed bound and the sound speed (two Heron corrections from the FP32
    reciprocal square root) is within 1 ulp of CUDA's correctly rounded sqrt over the FP32 normal range,
    and takes sqrt itself outside it."""
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import math_selftest

    rng = np.random.default_rng(9)
    x = np.concatenate([np.exp(rng.uniform(np.log(1e-30), np.log(1e30), 400000)),
                        1.0 + rng.uniform(0, 1e-6, 10000), [1.0, 2.0, 4.0, 0.25, 1e-300, 1e300, 0.0]])
    xd = torch.from_numpy(x).cuda()
    mine, ref = math_selftest(5, 1, xd).cpu().numpy(), math_selftest(6, 1, xd).cpu().numpy()
    assert (np.abs(mine - ref) <= np.spacing(ref)).all()
    assert mine[-3:].tolist() == ref[-3:].tolist()


def _binary64_pairs(rng, n):
    """Operand pairs for the integer-pipe product and sum: any bit patterns, magnitudes near 1, opposite
    signs with close exponents (cancellation), significands with trailing zeros (exact results and ties),
    exponents near both ends of the range, and zeros, infinities, NaN and subnormals."""
    bits = rng.integers(0, 2**63, (8, n), dtype=np.int64).astype(np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, (8, n)).astype(np.uint64)
    frac, sign = bits & np.uint64(0xFFFFFFFFFFFFF), bits >> np.uint64(63)

    def make(s, field, f):
        return ((s << np.uint64(63)) | (field.astype(np.uint64) << np.uint64(52)) | f).view(np.float64)

    fields = [rng.integers(1000, 1047, n), rng.integers(1, 2047, n), rng.integers(1, 40, n),
              rng.integers(2007, 2047, n)]
    a = [bits[0].view(np.float64), make(sign[1], fields[0], frac[1]), make(sign[2], fields[1], frac[2])]
    b = [bits[1].view(np.float64), make(sign[3], fields[0], frac[3]), -a[2] * (1 + np.ldexp(1.0, -rng.integers(1, 60, n)))]
    shift = rng.integers(0, 32, n).astype(np.uint64)
    a.append(make(sign[4], fields[1], (frac[4] >> shift) << shift))
    b.append(make(sign[5], fields[1], (frac[5] >> shift) << shift))
    a.append(make(sign[6], np.where(fields[2] % 2 == 0, fields[2], fields[3]), frac[6]))
    b.append(make(sign[7], np.where(fields[2] % 3 == 0, fields[2], fields[3]), frac[7]))
    special = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, 5e-324, -2.5e-320, 2.2250738585072014e-308,
                        1.7976931348623157e308, 0.5])
    a.append(np.where(rng.random(n) < 0.5, special[rng.integers(0, 12, n)], a[1]))
    b.append(special[rng.integers(0, 12, n)])
    ia, ib = rng.integers(1, 2**27, n) | 1, rng.integers(1, 2**28, n) | 1
    a.append(np.ldexp(ia.astype(np.float64), rng.integers(-100, 100, n)))
    b.append(np.ldexp(ib.astype(np.float64), rng.integers(-100, 100, n)) * rng.choice([-1.0, 1.0], n))
    A, B = np.concatenate(a), np.concatenate(b)
    return np.stack([A, B], axis=1).reshape(-1)


def test_integer_binary64_against_cuda(torch_cuda):
    """The integer-pipe product and sum of the sweep kernels give the FP64 instructions' results bit for bit
    (any NaN for any NaN) over 1.4 million operand pairs, and agree with numpy's binary64 arithmetic; the
    scaling by 2^k agrees with the product by 2^k."""
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import math_selftest

    x = _binary64_pairs(np.random.default_rng(11), 200000)
    xd = torch.from_numpy(x).cuda()
    a, b = x[0::2], x[1::2]
    with np.errstate(all="ignore"):
        host = {7: a * b, 9: a + b}
    for soft, hw in ((7, 8), (9, 10)):
        mine, ref = math_selftest(soft, 1, xd).cpu().numpy(), math_selftest(hw, 1, xd).cpu().numpy()
        nan = np.isnan(ref)
        assert (np.isnan(mine) == nan).all()
        assert (mine[~nan].view(np.uint64) == ref[~nan].view(np.uint64)).all()
        assert (ref[~nan].view(np.uint64) == host[soft][~nan].view(np.uint64)).all()
    # x 2^k by the exponent field against numpy's ldexp (the same rounding as the product by 2^k)
    rng = np.random.default_rng(12)
    k = np.clip(rng.integers(-60, 61, a.size) + np.where(rng.random(a.size) < 0.1, rng.integers(-1022, 1023, a.size), 0),
                -1022, 1023)
    xk = np.stack([a, k.astype(np.float64)], axis=1).reshape(-1)
    mine = math_selftest(11, 1, torch.from_numpy(xk).cuda()).cpu().numpy()
    with np.errstate(all="ignore"):
        ref = a * np.ldexp(1.0, k)
    nan = np.isnan(ref)
    assert (np.isnan(mine) == nan).all()
    assert (mine[~nan].view(np.uint64) == ref[~nan].view(np.uint64)).all()


def test_integer_float_conversions(torch_cuda):
    """The FP64 -> FP32 -> FP64 conversions of the FP32 certificates, done with integer operations only:
    truncation to 23 significand bits in the FP32 normal range, signed zeros kept, NaN for everything
    outside that range (subnormal in FP32, overflow, inf, NaN), so that a certificate fails instead of
    using an inexact value."""
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import math_selftest

    rng = np.random.default_rng(7)
    mags = np.exp(rng.uniform(np.log(1e-45), np.log(1e45), 100000))
    x = np.concatenate([mags * rng.choice([-1.0, 1.0], mags.size),
                        [0.0, -0.0, np.inf, -np.inf, np.nan, 2.0 ** -126, -(2.0 ** -126), 2.0 ** -127,
                         np.nextafter(2.0 ** 128, 0), 2.0 ** 128, 1.0, -3.0, 5e-324]])
    got = math_selftest(4, 1, torch.from_numpy(x).cuda()).cpu().numpy()
    bits = x.view(np.uint64)
    trunc = (bits & ~np.uint64((1 << 29) - 1)).view(np.float64)
    normal = (np.abs(x) >= 2.0 ** -126) & (np.abs(x) < 2.0 ** 128)
    zero = x == 0.0
    assert (got[normal] == trunc[normal]).all()
    assert (got[zero] == 0.0).all() and (np.signbit(got[zero]) == np.signbit(x[zero])).all()
    assert np.isnan(got[~normal & ~zero]).all()
