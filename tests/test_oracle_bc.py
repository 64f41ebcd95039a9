"""Pins of the oracle's in- and outflow boundary condition (Sec. 4.1, eqs. (eq:supersonic_inoutflow) and
(eq:characteristics)) against what fixes it: the supersonic cases take the data or the interior state
exactly; in the subsonic case the characteristic variables of the boundary state (computed here from their
definition) are the data's on incoming and the interior state's on outgoing characteristics; a uniform
flow with matching data is preserved; a shock leaves the domain without the reflection a wall makes."""
import numpy as np
import pytest

from paper_2402_04514_gb300 import assembly, workloads
from tests import riemann_exact

G = 1.4


def _prim(U):
    rho = U[0]
    v = U[1:-1] / rho
    p = (G - 1.0) * (U[-1] - 0.5 * rho * (v * v).sum())
    return rho, v, p


def _chars(U, n):
    """R = {v_n - 2a/(g-1), p/rho^g, v - (v.n) n, v_n + 2a/(g-1)} of Sec. 4.1, eq. (eq:characteristics)."""
    rho, v, p = _prim(U)
    a = np.sqrt(G * p / rho)
    vn = v @ n
    return vn - 2 * a / (G - 1), p / rho ** G, v - vn * n, vn + 2 * a / (G - 1), vn, a


def _state(rng, speed):
    rho, p = np.exp(rng.uniform(np.log(0.2), np.log(5.0), 2))
    ang = rng.uniform(0, 2 * np.pi)
    v = speed * np.array([np.cos(ang), np.sin(ang)])
    return workloads.prim_to_cons(np.array([rho]), v.reshape(2, 1), np.array([p]), G)[:, 0]


def test_supersonic_cases_take_data_or_interior_exactly():
    from oracle.oracle import inoutflow_state

    rng = np.random.default_rng(1)
    n = np.array([0.6, 0.8])
    hits = {"in": 0, "out": 0}
    for _ in range(400):
        Ui, Ud = _state(rng, rng.uniform(0, 8)), _state(rng, rng.uniform(0, 8))
        *_, vn, a = _chars(Ui, n)
        UB = inoutflow_state(Ui, Ud, n, G)
        if vn < -a:
            assert np.array_equal(UB, Ud)
            hits["in"] += 1
        elif vn >= a:
            assert np.array_equal(UB, Ui)
            hits["out"] += 1
    assert hits["in"] > 20 and hits["out"] > 20


def test_subsonic_characteristics_come_from_the_right_side():
    from oracle.oracle import inoutflow_state

    rng = np.random.default_rng(2)
    n = np.array([-0.8, 0.6])
    checked = 0
    for _ in range(400):
        Ui, Ud = _state(rng, rng.uniform(0, 1.0)), _state(rng, rng.uniform(0, 1.0))
        Ri, Rd = _chars(Ui, n), _chars(Ud, n)
        if not (-Ri[5] <= Ri[4] < Ri[5]):
            continue
        UB = inoutflow_state(Ui, Ud, n, G)
        rho, _, p = _prim(UB)
        if not (Ri[3] > Rd[0]):  # the blend has no admissible state: the interior state is used
            assert np.array_equal(UB, Ui)
            continue
        assert rho > 0 and p > 0
        RB = _chars(UB, n)
        src = Rd if Ri[4] <= 0 else Ri  # v_n <= 0 at the interior state: the middle waves come in
        assert abs(RB[0] - Rd[0]) <= 1e-12 * (abs(Rd[0]) + Rd[5])
        assert abs(RB[3] - Ri[3]) <= 1e-12 * (abs(Ri[3]) + Ri[5])
        assert abs(RB[1] / src[1] - 1) <= 1e-12
        assert np.abs(RB[2] - src[2]).max() <= 1e-12 * (1 + np.abs(src[2]).max())
        checked += 1
    assert checked > 100


def test_uniform_flow_with_matching_data_is_preserved():
    """Subsonic uniform flow on a Q1 mesh with in/outflow on every side and the flow as data: after 20
    SSPRK3 steps the state is unchanged to roundoff."""
    from oracle.oracle import Oracle

    sides = dict(left="inoutflow", right="inoutflow", bottom="inoutflow", top="inoutflow")
    P = assembly.assemble_2d(6, 6, 1, bc=sides)
    U0 = workloads.prim_to_cons(np.full(P.n, 1.0), np.stack([np.full(P.n, 0.3), np.full(P.n, -0.2)]),
                                np.full(P.n, 1.0), G)
    bd = U0[:, P.b_node]
    O = Oracle(P)
    U = U0.copy()
    for _ in range(20):
        U, f = O.ssprk3_step(U, O.max_dt(U, 0.5, bdata=bd), lambda t: bd)
        assert f == 0
    assert np.abs(U - U0).max() <= 1e-13


@pytest.mark.parametrize("order", [0, 2])
def test_shock_leaves_the_domain_without_reflection(order):
    """Sod's shock tube on [0,1] to t = 0.35: the shock has left through x = 1 (it reaches it at t = 0.286)
    and the rarefaction has not yet reached x = 0 (t = 0.42).  Reference: the same scheme on [-1, 2] with
    the same cells, where no wave reaches a boundary by then.  On [0,1] the L1 error of rho against the
    exact Riemann solution is within 15% of the reference's with in/outflow data (the initial states),
    and at least twice it with walls (the reflected shock)."""
    from oracle.oracle import Oracle

    errs = {}
    for name, bc, x0, x1, cells in (("inoutflow", "inoutflow", 0.0, 1.0, 200), ("slip", "slip", 0.0, 1.0, 200),
                                    ("reference", "slip", -1.0, 2.0, 600)):
        P = assembly.assemble_1d(cells, 1, x0=x0, x1=x1, bc=(bc, bc))
        x = P.x[0]
        U = workloads.sod(x)
        bd = workloads.sod(P.b_x[0]) if bc == "inoutflow" else None
        O = Oracle(P, params=dict(order=order))
        t = 0.0
        while t < 0.35 - 1e-14:
            tau = min(O.max_dt(U, 0.5, bdata=bd), 0.35 - t)
            U, f = O.ssprk3_step(U, tau, None if bd is None else (lambda s: bd))
            assert not (f & 1)
            t += tau
        rho_e, _, _ = riemann_exact.sample((x - 0.5) / 0.35, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, G)
        inside = (x >= 0.0) & (x <= 1.0)
        errs[name] = float((P.mi * np.abs(U[0] - rho_e))[inside].sum())
    assert errs["inoutflow"] <= 1.15 * errs["reference"], errs
    assert errs["slip"] >= 2.0 * errs["reference"], errs


def test_supersonic_stream_conditioning():
    """The nearly uniform supersonic stream of the in/outflow GPU tests is ill-conditioned: over its first
    20 SSP-RK3 steps the oracle's own step moves by more than the 3e-12 of three stages when its input
    changes by one ulp (random signs, three draws per step), because the entropy-viscosity ratio
    N = R/D of Sec. 5.2 divides quantities near their rounding level there (6.6e-12 seen).  The GPU tests
    hold that case to a per-step bound of 3e-11, at least three times the largest such move."""
    from oracle.oracle import Oracle
    from tests.helpers import inoutflow_case, rel_err

    P, U, bd = inoutflow_case("supersonic_stream")
    O = Oracle(P)
    rng = np.random.default_rng(0)
    Uo = np.ascontiguousarray(U).copy()
    floor = 0.0
    for _ in range(20):
        tau = O.max_dt(Uo, 0.5, bdata=bd)
        one, f = O.ssprk3_step(Uo, tau, lambda t: bd)
        assert f == 0
        for _ in range(3):
            pert = Uo * (1.0 + rng.choice([-1.0, 1.0], Uo.shape) * 2.0 ** -52)
            floor = max(floor, rel_err(O.ssprk3_step(pert, tau, lambda t: bd)[0], one))
        Uo = one
    assert 3e-12 < floor < 1e-11
