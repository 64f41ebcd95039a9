"""Pins of the oracle's Runge-Kutta steps (oracle/ssprk.py) against what fixes them independently of the
code: the order conditions of the Butcher tableau derived from the Shu-Osher coefficients, the SSP
coefficient, the stability polynomial on y' = lambda y, fourth-order convergence in time on the Euler
operator, and the paper's vortex table with its own integrator (SSPRK(5,4), Sec. 6.2)."""
import math

import numpy as np
import pytest

from oracle import ssprk
from paper_2402_04514_gb300 import workloads
from tests.helpers import consolidated_l1, dirichlet_vortex_problem

METHODS = {"ssprk3": (ssprk.SSPRK3_ALPHA, ssprk.SSPRK3_BETA, 3), "ssprk54": (ssprk.SSPRK54_ALPHA, ssprk.SSPRK54_BETA, 4)}


def _order_residuals(A, b, c, order):
    """Residuals of the order conditions of an explicit Runge-Kutta method up to `order` (Butcher)."""
    r = [b.sum() - 1.0, b @ c - 0.5]
    if order >= 3:
        r += [b @ c ** 2 - 1.0 / 3.0, b @ (A @ c) - 1.0 / 6.0]
    if order >= 4:
        r += [b @ c ** 3 - 0.25, b @ (c * (A @ c)) - 1.0 / 8.0, b @ (A @ c ** 2) - 1.0 / 12.0,
              b @ (A @ (A @ c)) - 1.0 / 24.0]
    return np.abs(np.array(r))


@pytest.mark.parametrize("name", sorted(METHODS))
def test_order_conditions_and_convexity(name):
    alpha, beta, order = METHODS[name]
    for row in alpha:
        assert abs(sum(row) - 1.0) <= 2e-15 and min(row) >= 0.0
    assert min(min(r) for r in beta) >= 0.0
    A, b, c = ssprk.butcher(alpha, beta)
    assert _order_residuals(A, b, c, order).max() <= 1e-14
    # and the next order fails (these are not higher-order methods)
    if order == 3:
        assert _order_residuals(A, b, c, 4).max() > 1e-3


def test_ssp_coefficients():
    assert ssprk.ssp_coefficient(ssprk.SSPRK3_ALPHA, ssprk.SSPRK3_BETA) == 1.0
    C = ssprk.ssp_coefficient(ssprk.SSPRK54_ALPHA, ssprk.SSPRK54_BETA)
    assert abs(C - 1.508180049) < 1e-8  # the optimal value of the five-stage fourth-order family


def _caught(alpha, beta):
    """The pins above reject the table: a row of alpha off one, or an order condition off."""
    if max(abs(sum(r) - 1.0) for r in alpha) > 1e-9:
        return True
    A, b, c = ssprk.butcher(alpha, beta)
    return _order_residuals(A, b, c, 4).max() > 1e-9


def test_any_mistyped_coefficient_is_caught():
    """Perturbing any one nonzero coefficient of either table by 1e-7 is rejected by the row sums or the
    order conditions, so the pins fix every printed digit down to that size."""
    for i in range(5):
        for j in range(i + 1):
            for table in ("alpha", "beta"):
                alpha = [list(r) for r in ssprk.SSPRK54_ALPHA]
                beta = [list(r) for r in ssprk.SSPRK54_BETA]
                t = alpha if table == "alpha" else beta
                if t[i][j] == 0.0:
                    continue
                t[i][j] += 1e-7
                assert _caught(alpha, beta), (table, i, j)
    assert not _caught(ssprk.SSPRK54_ALPHA, ssprk.SSPRK54_BETA)


@pytest.mark.parametrize("name", sorted(METHODS))
def test_stability_polynomial(name):
    """On y' = lambda y the step is a polynomial R(z); R(z) - e^z = O(z^(p+1)), checked by the ratio of
    the errors at z and z/2 (2^(p+1) for small z), through the same combinator the Euler steps use."""
    alpha, beta, p = METHODS[name]
    lam = -1.3 + 0.4j

    def step(dt):
        y, _ = ssprk.shu_osher_step(np.array([1.0 + 0.0j]), dt, lambda u, tau, t: (u + tau * lam * u, 0),
                                    alpha, beta)
        return y[0]

    errs = [abs(step(h) - np.exp(lam * h)) for h in (0.02, 0.01)]
    assert abs(math.log2(errs[0] / errs[1]) - (p + 1)) < 0.1


def test_fourth_order_in_time_on_the_euler_operator():
    """The high-order scheme without the entropy-viscosity switch (c_ev = 0: the minimal viscosity of
    Sec. 5.1 only, a smooth operator here) on the vortex, on a fixed Q2 mesh: halving dt divides the
    SSPRK(5,4) error (against dt/32) by about 16.  (With the switch, d^H = max(d^min, d^ev) is not smooth
    in U and the temporal rate is erratic.)"""
    from oracle.oracle import HIGH, Oracle

    P, U0, bdata = dirichlet_vortex_problem(6, 2)
    O = Oracle(P, gamma=5.0 / 3.0, params=dict(order=HIGH, c_ev=0.0))
    dt0 = 0.8 * ssprk.ssp_coefficient(ssprk.SSPRK54_ALPHA, ssprk.SSPRK54_BETA) * O.max_dt(U0, 1.0, bdata=bdata(0.0))
    tF = 4 * dt0

    def run(dt):
        U, t = U0.copy(), 0.0
        while t < tF - 1e-14:
            h = min(dt, tF - t)
            U, f = O.ssprk54_step(U, h, bdata, t)
            assert f == 0
            t += h
        return U

    dts = (dt0, dt0 / 2, dt0 / 4)
    ref = run(dt0 / 32)
    e = [np.abs(run(dt) - ref).max() for dt in dts]
    rates = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(rates) > 3.7, rates


def test_vortex_with_the_papers_integrator_against_its_table():
    """Sec. 6.2, test case (i) at 2304 DoFs (gamma = 5/3, exact Dirichlet data, t_F = 2) with SSPRK(5,4)
    at Cr = 0.5 per forward-Euler stage (dt = 0.5 C dt_FE): the limited Q1 and Q2 L1 errors against
    Appendix A, Table ErrorIsentropicConvex (golden file).  Q1 within 20%, Q2 within 6%."""
    from oracle.oracle import Oracle
    from tests.helpers import load_vortex_tables

    tab = load_vortex_tables()
    C = ssprk.ssp_coefficient(ssprk.SSPRK54_ALPHA, ssprk.SSPRK54_BETA)
    g = 5.0 / 3.0
    for ne, k, tol in ((24, 1, 0.2), (16, 2, 0.06)):
        P, U, bdata = dirichlet_vortex_problem(ne, k, gamma=g)
        O = Oracle(P, gamma=g, openmp=True)  # the multi-core build: bit-identical to the pinned one
        t, tF = 0.0, 2.0
        while t < tF - 1e-12:
            dt = min(0.5 * C * O.max_dt(U, 1.0, bdata=bdata(t)), tF - t)
            U, f = O.ssprk54_step(U, dt, bdata, t)
            assert f == 0
            t += dt
        e = consolidated_l1(P, U, workloads.vortex(P.x[0], P.x[1], tF, gamma=g))
        assert abs(e / tab["limited"][k][0] - 1.0) < tol, (k, e)
