"""The high-order scheme of Sec. 5 on the isentropic vortex of Sec. 6.2, test case (i), in the oracle (no
GPU): at 2304 DoFs (Q2 on 16^2 and Q3 on 12^2 elements; gamma = 5/3, exact Dirichlet data at every stage
time, SSPRK(5,4) at Cr = 0.5, t_F = 2) its L1 error equals the one Appendix A, Table ErrorIsentropicConvex
prints within 12% (Q2) and 2% (Q3).  This pins the entropy-viscosity indicator with c_ev = 1/2 and 1/4
(Sec. 5.2), the minimal viscosity of eq. (ViscMin) with p_k = 1/2 and 0 (Sec. 5.1), the consistent-mass
element solve of eq. (HighScheme) and the time stepping together: a wrong constant or a dropped term moves
the Q3 error by far more than 2%.  (The table is for the limited scheme; on this smooth test the paper's
limiter leaves the high-order result in place.  With the relaxation's mesh size of eq. (ViscMinConst2)'s
passage as printed, h_i from the node's lumped mass, the limiter here still acts in the vortex core; with
h_i from the measure of the node's element it does not, and the limited error matches the table too.)
The oracle runs its multi-core build (bit-identical to the pinned single-thread one)."""
import numpy as np
import pytest

from paper_2402_04514_gb300 import workloads
from tests.helpers import consolidated_l1, dirichlet_vortex_problem, load_vortex_tables

GAMMA = 5.0 / 3.0


def _error(oracle_mod, ne, k, **params):
    from oracle import ssprk

    P, U, bdata = dirichlet_vortex_problem(ne, k)
    O = oracle_mod.Oracle(P, gamma=GAMMA, params=params, openmp=True)
    C = ssprk.ssp_coefficient(ssprk.SSPRK54_ALPHA, ssprk.SSPRK54_BETA)
    t, tF = 0.0, 2.0
    while t < tF - 1e-12:
        dt = min(0.5 * C * O.max_dt(U, 1.0, bdata=bdata(t)), tF - t)
        U, flags = O.ssprk54_step(U, dt, bdata, t)
        assert flags == 0
        t += dt
    return consolidated_l1(P, U, workloads.vortex(P.x[0], P.x[1], tF, gamma=GAMMA))


@pytest.mark.parametrize("k,ne,tol", [(2, 16, 0.12), (3, 12, 0.02)])
def test_high_order_vortex_error_matches_the_table(oracle_mod, k, ne, tol):
    want = load_vortex_tables()["limited"][k][0]
    got = _error(oracle_mod, ne, k, order=oracle_mod.HIGH)
    assert abs(got / want - 1.0) <= tol, (k, got, want)


def test_limited_q3_vortex_error_with_the_element_measure(oracle_mod):
    """The limited scheme with the relaxation's mesh size taken from the element (relax_measure = 1,
    h_i = (|K_i| / |Omega|)^{1/d}): its Q3 error at 2304 DoFs equals the table's within 2% (with h_i from
    the node's lumped mass as printed the limited Q3 error is 1.9 times the table's: the limiter then acts in
    the vortex core, and the paper's results show it did not).  The GPU tests take Q2 and finer meshes."""
    want = load_vortex_tables()["limited"][3][0]
    got = _error(oracle_mod, 12, 3, relax_measure=1)
    assert abs(got / want - 1.0) <= 0.02, (got, want)
