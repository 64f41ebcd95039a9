"""The boundary-condition validation of Sec. 6.4 (subsec. BCvalidation) on the oracle (no GPU): the
modified isentropic vortex advected out through the top right corner with the four ways of giving the
boundary its data (tests/bc_validation.py).  The paper's Table ErrorBoundaryConditions fixes two
properties that a plausible mistake in the in/outflow construction of Sec. 4.1 breaks:
  - with supersonic flow through every side (M = 2) the far-field data (c) give the same solution as the
    exact data (b): the in/outflow state takes the data only where the flow enters, and at the inflow
    sides the exact solution differs from the far field only by the vortex's exponentially small tail
    (the table prints equal errors, 2.41e-3 at 2304 DoFs);
  - with a subsonic outflow (M = 1) the far-field data do not converge (rate 0.35 from 2304 to 9216
    DoFs): the incoming characteristic of the subsonic outflow takes the far field where the vortex is.
The oracle runs in its multi-core build (bit-identical to the pinned single-thread build)."""
import math

from tests import bc_validation as bv


def test_supersonic_far_field_data_equal_exact_data(oracle_mod):
    e_b = bv.run_oracle(24, "b", 2.0)
    e_c = bv.run_oracle(24, "c", 2.0)
    assert abs(e_c / e_b - 1.0) < 0.01, (e_b, e_c)
    assert bv.PAPER["c"][2.0][0] == bv.PAPER["b"][2.0][0]


def test_far_field_data_do_not_converge_with_a_subsonic_outflow(oracle_mod):
    e24 = bv.run_oracle(24, "c", 1.0)
    e48 = bv.run_oracle(48, "c", 1.0)
    rate = math.log2(e24 / e48)
    assert rate < 0.8, (e24, e48, rate)
    assert bv.PAPER["c"][1.0][2] < 0.8
