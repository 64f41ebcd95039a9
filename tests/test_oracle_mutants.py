"""The pins catch plausible mistakes: each mutant below is a copy of oracle.c with one planted error (a
dropped term, a flipped sign, a swapped operand or index), compiled on the CPU; the pins of
test_oracle_pins.py, test_oracle_hand.py and test_oracle_bc.py must reject every mutant.  The real oracle is untouched."""
import os
import subprocess
import tempfile

import pytest

from oracle import oracle as om
from tests import test_oracle_bc as bc
from tests import test_oracle_hand as hand
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(om.__file__), "oracle.c")

MUTANTS = {
    "drop_boundary_viscosity": ("for (int q = 0; q < m; ++q) acc[q] += fv[q] - dB[b] * (Ub[q] - Ui[q]);",
                                "for (int q = 0; q < m; ++q) acc[q] += fv[q];"),
    "viscosity_sign": ("acc[q] += fv[q] - dL[e] * (Uj[q] - Ui[q]);", "acc[q] += fv[q] + dL[e] * (Uj[q] - Ui[q]);"),
    "lambda_swapped_velocities": ("double num = aL + aR - 0.5 * (g - 1.0) * (uR - uL);",
                                  "double num = aL + aR - 0.5 * (g - 1.0) * (uL - uR);"),
    "bar_state_sign": ("out[q] = 0.5 * (Ui[q] + Uj[q]) - cn / (2.0 * dij) * (fj[q] - fi[q]);",
                       "out[q] = 0.5 * (Ui[q] + Uj[q]) + cn / (2.0 * dij) * (fj[q] - fi[q]);"),
    "mass_term_sign": ("-\n                           mij * (dUH[q * n + j] - dUH[q * n + i]);",
                       "+\n                           mij * (dUH[q * n + j] - dUH[q * n + i]);"),
    "limiter_max_instead_of_min": ("lsym[e] = fmin(lraw[e], lraw[transpose_entry(P, i, P->col_idx[e])]);",
                                   "lsym[e] = fmax(lraw[e], lraw[transpose_entry(P, i, P->col_idx[e])]);"),
    "line_search_ignores_entropy": ("  double fb = psi(U0, Pv, l, d, g, smin);\n  if (fb >= 0.0) return l;",
                                    "  double fb = psi(U0, Pv, l, d, g, smin);\n  return l;"),
    "relaxation_swapped": ("rmin[i] = rm * lo; rmax[i] = rp * hi; smin[i] = rm * sl;",
                           "rmin[i] = rp * lo; rmax[i] = rm * hi; smin[i] = rm * sl;"),
    "slip_half_reflection": ("UB[1 + k] = Ui[1 + k] - 2.0 * mn * nrm[k];", "UB[1 + k] = Ui[1 + k] - mn * nrm[k];"),
    "cfl_factor_dropped": ("if (dii[i] < 0.0) t = fmin(t, -P->mi[i] / (2.0 * dii[i]));",
                           "if (dii[i] < 0.0) t = fmin(t, -P->mi[i] / dii[i]);"),
    # solve with the lumped mass instead of the consistent element mass M_K
    "consistent_mass_dropped": ("element_solve(P->MK + K * nl * nl, nl, m, Bblk);",
                                "for (int a = 0; a < nl; ++a) for (int q = 0; q < m; ++q) Bblk[a * m + q] /= "
                                "P->mi[K * nl + a];"),
    "ev_uses_only_own_residual": ("fmin(P->c_ev * fmax(fabs(N[i]), fabs(N[j])), 1.0);",
                                  "fmin(P->c_ev * fabs(N[i]), 1.0);"),
    "entropy_gradient_sign": ("grad[d + 1] = pref * ((g - 1.0) / pi);", "grad[d + 1] = -pref * ((g - 1.0) / pi);"),
    "entropy_flux_difference_reversed": ("psum += dot(Uj + 1, c, d) * (fj - fi);", "psum += dot(Uj + 1, c, d) * (fi - fj);"),
    "bounds_skip_bar_states": ("lo = fmin(lo, fmin(Uk[0], Ubk[0]));", "lo = fmin(lo, Uk[0]);"),
    # in/outflow boundary state (Sec. 4.1)
    "inoutflow_incoming_riemann_invariant_from_interior": ("double R1 = vnd - 2.0 * ad / (g - 1.0);",
                                                          "double R1 = vni - 2.0 * ai / (g - 1.0);"),
    "inoutflow_entropy_from_the_wrong_side": (
        "double R2 = vni <= 0.0 ? pd / pow(Ud[0], g) : pi / pow(Ui[0], g);",
        "double R2 = vni <= 0.0 ? pi / pow(Ui[0], g) : pd / pow(Ud[0], g);"),
    "supersonic_inflow_keeps_the_interior": ("  if (vni < -ai) {\n    for (int q = 0; q < m; ++q) UB[q] = Ud[q];",
                                             "  if (vni < -ai) {\n    for (int q = 0; q < m; ++q) UB[q] = Ui[q];"),
    # the limiter's direction and closed form (Sec. 5.4)
    "limiter_kappa_dropped": ("Pv[q] = Arem[q * nnz + e] / (kappa * P->mi[i]);", "Pv[q] = Arem[q * nnz + e] / P->mi[i];"),
    "density_bound_from_the_wrong_side": ("if (U0[0] + Pv[0] > rmax) l = (rmax - U0[0]) / Pv[0];",
                                          "if (U0[0] + Pv[0] > rmax) l = (rmin - U0[0]) / Pv[0];"),
    # the relaxed local bounds (Sec. 5.4, eq. (eq:local_bounds), (ViscMinConst2))
    "bounds_upper_relaxation_doubled": ("double rm = 1.0 - P->c_r * hh, rp = 1.0 + P->c_r * hh;",
                                        "double rm = 1.0 - P->c_r * hh, rp = 1.0 + 2.0 * P->c_r * hh;"),
    "bounds_one_hop_only": ("for (long ek = P->row_ptr[j]; ek < P->row_ptr[j + 1]; ++ek) {",
                            "for (long ek = P->row_ptr[j]; ek < P->row_ptr[j + 1] && j == i; ++ek) {"),
    "bounds_mesh_size_without_the_dimension_root": ("double hh = pow(pow(meas / P->omega, 1.0 / d), P->p_r);",
                                                    "double hh = pow(meas / P->omega, P->p_r);"),
    "relaxation_element_measure_from_one_node": ("for (long a = (i / nl) * nl; a < (i / nl + 1) * nl; ++a) meas += P->mi[a];",
                                                 "for (long a = (i / nl) * nl; a < (i / nl + 1) * nl; ++a) meas = P->mi[a];"),
    # the minimal and boundary high-order viscosities (Sec. 5.1, eq. (ViscMin); the boundary reading)
    "minimal_viscosity_power_dropped": ("dmin = P->c_k * pow(hij, P->p_k) * dL[e];", "dmin = P->c_k * dL[e];"),
    "minimal_viscosity_mesh_size_of_the_row_node": (
        "double hij = pow(0.5 * (P->mi[i] + P->mi[j]) / P->omega, 1.0 / d);",
        "double hij = pow(P->mi[i] / P->omega, 1.0 / d);"),
    "boundary_high_order_viscosity_is_the_low_order_one": (
        "dBH[b] = fmax(P->c_k * pow(hi, P->p_k), fmin(P->c_ev * fabs(N[i]), 1.0)) * dB[b];", "dBH[b] = dB[b];"),
    # dimension handling that only a 3D mesh exercises
    "flux_pressure_only_in_the_first_two_directions": (
        "for (int k = 0; k < d; ++k) out[1 + k] = U[1 + k] * vc + p * c[k];",
        "for (int k = 0; k < d; ++k) out[1 + k] = U[1 + k] * vc + (k < 2 ? p * c[k] : 0.0);"),
    "kinetic_energy_of_the_first_two_components": ("for (int k = 0; k < d; ++k) m2 += U[1 + k] * U[1 + k];",
                                                   "for (int k = 0; k < d && k < 2; ++k) m2 += U[1 + k] * U[1 + k];"),
}

FAST_PINS = [
    lambda O: pins.test_lambda_max_bounds_exact_wave_speed(O, 1.4),
    lambda O: pins.test_lambda_max_symmetry(O),
    lambda O: pins.test_constant_state_preserved(O),
    lambda O: pins.test_convex_reformulation(O, 2),
    lambda O: pins.test_low_order_invariants(O, 2),
    lambda O: [pins.test_conservation(O, order, 2) for order in (0, 1, 2)],
    lambda O: pins.test_high_low_identity_and_limiter_knobs(O, 2),
    lambda O: pins.test_limiter_is_identity_when_bounds_are_loose(O),
    lambda O: pins.test_limited_state_within_local_bounds(O, 2, 4.0),
    lambda O: pins.test_limited_state_within_local_bounds(O, 2, 0.0),
    lambda O: pins.test_sod_exact_solution(O),
    lambda O: pins.test_line_search_converges_to_the_root(O),
    lambda O: pins.test_stage_limiter_factors_by_brute_force(O),
    lambda O: pins.test_viscosity_and_time_step_of_a_uniform_flow(O),
    lambda O: pins.test_entropy_indicator_vanishes_in_smooth_flow(O),
    lambda O: [hand.test_relaxed_local_bounds_by_hand(O, c) for c in range(len(hand.CASES))],
    lambda O: [hand.test_high_order_viscosity_by_hand(O, c) for c in range(len(hand.CASES))],
    lambda O: [hand.test_relaxed_local_bounds_by_hand_element_measure(O, c) for c in hand.ELEMENT_CASES],
]


DIM3_PINS = [
    lambda O: pins.test_3d_reduces_to_1d(O, 2, "LOW"),
    lambda O: pins.test_3d_limited_stage_invariants(O),
]


BC_PINS = [
    lambda O: bc.test_supersonic_cases_take_data_or_interior_exactly(),
    lambda O: bc.test_subsonic_characteristics_come_from_the_right_side(),
    lambda O: bc.test_shock_leaves_the_domain_without_reflection(2),
]


def _vortex_q1_limited(O):
    tab = pins.load_vortex_tables()
    e1 = pins._vortex_error(O, 24, 1, O.LIMITED)
    assert abs(e1 / tab["limited"][1][0] - 1.0) < 0.2, e1


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, monkeypatch):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "oracle.c")
        open(c, "w").write(src.replace(old, new))
        subprocess.check_call(["cp", os.path.join(os.path.dirname(SRC), "oracle.h"), d])
        so = os.path.join(d, "liboracle_mutant.so")
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", c, "-o", so, "-lm"])
        monkeypatch.setattr(om, "_libs", {})
        monkeypatch.setattr(om, "build", lambda force=False, openmp=False: so)
        caught = []
        for pin in FAST_PINS + BC_PINS + DIM3_PINS + [_vortex_q1_limited]:
            try:
                pin(om)
            except (AssertionError, ValueError, FloatingPointError):
                caught.append(pin)
                break
        assert caught, f"no pin rejects mutant {name}"
