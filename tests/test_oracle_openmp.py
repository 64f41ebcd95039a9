"""The multi-core timing build of the oracle (row loops shared by OpenMP, used only to time the CPU
baseline) gives bit-identical results to the pinned single-thread build: every row writes only its own
entries.  No GPU."""
import numpy as np
import pytest

from tests.helpers import four_quadrant_problem, octant_problem


@pytest.mark.parametrize("case", ["fq_q2", "oct_q1_3d"])
def test_openmp_build_is_bit_identical(oracle_mod, case, monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "4")
    P, U = four_quadrant_problem(12, 2, seed=1) if case == "fq_q2" else octant_problem((5, 4, 4), 1, seed=2)
    one = oracle_mod.Oracle(P)
    many = oracle_mod.Oracle(P, openmp=True)
    assert oracle_mod.threads(False) == 1
    tau = one.max_dt(U, 0.5)
    assert many.max_dt(U, 0.5) == tau
    for _ in range(2):
        a, fa, ta = one.stage(U, tau, trace=True)
        b, fb, tb = many.stage(U, tau, trace=True)
        assert fa == fb and np.array_equal(a, b)
        for key in ta:
            assert np.array_equal(ta[key], tb[key]), key
        U = a
