"""Pins of the discretisation data (input generator): the identities of Sec. 3.2 and hand values."""
import numpy as np
import pytest

from paper_2402_04514_gb300 import assembly
from tests.helpers import transpose_map


def _all_problems():
    return [
        assembly.assemble_1d(7, 1),
        assembly.assemble_1d(5, 2, periodic=True),
        assembly.assemble_1d(4, 3, x0=-1.0, x1=2.0),
        assembly.assemble_2d(3, 4, 1),
        assembly.assemble_2d(3, 3, 2, periodic=(True, False)),
        assembly.assemble_2d(2, 3, 3, box=(-1.0, 2.0, 0.0, 1.0)),
        assembly.assemble_2d(4, 4, 2, box=(-5, 5, -5, 5), periodic=(True, True)),
        assembly.assemble_3d(2, 3, 2, 1),
        assembly.assemble_3d(2, 2, 3, 2, box=(-1.0, 1.0, 0.0, 0.5, 0.0, 2.0), periodic=(False, True, False)),
    ]


@pytest.mark.parametrize("P", _all_problems(), ids=lambda P: f"d{P.dim}k{P.degree}n{P.n}")
def test_partition_of_unity_and_skew(P):
    """Lemma LemPart (eq. (PartitionBetter)) and Lemma PropSkew (eq. (skewsymm))."""
    tr, rows = transpose_map(P)
    for c in range(P.dim):
        s = np.zeros(P.n)
        np.add.at(s, rows, P.cij[c])
        np.add.at(s, P.b_node, P.b_c[c])
        assert np.abs(s).max() < 1e-14
        assert np.array_equal(P.cij[c][tr], -P.cij[c])  # exact, as the library requires
    assert np.array_equal(P.coloc[tr], P.coloc)


@pytest.mark.parametrize("P", _all_problems(), ids=lambda P: f"d{P.dim}k{P.degree}n{P.n}")
def test_mass(P):
    """eq. (eq:mass_matrices): sum_i m_i = |Omega|, consistent rows sum to m_i, M_K symmetric positive."""
    assert abs(P.mi.sum() - P.omega_measure) < 1e-13 * P.omega_measure
    assert np.abs(P.MK.sum(2).reshape(-1) - P.mi).max() < 1e-15 * max(1.0, P.mi.max()) * 10
    assert np.allclose(P.MK, np.swapaxes(P.MK, 1, 2))
    assert np.linalg.eigvalsh(P.MK[0]).min() > 0


@pytest.mark.parametrize("P", [p for p in _all_problems() if p.nb > 0 or True],
                         ids=lambda P: f"d{P.dim}k{P.degree}n{P.n}")
def test_rows_hold_element_and_collocated_partners(P):
    tr, rows = transpose_map(P)
    same = (rows // P.n_loc) == (P.col_idx // P.n_loc)
    cnt = np.bincount(rows[same], minlength=P.n)
    assert (cnt == P.n_loc - 1).all()
    dxa = np.abs(P.x[:, rows] - P.x[:, P.col_idx])
    dx = dxa.max(0)
    # collocated partners coincide, except across a periodic seam, where they lie more than half the
    # domain's extent apart along the periodic axis
    periodic_seam = P.coloc.astype(bool) & (dx > 1e-12)
    span = P.x.max(1) - P.x.min(1)
    assert (dxa[:, periodic_seam] > 0.5 * span[:, None]).any(0).all() if periodic_seam.any() else True
    assert (dx[~P.coloc.astype(bool)] > 0).all()
    assert not (P.coloc.astype(bool) & same).any()


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_polynomial_consistency(dim, k):
    """For a continuous u in Q^k: sum_j u_j c_ij + u_i c_i^d = m_i grad u(x_i) (eq. (eq:cij_def1),
    eq. (eq:cij_def2) with the face terms cancelling between collocated nodes)."""
    if dim == 1:
        P = assembly.assemble_1d(5, k, x0=-1.0, x1=1.5)
        x = P.x[0]
        u = 0.3 + 0.7 * x + (x ** k if k > 1 else 0.0)
        grad = [0.7 + (k * x ** (k - 1) if k > 1 else 0.0)]
    elif dim == 2:
        P = assembly.assemble_2d(3, 2, k, box=(-1.0, 2.0, 0.5, 1.5))
        x, y = P.x
        u = 0.3 + 0.7 * x - 1.1 * y + 0.2 * x * y + 0.1 * x ** k * y ** k
        grad = [0.7 + 0.2 * y + 0.1 * k * x ** (k - 1) * y ** k, -1.1 + 0.2 * x + 0.1 * k * x ** k * y ** (k - 1)]
    else:
        if k == 3:
            pytest.skip("Q3 in 3D has 64 nodes per element (the library takes at most 32)")
        P = assembly.assemble_3d(2, 3, 2, k, box=(-1.0, 2.0, 0.5, 1.5, 0.0, 1.0))
        x, y, z = P.x
        u = 0.3 + 0.7 * x - 1.1 * y + 0.4 * z + 0.2 * x * y * z + 0.1 * x ** k * y ** k * z ** k
        grad = [0.7 + 0.2 * y * z + 0.1 * k * x ** (k - 1) * y ** k * z ** k,
                -1.1 + 0.2 * x * z + 0.1 * k * x ** k * y ** (k - 1) * z ** k,
                0.4 + 0.2 * x * y + 0.1 * k * x ** k * y ** k * z ** (k - 1)]
    rows = np.repeat(np.arange(P.n), np.diff(P.row_ptr))
    for c in range(dim):
        s = np.zeros(P.n)
        np.add.at(s, rows, u[P.col_idx] * P.cij[c])
        np.add.at(s, P.b_node, u[P.b_node] * P.b_c[c])
        assert np.abs(s - P.mi * grad[c]).max() < 1e-12


def test_hand_values_1d_q1():
    """Q1 on [0, 1] with 4 cells, worked by hand from eq. (eq:cij_def2): in-element c_ij = +-1/2,
    face c_ij = n/2, c_i^d = n/2, m_i = h/2, M_K = h/6 [[2, 1], [1, 2]]."""
    P = assembly.assemble_1d(4, 1)
    h = 0.25
    assert np.allclose(P.mi, h / 2)
    assert np.allclose(P.MK[0], h / 6 * np.array([[2.0, 1.0], [1.0, 2.0]]))
    rows = np.repeat(np.arange(P.n), np.diff(P.row_ptr))
    C = {(int(i), int(j)): c for i, j, c in zip(rows, P.col_idx, P.cij[0])}
    assert C[(0, 1)] == 0.5 and C[(1, 0)] == -0.5  # in element 0
    assert C[(1, 2)] == 0.5 and C[(2, 1)] == -0.5  # face x = 0.25, outward normals +1 / -1
    assert list(P.b_node) == [0, 7] and list(P.b_c[0]) == [-0.5, 0.5]
    assert len(C) == 2 * 4 + 2 * 3


def test_q2_row_lengths():
    """2D Q2: 8 in-element entries (4 with c_ij != 0) plus 2/1/0 face partners at corner/edge/centre."""
    P = assembly.assemble_2d(3, 3, 2, periodic=(True, True))
    r = np.diff(P.row_ptr).reshape(-1, 9)
    assert (r[:, [0, 2, 6, 8]] == 10).all() and (r[:, [1, 3, 5, 7]] == 9).all() and (r[:, 4] == 8).all()
    nz = (np.abs(P.cij).sum(0) > 0)
    rows = np.repeat(np.arange(P.n), np.diff(P.row_ptr))
    stencil = np.bincount(rows[nz], minlength=P.n).reshape(-1, 9)
    assert (stencil[:, 4] == 4).all() and (stencil[:, 0] == 6).all()
