"""Brute-force evaluation, on meshes of two to four elements, of the parts of a limited stage that the
invariants alone do not fix: the relaxed local bounds of Sec. 5.4, eq. (eq:local_bounds) with the
constants of eq. (ViscMinConst2), the minimal viscosity of Sec. 5.1, eq. (ViscMin), the entropy viscosity
of Sec. 5.2, and the high-order boundary viscosity (the ghost node read as collocated with x_i).  No GPU.

The oracle's traced values are compared with an evaluation written from the equations in a different
form: index sets from a dense adjacency matrix (I(i) = {j : c_ij != 0}) and its boolean square,
collocated pairs from the node coordinates, bar states and specific entropies recomputed in long double
from the input state, and the paper's constants (c_r = 4, p_r = 3/2, c_k = 1, p_k = 1/2 for even and 0
for odd degree, c_ev = 1, 1/2, 1/4 for k = 1, 2, 3) written here rather than read from the oracle.
Inputs taken from the trace: d_ij^L, d_i^{d,L} and N_i, which other pins fix (the exact Riemann bound, the
uniform-flow viscosities, |N| <= 1 and its decay in smooth flow).  Each case also checks that it
discriminates: two-hop bounds that differ from one-hop ones, minimal viscosities that decide d^H, and
collocated pairs of unequal lumped mass."""
import numpy as np
import pytest

from paper_2402_04514_gb300 import assembly, workloads

LD = np.longdouble
G = 1.4
C_R, P_R = 4.0, 1.5
C_K = 1.0


def p_k(k):
    return 0.5 if k % 2 == 0 else 0.0


def c_ev(k):
    return {1: 1.0, 2: 0.5, 3: 0.25}[k]


def graded_1d(widths, k, bc=("slip", "slip")):
    """Q^k on cells of the given widths covering [0, sum(widths)]: in 1D c_ij does not depend on the cell
    width, m_i = w_a h_K and M_K = h_K times the reference mass, so a uniform mesh is rescaled per cell."""
    widths = np.asarray(widths, float)
    E = len(widths)
    P = assembly.assemble_1d(E, k, 0.0, float(widths.sum()), bc=bc)
    h0 = widths.sum() / E
    scale = np.repeat(widths / h0, k + 1)
    P.mi = P.mi * scale
    P.MK = P.MK * (widths / h0)[:, None, None]
    xi, _ = assembly.gauss_lobatto(k)
    left = np.concatenate([[0.0], np.cumsum(widths)[:-1]])
    P.x = (left[:, None] + xi[None, :] * widths[:, None]).reshape(1, -1)
    P.b_x = P.x[:, P.b_node]
    return P


def _state(U, i):
    return np.asarray(U[:, i], LD)


def _flux_dot(V, c):
    """f(V) c for the Euler flux of Sec. 2.2 (eq:euler_flux), V = (rho, m, E), in long double."""
    d = len(c)
    rho, m, E = V[0], V[1:1 + d], V[1 + d]
    p = LD(G - 1.0) * (E - (m * m).sum() / (2 * rho))
    vc = (m * c).sum() / rho
    return np.concatenate([[(m * c).sum()], m * vc + p * c, [(E + p) * vc]])


def _s_tilde(V):
    d = len(V) - 2
    rho = V[0]
    eps = V[-1] - (V[1:1 + d] ** 2).sum() / (2 * rho)
    return rho ** LD(-G) * eps


def _bar(Va, Vb, c, dab):
    """(Va + Vb)/2 - (f(Vb) - f(Va)) c / (2 d): the bar state of eqs. (UsualBarState), (BoundaryBarState)
    with c = c_ab (= |c| n)."""
    return (Va + Vb) / 2 - (_flux_dot(Vb, c) - _flux_dot(Va, c)) / (2 * LD(dab))


def _adjacency(P):
    """Dense A[i, j] = (c_ij != 0) and the position of each (i, j) entry in the CSR arrays."""
    n = P.n
    A = np.zeros((n, n), bool)
    pos = -np.ones((n, n), np.int64)
    rows = np.repeat(np.arange(n), np.diff(P.row_ptr))
    for e, (i, j) in enumerate(zip(rows, P.col_idx)):
        pos[i, j] = e
        A[i, j] = bool(np.any(P.cij[:, e] != 0.0))
    assert not A.diagonal().any()
    return A, pos


def _hand_bounds(P, U, tr, hops=2, element=False):
    """rho_min, rho_max, s_min of eq. (eq:local_bounds) by brute force: states over the two-hop set
    (I(i) and i, then I(j) and j), bar states U_jk over j in I(i) and i, k in I(j), the boundary bar states
    of node i itself, relaxed by r_h^+- = 1 +- c_r h_i^{p_r}, h_i = (m_i / |Omega|)^{1/d}.  hops=1 gives
    the one-hop variant, used only to show that a case tells the two apart.  element=True takes h_i from the
    measure of i's element (the sum of its nodes' lumped masses) instead of m_i."""
    n, d = P.n, P.dim
    A, pos = _adjacency(P)
    A1 = A | np.eye(n, dtype=bool)
    reach = (A1.astype(int) @ A1.astype(int)) > 0 if hops == 2 else A1
    bar_rows = A1 if hops == 2 else np.eye(n, dtype=bool)
    rho = np.array([_state(U, k)[0] for k in range(n)])
    st = np.array([_s_tilde(_state(U, k)) for k in range(n)])
    bar_rho = np.full((n, n), np.inf, dtype=LD)
    bar_rho_hi = np.full((n, n), -np.inf, dtype=LD)
    bar_s = np.full((n, n), np.inf, dtype=LD)
    for j in range(n):
        for k in np.flatnonzero(A[j]):
            e = pos[j, k]
            Ub = _bar(_state(U, j), _state(U, k), np.asarray(P.cij[:, e], LD), tr["dL"][e])
            bar_rho[j, k] = bar_rho_hi[j, k] = Ub[0]
            bar_s[j, k] = _s_tilde(Ub)
    out = {key: np.zeros(n, dtype=LD) for key in ("rho_min", "rho_max", "s_min")}
    for i in range(n):
        S = np.flatnonzero(reach[i])
        J = np.flatnonzero(bar_rows[i])
        lo = min(rho[S].min(), bar_rho[J].min())
        hi = max(rho[S].max(), bar_rho_hi[J].max())
        sl = min(st[S].min(), bar_s[J].min())
        for b in np.flatnonzero(P.b_node == i):
            Ui = _state(U, i)
            cb = np.asarray(P.b_c[:, b], LD)
            nrm = cb / np.sqrt((cb * cb).sum())
            assert P.b_type[b] == assembly.SLIP
            Ug = Ui.copy()
            Ug[1:1 + d] = Ui[1:1 + d] - 2 * (Ui[1:1 + d] * nrm).sum() * nrm
            Ub = _bar(Ui, Ug, cb, tr["dB"][b])
            lo, hi, sl = min(lo, Ub[0]), max(hi, Ub[0]), min(sl, _s_tilde(Ub))
        meas = LD(P.mi[i])
        if element:
            K = i // P.n_loc
            meas = np.asarray(P.mi[K * P.n_loc:(K + 1) * P.n_loc], LD).sum()
        h = (meas / LD(P.omega_measure)) ** (LD(1) / d)
        r = LD(C_R) * h ** LD(P_R)
        out["rho_min"][i] = (1 - r) * lo
        out["rho_max"][i] = (1 + r) * hi
        out["s_min"][i] = (1 - r) * sl
    return out


def _hand_high_order_viscosity(P, tr, k):
    """d^H_ij = max(d^min_ij, d^ev_ij) (Sec. 5, eq. (HighOrderViscosity)) with d^min of eq. (ViscMin) on
    collocated pairs (x_i = x_j, found from the coordinates) and d^ev = d^L min(c_ev max(|N_i|, |N_j|), 1)
    of Sec. 5.2; the boundary viscosity with the ghost node collocated with x_i:
    d^{d,H} = max(c_k h_i^{p_k}, min(c_ev |N_i|, 1)) d^{d,L}, h_i = (m_i / |Omega|)^{1/d}."""
    n, d = P.n, P.dim
    rows = np.repeat(np.arange(n), np.diff(P.row_ptr))
    N = np.asarray(tr["N"], LD)
    dL = np.asarray(tr["dL"], LD)
    dH = np.zeros(P.nnz, dtype=LD)
    dmin_wins = 0
    unequal = 0
    for e, (i, j) in enumerate(zip(rows, P.col_idx)):
        same_place = np.all(P.x[:, i] == P.x[:, j])
        dmin = LD(0)
        if same_place:
            h = (LD(0.5) * (LD(P.mi[i]) + LD(P.mi[j])) / LD(P.omega_measure)) ** (LD(1) / d)
            dmin = LD(C_K) * h ** LD(p_k(k)) * dL[e]
        dev = dL[e] * min(LD(c_ev(k)) * max(abs(N[i]), abs(N[j])), LD(1))
        dH[e] = max(dmin, dev)
        if same_place and dmin > dev:
            dmin_wins += 1
            unequal += P.mi[i] != P.mi[j]
    dBH = np.zeros(P.nb, dtype=LD)
    for b, i in enumerate(P.b_node):
        h = (LD(P.mi[i]) / LD(P.omega_measure)) ** (LD(1) / d)
        dBH[b] = max(LD(C_K) * h ** LD(p_k(k)), min(LD(c_ev(k)) * abs(N[i]), LD(1))) * LD(tr["dB"][b])
    return dH, dBH, dmin_wins, unequal


def _rel(a, b):
    a = np.asarray(a, LD)
    b = np.asarray(b, LD)
    return float(np.abs(a - b).max() / np.abs(b).max())


def _two_state_1d(P, x_split, left, right):
    return workloads.sod(P.x[0], gamma=G, x_split=x_split, left=left, right=right)


def _cases():
    """(name, problem, state, degree): a 1D mesh of two Q1 elements, 2 x 2 Q1 and Q2 meshes with
    four-quadrant data (split off the element faces, so that the jump sits inside elements), and graded 1D
    Q2 and Q3 meshes whose collocated pairs have unequal lumped masses."""
    out = []
    P = assembly.assemble_1d(2, 1)
    out.append(("1d_q1_two_elements", P, _two_state_1d(P, 0.3, (1.0, 0.2, 1.0), (0.3, -0.4, 0.2)), 1))
    for k in (1, 2):
        P = assembly.assemble_2d(2, 2, k)
        U = workloads.four_quadrant(P.x[0], P.x[1], gamma=G, seed=3, split=(0.4, 0.6))
        out.append((f"2d_q{k}_2x2", P, U, k))
    for k in (2, 3):
        P = graded_1d([0.15, 0.35, 0.2, 0.3], k)
        rng = np.random.default_rng(k)
        x = P.x[0]
        rho = np.where(x < 0.62, 1.0, 0.45) + 0.02 * rng.uniform(-1, 1, P.n) * (x > 0.62)
        U = workloads.prim_to_cons(rho, np.where(x < 0.62, 0.3, -0.2)[None, :], np.where(x < 0.62, 1.0, 0.3), G)
        out.append((f"1d_q{k}_graded", P, U, k))
    return out


CASES = _cases()


def _limited_stage(oracle_mod, P, U, k, **extra):
    O = oracle_mod.Oracle(P, gamma=G, params=extra)
    assert (O.params["c_r"], O.params["p_r"], O.params["c_k"], O.params["p_k"], O.params["c_ev"]) == (
        C_R, P_R, C_K, p_k(k), c_ev(k))
    _, flags, tr = O.stage(U, O.max_dt(U, 0.5), trace=True)
    assert flags == 0
    return tr


@pytest.mark.parametrize("case", range(len(CASES)), ids=[c[0] for c in CASES])
def test_relaxed_local_bounds_by_hand(oracle_mod, case):
    """Every traced rho_min, rho_max and s_min equals the brute-force evaluation of eq. (eq:local_bounds)
    within 1e-13 relative; on the 2D and the two-element meshes some node's two-hop bounds differ from its
    one-hop bounds, so the inner set I(j) is exercised."""
    name, P, U, k = CASES[case]
    tr = _limited_stage(oracle_mod, P, U, k)
    want = _hand_bounds(P, U, tr)
    for key in ("rho_min", "rho_max", "s_min"):
        assert _rel(tr[key], want[key]) <= 1e-13, (name, key, _rel(tr[key], want[key]))
    if not name.endswith("graded"):
        one = _hand_bounds(P, U, tr, hops=1)
        assert any((one[key] != want[key]).any() for key in ("rho_min", "rho_max", "s_min")), name


@pytest.mark.parametrize("case", range(len(CASES)), ids=[c[0] for c in CASES])
def test_high_order_viscosity_by_hand(oracle_mod, case):
    """Every traced d^H_ij and d^{d,H} equals the evaluation of eq. (HighOrderViscosity), (ViscMin) and
    d^ev within 1e-13 relative.  For even degree the minimal viscosity decides d^H on some collocated pair
    and d^{d,H} differs from d^{d,L} somewhere; on the graded meshes some such pair joins nodes of unequal
    lumped mass, so h_ij = (0.5 (m_i + m_j) / |Omega|)^{1/d} is exercised."""
    name, P, U, k = CASES[case]
    tr = _limited_stage(oracle_mod, P, U, k)
    dH, dBH, dmin_wins, unequal = _hand_high_order_viscosity(P, tr, k)
    assert _rel(tr["dH"], dH) <= 1e-13, (name, _rel(tr["dH"], dH))
    if P.nb:
        assert _rel(tr["dBH"], dBH) <= 1e-13, (name, _rel(tr["dBH"], dBH))
    if k % 2 == 0:
        assert dmin_wins > 0, name
        assert (np.asarray(tr["dBH"]) != np.asarray(tr["dB"])).any(), name
    if name.endswith("graded"):
        assert unequal > 0, name


ELEMENT_CASES = ["2d_q2_4x4", "1d_q2_graded"]


def _element_case(name):
    if name == "2d_q2_4x4":
        P = assembly.assemble_2d(4, 4, 2)
        return P, workloads.four_quadrant(P.x[0], P.x[1], gamma=G, seed=3, split=(0.4, 0.6)), 2
    return next((P, U, k) for n, P, U, k in CASES if n == name)


@pytest.mark.parametrize("name", ELEMENT_CASES)
def test_relaxed_local_bounds_by_hand_element_measure(oracle_mod, name):
    """The same brute force with the relaxation's mesh size taken from the element (relax_measure = 1):
    h_i = (|K_i| / |Omega|)^{1/d}, |K_i| the sum of the lumped masses of i's element; within 1e-13, and
    different from the node-measure bounds (every node of a Q2 element has m_i < |K_i|)."""
    P, U, k = _element_case(name)
    tr = _limited_stage(oracle_mod, P, U, k, relax_measure=1)
    want = _hand_bounds(P, U, tr, element=True)
    for key in ("rho_min", "rho_max", "s_min"):
        assert _rel(tr[key], want[key]) <= 1e-13, (name, key, _rel(tr[key], want[key]))
    node = _hand_bounds(P, U, tr)
    assert (np.abs(node["rho_max"] - want["rho_max"]) > 1e-6 * np.abs(want["rho_max"])).all()
