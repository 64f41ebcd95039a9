"""Shared test helpers: problem builders, error norms, golden-file loading."""
from __future__ import annotations

import os

import numpy as np

from paper_2402_04514_gb300 import assembly, workloads

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_vortex_tables():
    rows = []
    with open(os.path.join(GOLDEN, "vortex_l1_tables.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    a = np.array(rows)
    return dict(dofs=a[:, 0].astype(int), limited={1: a[:, 1], 2: a[:, 2], 3: a[:, 3]},
                first_order={1: a[:, 4], 2: a[:, 5], 3: a[:, 6]})


def four_quadrant_problem(ne, degree, seed=0, gamma=1.4):
    P = assembly.assemble_2d(ne, ne, degree)
    U = workloads.four_quadrant(P.x[0], P.x[1], gamma=gamma, seed=seed)
    return P, U


def octant_problem(shape, degree, seed=0, gamma=1.4, bc=None):
    """A 3D Riemann problem on [0,1]^3: eight octants split at 0.5 with states drawn from default_rng(seed)
    (rho, p ~ U[0.1, 2], velocity components ~ U[-1, 1])."""
    P = assembly.assemble_3d(*shape, degree, bc=bc)
    rng = np.random.default_rng(seed)
    x, y, z = P.x
    o = (x > 0.5).astype(int) + 2 * (y > 0.5) + 4 * (z > 0.5)
    rho, p = rng.uniform(0.1, 2.0, 8)[o], rng.uniform(0.1, 2.0, 8)[o]
    U = workloads.prim_to_cons(rho, rng.uniform(-1.0, 1.0, (3, 8))[:, o], p, gamma)
    return P, U


def periodic_vortex_problem(ne, degree, gamma=1.4):
    P = assembly.assemble_2d(ne, ne, degree, box=(-5.0, 5.0, -5.0, 5.0), periodic=(True, True))
    U = workloads.vortex(P.x[0], P.x[1], 0.0, gamma=gamma)
    return P, U


def dirichlet_vortex_problem(ne, degree, gamma=5.0 / 3.0):
    sides = dict(left="dirichlet", right="dirichlet", bottom="dirichlet", top="dirichlet")
    P = assembly.assemble_2d(ne, ne, degree, box=(-5.0, 5.0, -5.0, 5.0), bc=sides)
    U = workloads.vortex(P.x[0], P.x[1], 0.0, gamma=gamma)

    def bdata(t):
        return workloads.vortex(P.b_x[0], P.b_x[1], t, gamma=gamma)

    return P, U, bdata


def consolidated_l1(P, U, Ue):
    """Sec. 6.2 error: sum over rho, momentum, E of ||q_h - q||_L1 / ||q||_L1 (lumped quadrature;
    |.| of the momentum is the Euclidean norm)."""
    d = P.dim
    err = 0.0
    for sl in (slice(0, 1), slice(1, d + 1), slice(d + 1, d + 2)):
        dif = np.sqrt(((U[sl] - Ue[sl]) ** 2).sum(0))
        ref = np.sqrt((Ue[sl] ** 2).sum(0))
        err += float((P.mi * dif).sum() / (P.mi * ref).sum())
    return err


def transpose_map(P):
    n = P.n
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(P.row_ptr))
    key = rows * n + P.col_idx
    tkey = P.col_idx.astype(np.int64) * n + rows
    order = np.argsort(key)
    pos = np.searchsorted(key[order], tkey)
    tr = order[pos]
    assert (key[tr] == tkey).all()
    return tr, rows


def entropy(U, gamma):
    """Sec. 2.2, eq. (EntropyEuler): s = log(rho^{-gamma} p), eta = -rho s, q = -m s."""
    d = U.shape[0] - 2
    rho = U[0]
    p = (gamma - 1.0) * (U[d + 1] - 0.5 * (U[1:d + 1] ** 2).sum(0) / rho)
    s = np.log(rho ** (-gamma) * p)
    return s, -rho * s, -U[1:d + 1] * s


def rel_err(a, b):
    """Per-component max |a - b| / max |b| (the parity norm), maximised over components."""
    a = np.atleast_2d(a)
    b = np.atleast_2d(b)
    out = 0.0
    for c in range(b.shape[0]):
        scale = max(np.abs(b[c]).max(), 1e-300)
        out = max(out, float(np.abs(a[c] - b[c]).max() / scale))
    return out


def inoutflow_case(name):
    """The in/outflow cases of the GPU tests: (problem, initial state, boundary data [m][nb])."""
    if name == "sod1d_open":
        P = assembly.assemble_1d(200, 1, bc=("inoutflow", "inoutflow"))
        U = workloads.sod(P.x[0])
        return P, U, np.ascontiguousarray(workloads.sod(P.b_x[0]))
    if name == "oct_q1_3d_open":
        P, U = octant_problem((5, 4, 4), 1, seed=3, bc=dict(left="inoutflow", right="inoutflow", back="inoutflow"))
        return P, U, np.ascontiguousarray(U[:, P.b_node])
    if name == "fq_q2_open_sides":
        P = assembly.assemble_2d(13, 13, 2, bc=dict(left="inoutflow", right="inoutflow"))
        U = workloads.four_quadrant(P.x[0], P.x[1], seed=0)
        return P, U, np.ascontiguousarray(U[:, P.b_node])
    # supersonic stream (Mach ~2.6 along x) over a density bump
    sides = dict(left="inoutflow", right="inoutflow", bottom="inoutflow", top="inoutflow")
    P = assembly.assemble_2d(16, 16, 1, bc=sides)
    x, y = P.x
    rho = 1.0 + 0.5 * np.exp(-40 * ((x - 0.4) ** 2 + (y - 0.5) ** 2))
    U = workloads.prim_to_cons(rho, np.stack([np.full(P.n, 3.0), np.full(P.n, 0.5)]), np.full(P.n, 1.0), 1.4)
    bd = workloads.prim_to_cons(np.full(P.nb, 1.0), np.stack([np.full(P.nb, 3.0), np.full(P.nb, 0.5)]),
                                np.full(P.nb, 1.0), 1.4)
    return P, U, np.ascontiguousarray(bd)
