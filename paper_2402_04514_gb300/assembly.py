"""Discretisation data for the graph-based dG scheme: Q^k Gauss-Lobatto elements on uniform meshes.

This module builds the *inputs* of a stage (Sec. 2.3, Eqs. (2.4)-(2.6) and the multi-valued boundary
split of Sec. 4.2): the stencil as CSR, the vector-valued matrix c_ij, the lumped mass m_i, the
consistent element mass blocks M_K and the boundary entries (i, c_i^{d,k}, type).  It contains none of
the stage arithmetic (fluxes, viscosities, limiter); both the CUDA library and the CPU oracle consume
what it produces.

Quadrature (the paper does not fix it): the Gauss-Lobatto points of the nodal basis are also the
quadrature points for c_ij^K, c_ij^{dK}, c_i^d and m_i.  This collocated choice is a summation-by-parts
pair, so c_ii = 0, the partition of unity (Lemma 3.1) and the skew symmetry c_ij = -c_ji (Lemma 3.2)
hold exactly, and face coupling only links collocated nodes.  The consistent mass m_ij is integrated
exactly (Gauss-Legendre with k+1 points per direction).

Node numbering is element-contiguous: element e owns nodes [e*n_loc, (e+1)*n_loc); in 2D the local
node (a, b) (a along x, b along y) has local index b*(k+1) + a and elements are numbered ey*nx + ex; in 3D
the local node (a, b, c) has local index (c*(k+1) + b)*(k+1) + a and elements are numbered
(ez*ny + ey)*nx + ex.
Each CSR row i lists every other node of its element (m_ij != 0 couples them all) and its collocated
face partners; entries whose c_ij is zero (the in-element nodes that share neither the x-line nor the
y-line of i) are kept because the consistent mass couples them in the high-order update (Eq. (5.1)).
Row order: in-element stencil entries, face partners, then mass-only entries.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SLIP = 0
DIRICHLET = 1
INOUTFLOW = 2
BC_CODES = {"slip": SLIP, "dirichlet": DIRICHLET, "inoutflow": INOUTFLOW}

# Boundary part ids (one per side; corners carry one entry per side, Sec. 4.2).
PART_LEFT, PART_RIGHT, PART_BOTTOM, PART_TOP, PART_FRONT, PART_BACK = 0, 1, 2, 3, 4, 5


@dataclass
class Problem:
    """One mesh instance in the layout the stage consumes (all host numpy arrays)."""

    dim: int
    degree: int
    n: int
    n_loc: int
    row_ptr: np.ndarray  # int64 [n+1]
    col_idx: np.ndarray  # int32 [nnz]
    cij: np.ndarray  # float64 [dim][nnz]
    coloc: np.ndarray  # uint8 [nnz]; 1 iff x_i == x_j (face partner)
    mi: np.ndarray  # float64 [n]
    MK: np.ndarray  # float64 [n_elem][n_loc][n_loc]
    b_node: np.ndarray  # int32 [nb]
    b_c: np.ndarray  # float64 [dim][nb]
    b_type: np.ndarray  # int32 [nb]
    b_part: np.ndarray  # int32 [nb]
    omega_measure: float
    x: np.ndarray  # float64 [dim][n] node coordinates
    b_x: np.ndarray = field(default=None)  # float64 [dim][nb] coordinates of the boundary node

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def nb(self) -> int:
        return int(self.b_node.shape[0])

    @property
    def m(self) -> int:
        return self.dim + 2

    @property
    def n_elem(self) -> int:
        return self.n // self.n_loc


def gauss_lobatto(k: int):
    """Gauss-Lobatto points and weights of degree k on [0, 1] (k+1 points)."""
    if k < 1:
        raise ValueError("degree must be >= 1")
    P = np.polynomial.legendre.Legendre.basis(k)
    interior = np.sort(P.deriv().roots().real) if k > 1 else np.zeros(0)
    x = np.concatenate([[-1.0], interior, [1.0]])
    w = 2.0 / (k * (k + 1) * P(x) ** 2)
    xi = 0.5 * (x + 1.0)
    xi[0], xi[-1] = 0.0, 1.0
    if k % 2 == 0:
        xi[k // 2] = 0.5
    wi = 0.5 * w
    wi = 0.5 * (wi + wi[::-1])  # exact mirror symmetry
    return xi, wi


def _bary_weights(xi):
    n = len(xi)
    lam = np.ones(n)
    for a in range(n):
        for b in range(n):
            if a != b:
                lam[a] /= xi[a] - xi[b]
    return lam


def lagrange_eval(xi, t):
    """L[q, b] = ell_b(t_q) for the Lagrange basis on nodes xi."""
    n = len(xi)
    L = np.ones((len(t), n))
    for b in range(n):
        for c in range(n):
            if c != b:
                L[:, b] *= (t - xi[c]) / (xi[b] - xi[c])
    return L


def sbp_matrix(xi, wi):
    """Q[a, b] = w_a ell_b'(xi_a), made exactly skew off the diagonal (Lemma 3.2)."""
    lam = _bary_weights(xi)
    n = len(xi)
    D = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            if a != b:
                D[a, b] = (lam[b] / lam[a]) / (xi[a] - xi[b])
    Q = wi[:, None] * D
    for a in range(n):
        for b in range(a + 1, n):
            q = 0.5 * (Q[a, b] - Q[b, a])
            Q[a, b], Q[b, a] = q, -q
    return Q


def ref_mass(xi):
    """Exact reference mass matrix int_0^1 ell_a ell_b (Gauss-Legendre, k+1 points)."""
    n = len(xi)
    t, w = np.polynomial.legendre.leggauss(n)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    L = lagrange_eval(xi, t)
    M = (L * w[:, None]).T @ L
    return 0.5 * (M + M.T)


def _compress(valid, *arrays):
    flat = valid.reshape(-1)
    return [a.reshape(-1)[flat] for a in arrays]


def assemble_1d(n_cells: int, degree: int, x0: float = 0.0, x1: float = 1.0,
                periodic: bool = False, bc=("slip", "slip")) -> Problem:
    """Q^k dG on n_cells uniform cells of [x0, x1]; bc = (left, right) types unless periodic."""
    k = degree
    nl = k + 1
    E = n_cells
    h = (x1 - x0) / E
    xi, wi = gauss_lobatto(k)
    Q = sbp_matrix(xi, wi)
    Mr = ref_mass(xi)
    n = E * nl
    e = np.arange(E)
    maxr = nl - 1 + 1
    col = np.zeros((E, nl, maxr), np.int64)
    cx = np.zeros((E, nl, maxr))
    co = np.zeros((E, nl, maxr), np.uint8)
    valid = np.zeros((E, nl, maxr), bool)
    b_node, b_c, b_part = [], [], []
    for a in range(nl):
        s = 0
        for a2 in range(nl):  # in-element: every other node is in the stencil in 1D
            if a2 == a:
                continue
            col[:, a, s] = e * nl + a2
            cx[:, a, s] = Q[a, a2]
            valid[:, a, s] = True
            s += 1
        if a in (0, k):
            sgn = -1.0 if a == 0 else 1.0
            nb_e = e - 1 if a == 0 else e + 1
            other = k if a == 0 else 0
            if periodic:
                nb_e = nb_e % E
                inside = np.ones(E, bool)
            else:
                inside = (nb_e >= 0) & (nb_e < E)
            col[inside, a, s] = nb_e[inside] * nl + other
            cx[inside, a, s] = 0.5 * sgn
            co[inside, a, s] = 1
            valid[inside, a, s] = True
            bnd = ~inside
            if bnd.any():
                b_node.append(e[bnd] * nl + a)
                b_c.append(np.full(bnd.sum(), 0.5 * sgn))
                b_part.append(np.full(bnd.sum(), PART_LEFT if a == 0 else PART_RIGHT))
    counts = valid.reshape(n, maxr).sum(1)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col_c, cx_c, co_c = _compress(valid, col, cx, co)
    mi = (np.tile(wi, E) * h).astype(np.float64)
    MK = np.broadcast_to(Mr * h, (E, nl, nl)).copy()
    b_node = np.concatenate(b_node).astype(np.int32) if b_node else np.zeros(0, np.int32)
    b_cx = np.concatenate(b_c) if b_c else np.zeros(0)
    b_part = np.concatenate(b_part).astype(np.int32) if b_part else np.zeros(0, np.int32)
    order = np.argsort(b_node, kind="stable")
    b_node, b_cx, b_part = b_node[order], b_cx[order], b_part[order]
    types = np.array([BC_CODES[bc[0]], BC_CODES[bc[1]]], np.int32)
    x = (x0 + (e[:, None] + xi[None, :]) * h).reshape(1, n)
    return Problem(dim=1, degree=k, n=n, n_loc=nl, row_ptr=row_ptr, col_idx=col_c.astype(np.int32),
                   cij=cx_c.reshape(1, -1).copy(), coloc=co_c.astype(np.uint8), mi=mi, MK=MK,
                   b_node=b_node, b_c=b_cx.reshape(1, -1).copy(), b_type=types[b_part] if len(b_part) else
                   np.zeros(0, np.int32), b_part=b_part, omega_measure=float(x1 - x0), x=x,
                   b_x=x[:, b_node])


def assemble_2d(nx: int, ny: int, degree: int, box=(0.0, 1.0, 0.0, 1.0),
                periodic=(False, False), bc=None) -> Problem:
    """Q^k dG on an nx x ny uniform quad mesh of box = (x0, x1, y0, y1).

    bc maps 'left'/'right'/'bottom'/'top' to 'slip', 'dirichlet' or 'inoutflow' (sides that are not periodic).
    """
    k = degree
    p1 = k + 1
    nl = p1 * p1
    x0, x1, y0, y1 = box
    hx = (x1 - x0) / nx
    hy = (y1 - y0) / ny
    bc = {**dict(left="slip", right="slip", bottom="slip", top="slip"), **(bc or {})}
    xi, wi = gauss_lobatto(k)
    Q = sbp_matrix(xi, wi)
    Mr = ref_mass(xi)
    E = nx * ny
    n = E * nl
    e = np.arange(E, dtype=np.int64)
    ex = e % nx
    ey = e // nx
    maxr = nl - 1 + 2
    col = np.zeros((E, nl, maxr), np.int64)
    cx = np.zeros((E, nl, maxr))
    cy = np.zeros((E, nl, maxr))
    co = np.zeros((E, nl, maxr), np.uint8)
    valid = np.zeros((E, nl, maxr), bool)
    bnodes, bcx, bcy, bparts = [], [], [], []
    for b in range(p1):
        for a in range(p1):
            l = b * p1 + a
            s = 0
            for a2 in range(p1):  # same x-line: c = (w_b hy Q[a, a2], 0)
                if a2 != a:
                    col[:, l, s] = e * nl + b * p1 + a2
                    cx[:, l, s] = wi[b] * hy * Q[a, a2]
                    valid[:, l, s] = True
                    s += 1
            for b2 in range(p1):  # same y-line: c = (0, w_a hx Q[b, b2])
                if b2 != b:
                    col[:, l, s] = e * nl + b2 * p1 + a
                    cy[:, l, s] = wi[a] * hx * Q[b, b2]
                    valid[:, l, s] = True
                    s += 1
            # face partners (collocated); sides of the domain become boundary entries
            for axis, idx, side_lo in ((0, a, "left"), (1, b, "bottom")):
                if idx not in (0, k):
                    continue
                lo = idx == 0
                sgn = -1.0 if lo else 1.0
                if axis == 0:
                    nex = ex - 1 if lo else ex + 1
                    if periodic[0]:
                        nex = nex % nx
                    inside = (nex >= 0) & (nex < nx)
                    ne = ey * nx + nex
                    other = b * p1 + (k if lo else 0)
                    val = 0.5 * wi[b] * hy * sgn
                    part = PART_LEFT if lo else PART_RIGHT
                else:
                    ney = ey - 1 if lo else ey + 1
                    if periodic[1]:
                        ney = ney % ny
                    inside = (ney >= 0) & (ney < ny)
                    ne = ney * nx + ex
                    other = (k if lo else 0) * p1 + a
                    val = 0.5 * wi[a] * hx * sgn
                    part = PART_BOTTOM if lo else PART_TOP
                col[inside, l, s] = ne[inside] * nl + other
                if axis == 0:
                    cx[inside, l, s] = val
                else:
                    cy[inside, l, s] = val
                co[inside, l, s] = 1
                valid[inside, l, s] = True
                s += 1
                bnd = ~inside
                if bnd.any():
                    cnt = int(bnd.sum())
                    bnodes.append(e[bnd] * nl + l)
                    bcx.append(np.full(cnt, val if axis == 0 else 0.0))
                    bcy.append(np.full(cnt, val if axis == 1 else 0.0))
                    bparts.append(np.full(cnt, part))
            for b2 in range(p1):  # mass-only entries (c_ij = 0)
                for a2 in range(p1):
                    if a2 != a and b2 != b:
                        col[:, l, s] = e * nl + b2 * p1 + a2
                        valid[:, l, s] = True
                        s += 1
    counts = valid.reshape(n, maxr).sum(1)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col_c, cx_c, cy_c, co_c = _compress(valid, col, cx, cy, co)
    del col, cx, cy, co, valid
    wloc = np.outer(wi, wi).reshape(-1)  # index b*p1 + a -> w_b * w_a
    mi = np.tile(wloc * hx * hy, E)
    MK = np.broadcast_to(np.kron(Mr, Mr) * (hx * hy), (E, nl, nl)).copy()
    if bnodes:
        b_node = np.concatenate(bnodes).astype(np.int32)
        b_cx = np.concatenate(bcx)
        b_cy = np.concatenate(bcy)
        b_part = np.concatenate(bparts).astype(np.int32)
        order = np.lexsort((b_part, b_node))
        b_node, b_cx, b_cy, b_part = b_node[order], b_cx[order], b_cy[order], b_part[order]
    else:
        b_node = np.zeros(0, np.int32)
        b_cx = b_cy = np.zeros(0)
        b_part = np.zeros(0, np.int32)
    types = np.array([BC_CODES[bc["left"]], BC_CODES[bc["right"]], BC_CODES[bc["bottom"]],
                      BC_CODES[bc["top"]]], np.int32)
    la = np.tile(np.arange(p1), p1)  # local a of local index l
    lb = np.repeat(np.arange(p1), p1)
    X = (x0 + (ex[:, None] + xi[la][None, :]) * hx).reshape(-1)
    Y = (y0 + (ey[:, None] + xi[lb][None, :]) * hy).reshape(-1)
    x = np.stack([X, Y])
    return Problem(dim=2, degree=k, n=n, n_loc=nl, row_ptr=row_ptr, col_idx=col_c.astype(np.int32),
                   cij=np.stack([cx_c, cy_c]), coloc=co_c.astype(np.uint8), mi=mi, MK=MK,
                   b_node=b_node, b_c=np.stack([b_cx, b_cy]),
                   b_type=types[b_part] if len(b_part) else np.zeros(0, np.int32), b_part=b_part,
                   omega_measure=float((x1 - x0) * (y1 - y0)), x=x, b_x=x[:, b_node])


def assemble_3d(nx: int, ny: int, nz: int, degree: int, box=(0.0, 1.0, 0.0, 1.0, 0.0, 1.0),
                periodic=(False, False, False), bc=None) -> Problem:
    """Q^k dG on an nx x ny x nz uniform hexahedral mesh of box = (x0, x1, y0, y1, z0, z1), the
    three-dimensional counterpart of assemble_2d.

    bc maps 'left'/'right' (x), 'bottom'/'top' (y) and 'front'/'back' (z) to 'slip', 'dirichlet' or
    'inoutflow' (sides that are not periodic)."""
    k = degree
    p1 = k + 1
    nl = p1 ** 3
    x0, x1, y0, y1, z0, z1 = box
    h = np.array([(x1 - x0) / nx, (y1 - y0) / ny, (z1 - z0) / nz])
    ns = (nx, ny, nz)
    bc = {**dict(left="slip", right="slip", bottom="slip", top="slip", front="slip", back="slip"), **(bc or {})}
    xi, wi = gauss_lobatto(k)
    Q = sbp_matrix(xi, wi)
    Mr = ref_mass(xi)
    E = nx * ny * nz
    n = E * nl
    e = np.arange(E, dtype=np.int64)
    eidx = (e % nx, (e // nx) % ny, e // (nx * ny))
    maxr = nl - 1 + 3
    col = np.zeros((E, nl, maxr), np.int64)
    cc = np.zeros((3, E, nl, maxr))
    co = np.zeros((E, nl, maxr), np.uint8)
    valid = np.zeros((E, nl, maxr), bool)
    bnodes, bcs, bparts = [], [], []

    def loc(a, b, c):
        return (c * p1 + b) * p1 + a

    parts = ((PART_LEFT, PART_RIGHT), (PART_BOTTOM, PART_TOP), (PART_FRONT, PART_BACK))
    for c in range(p1):
        for b in range(p1):
            for a in range(p1):
                ijk = (a, b, c)
                l = loc(a, b, c)
                s = 0
                for ax in range(3):  # the line of l along axis ax: c = Q[ijk_ax, t] times the other weights
                    o1, o2 = [d for d in range(3) if d != ax]
                    wt = wi[ijk[o1]] * wi[ijk[o2]] * h[o1] * h[o2]
                    for t in range(p1):
                        if t == ijk[ax]:
                            continue
                        q = list(ijk)
                        q[ax] = t
                        col[:, l, s] = e * nl + loc(*q)
                        cc[ax, :, l, s] = wt * Q[ijk[ax], t]
                        valid[:, l, s] = True
                        s += 1
                for ax in range(3):  # face partners (collocated); sides of the domain become boundary entries
                    if ijk[ax] not in (0, k):
                        continue
                    lo = ijk[ax] == 0
                    o1, o2 = [d for d in range(3) if d != ax]
                    val = 0.5 * wi[ijk[o1]] * wi[ijk[o2]] * h[o1] * h[o2] * (-1.0 if lo else 1.0)
                    nidx = [eidx[0].copy(), eidx[1].copy(), eidx[2].copy()]
                    nidx[ax] = nidx[ax] - 1 if lo else nidx[ax] + 1
                    if periodic[ax]:
                        nidx[ax] = nidx[ax] % ns[ax]
                    inside = (nidx[ax] >= 0) & (nidx[ax] < ns[ax])
                    ne = (nidx[2] * ny + nidx[1]) * nx + nidx[0]
                    q = list(ijk)
                    q[ax] = k if lo else 0
                    col[inside, l, s] = ne[inside] * nl + loc(*q)
                    cc[ax, inside, l, s] = val
                    co[inside, l, s] = 1
                    valid[inside, l, s] = True
                    s += 1
                    bnd = ~inside
                    if bnd.any():
                        cnt = int(bnd.sum())
                        bnodes.append(e[bnd] * nl + l)
                        bv = np.zeros((3, cnt))
                        bv[ax] = val
                        bcs.append(bv)
                        bparts.append(np.full(cnt, parts[ax][0 if lo else 1]))
                for cz in range(p1):  # mass-only entries (c_ij = 0): on none of the three lines of l
                    for by in range(p1):
                        for ax_ in range(p1):
                            if sum((ax_ != a, by != b, cz != c)) >= 2:
                                col[:, l, s] = e * nl + loc(ax_, by, cz)
                                valid[:, l, s] = True
                                s += 1
    counts = valid.reshape(n, maxr).sum(1)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col_c, cx_c, cy_c, cz_c, co_c = _compress(valid, col, cc[0], cc[1], cc[2], co)
    wloc = np.einsum("c,b,a->cba", wi, wi, wi).reshape(-1)  # index (c*p1 + b)*p1 + a
    vol = h.prod()
    mi = np.tile(wloc * vol, E)
    MK = np.broadcast_to(np.kron(np.kron(Mr, Mr), Mr) * vol, (E, nl, nl)).copy()
    if bnodes:
        b_node = np.concatenate(bnodes).astype(np.int32)
        b_c = np.concatenate(bcs, axis=1)
        b_part = np.concatenate(bparts).astype(np.int32)
        order = np.lexsort((b_part, b_node))
        b_node, b_c, b_part = b_node[order], b_c[:, order], b_part[order]
    else:
        b_node = np.zeros(0, np.int32)
        b_c = np.zeros((3, 0))
        b_part = np.zeros(0, np.int32)
    types = np.array([BC_CODES[bc[sd]] for sd in ("left", "right", "bottom", "top", "front", "back")], np.int32)
    la = np.tile(np.arange(p1), p1 * p1)
    lb = np.tile(np.repeat(np.arange(p1), p1), p1)
    lc = np.repeat(np.arange(p1), p1 * p1)
    X = (x0 + (eidx[0][:, None] + xi[la][None, :]) * h[0]).reshape(-1)
    Y = (y0 + (eidx[1][:, None] + xi[lb][None, :]) * h[1]).reshape(-1)
    Z = (z0 + (eidx[2][:, None] + xi[lc][None, :]) * h[2]).reshape(-1)
    x = np.stack([X, Y, Z])
    return Problem(dim=3, degree=k, n=n, n_loc=nl, row_ptr=row_ptr, col_idx=col_c.astype(np.int32),
                   cij=np.stack([cx_c, cy_c, cz_c]), coloc=co_c.astype(np.uint8), mi=mi, MK=MK,
                   b_node=b_node, b_c=b_c, b_type=types[b_part] if len(b_part) else np.zeros(0, np.int32),
                   b_part=b_part, omega_measure=float((x1 - x0) * (y1 - y0) * (z1 - z0)), x=x,
                   b_x=x[:, b_node])

