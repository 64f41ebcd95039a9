"""Algorithmic work of each sweep kernel per launch: compulsory HBM bytes and FP64 operations.

Bytes: every array a kernel must read is read once and every array it writes is written once (per-entry
arrays of nnz entries, per-node arrays of n nodes); neighbour states are counted once per node, not per
entry (an ideal cache).  FP64 operations: the arithmetic of the method as the kernels state it, counted
per stencil entry (c_ij != 0), per CSR entry and per node, with add/sub/mul = 1, fused multiply-add = 2,
and division, square root and power = 1 each (the usual floating-point operation count; their cost in
hardware is several to ~100 FMA issue slots, which is why the sweep is bound by arithmetic: the FP64 pipe
and, for the products the kernels move there, the integer pipe).
The line-search counts assume no bracketing iteration (the common case); iterations add work that is
not counted, so the FP64 fraction reported is a lower bound.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

KERNELS = ("prim", "maxdt", "low", "high", "limit2", "final", "edge", "lsfix", "tau", "clock", "axpy")


@dataclass
class Counts:
    dim: int
    n: int
    nnz: int  # CSR entries
    nnz_s: int  # entries with c_ij != 0
    nb: int
    n_loc: int

    @property
    def m(self):
        return self.dim + 2

    @staticmethod
    def of(problem):
        cs = np.abs(problem.cij).sum(0) > 0
        return Counts(problem.dim, int(problem.n), int(problem.col_idx.size), int(cs.sum()), int(problem.b_node.size),
                      int(problem.n_loc))


def bytes_per_launch(c: Counts) -> dict:
    m, d, n, nnz, s, nb, nl = c.m, c.dim, c.n, c.nnz, c.nnz_s, c.nb, c.n_loc
    NPRIM = 6
    rowptr = 4 * (n + 1)
    ent_geom = nnz * (4 + 8) + s * 8 * d  # col, |c| of every entry; n_ij of stencil entries
    return dict(
        prim=8 * m * n + 8 * NPRIM * n,
        maxdt=8 * m * n + 8 * 4 * n + rowptr + ent_geom + 8 * n,
        edge=(s // 2) * (4 * 2 + 4 + 4) + s * 8 * (1 + d) + 8 * (m + 5) * n + s * 8 * (m + 3),
        low=8 * m * n + 8 * 3 * n + rowptr + nnz * (4 + 8) + s * (4 + 8 * (m + 3) + 8 * m)
        + 8 * (2 * m + 1 + 3) * n + 8 * 3 * nb,
        high=8 * m * n * 2 + 8 * n + rowptr + nnz * (4 + 8 + 8 + 8) + 8 * s * 2 + 8 * n * nl
        + 8 * 3 * n * 2 + 8 * m * n + 8 * n * 3 + 8 * (m + 1) * nnz + 8 * (m + 1) * nb,
        limit2=rowptr + nnz * (4 + 8 + 8 * m) + 8 * m * n * 2 + 8 * 3 * n + 8 * 2 * n + 8 * nnz,
        final=rowptr + nnz * (4 + 8 * 2 + 8 * m) + 8 * m * n * 3 + 8 * n,
        lsfix=0,  # the deferred line searches: a data-dependent handful of entries, not counted
        tau=rowptr + 8 * nnz + 8 * n + 8 * (m + 6) * nb,
        clock=0,
        axpy=8 * m * n * 3,
    )


def flops_per_launch(c: Counts) -> dict:
    m, d, n, nnz, s, nb, nl = c.m, c.dim, c.n, c.nnz, c.nnz_s, c.nb, c.n_loc
    lam = 28  # wave-speed bound from the per-node primitives
    vel = 2 * (2 * d) + 2  # two normal velocities
    flux = 2 * (3 * d + 2)  # f(U_i) n and f(U_j) n
    ls = 2 * m + (3 * d + 3) + 3  # U0 + l P, eps, s_min rho^gamma (one psi evaluation)
    edge_pair = vel + lam + 2 + flux + 2 + m + 4 * m + (3 * d + 3 + 2)  # per undirected stencil edge
    low_entry = 1 + 4 * m + 3  # row sums of d, G and the entropy flux
    low_node = 3 * m + 3 + 3 + 1 + 3 * d + 4 * m + 5 * m + 1
    return dict(
        edge=(s // 2) * edge_pair,
        prim=n * (1 + 3 * d + 3 + 1 + 2 + 3 + 1 + 2),
        maxdt=s * (vel + lam + 2) + n * 3 + nb * (lam + vel + 10),
        low=s * low_entry + n * low_node + nb * (vel + lam + flux + 11 * m + 10),
        high=s * (4 + 3 * m) + n * (2 * nl * m + m + 3) + nnz * (4 * m + m + ls) + nb * (3 * m + ls),
        limit2=nnz * (2 * m + 2 + m + ls) + n * 2 * m + nb * (2 * m + m + 2 + ls),
        final=nnz * (2 + 2 * m) + n * 3 * m + nb * (2 + 2 * m),
        lsfix=0,
        tau=nnz + 2 * n + nb * (lam + vel + 10),
        clock=0,
        axpy=3 * m * n,
    )


# FP64 pipe peak from unit counts and clocks: 152 SMs x 2 FP64 FMA per clock per SM x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# The sweep kernels also run binary64 products on the integer pipe (csrc/softfp64.cuh).  One such product
# issues INT_MUL_ALU_INST instructions on the ALU pipe (ncu instruction counts of a kernel doing nothing
# else; the rest go to the FMA-heavy pipe, which is not the tighter one), and the ALU pipe retires 64
# thread-instructions per clock per SM, so the integer pipes add 64 / INT_MUL_ALU_INST products (1 flop each)
# per clock per SM.  The arithmetic roof of a kernel that keeps both pipes busy is the sum of the two.
INT_MUL_ALU_INST = 33
INT_MUL_PEAK_TFLOPS = 152 * 64 / INT_MUL_ALU_INST * 2.07e9 / 1e12
ALU_PEAK_TFLOPS = FP64_PEAK_TFLOPS + INT_MUL_PEAK_TFLOPS


def library_source_digest() -> str:
    """sha256 (first 16 hex digits) of the library's CUDA sources and public header.  A DRAM-traffic figure
    taken with ncu is only valid for the sources it was taken from; bench.py reports it only while this
    digest matches the one recorded beside the figure."""
    import glob
    import hashlib
    import os

    here = os.path.dirname(os.path.abspath(__file__))
    files = sorted(glob.glob(os.path.join(here, "csrc", "*.cu")) + glob.glob(os.path.join(here, "csrc", "*.cuh")))
    files.append(os.path.join(os.path.dirname(here), "include", "gdg.h"))
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(path: str, kernel: str, n_nodes: int, precision: str = "fp64"):
    """DRAM bytes (read + write) per launch of `kernel` from an ncu summary table (lines
    `kernel nodes dram_read_bytes dram_write_bytes source_digest [precision]`, precision fp64 when absent),
    scaled from the captured mesh to `n_nodes` (every array a sweep kernel touches grows in proportion to
    the node count).  None when the table is missing, has no row for the kernel and precision, or was
    taken from other sources."""
    try:
        with open(path) as fh:
            lines = [ln.split() for ln in fh if ln.strip() and not ln.lstrip().startswith("#")]
    except OSError:
        return None
    digest = library_source_digest()
    for f in lines:
        if len(f) in (5, 6) and f[0] == kernel and f[4] == digest and (f[5] if len(f) == 6 else "fp64") == precision:
            return (float(f[2]) + float(f[3])) * n_nodes / float(f[1])
    return None
