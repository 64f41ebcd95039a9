"""ctypes wrapper of the oracle (oracle.c): plain FP64 CPU stage of the graph-based dG scheme.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm
use it to check and time the CUDA library; the library never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
LIB_OMP = os.path.join(BUILD, "liboracle_omp.so")  # the same source with its row loops shared by OpenMP

LOW, HIGH, LIMITED = 0, 1, 2
F_INADMISSIBLE, F_CFL = 1, 2


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile oracle.c with gcc (-O2, no FP contraction, so the C arithmetic is evaluated as written).
    openmp=True builds the multi-core variant used only to time the CPU baseline: the same loops with their
    rows shared among threads, bit-identical results."""
    src = os.path.join(HERE, "oracle.c")
    lib_path = LIB_OMP if openmp else LIB
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(HERE, "oracle.h"))):
        return lib_path
    os.makedirs(BUILD, exist_ok=True)
    tmp = lib_path + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", *(["-fopenmp"] if openmp else []),
                           "-fPIC", "-shared", src, "-o", tmp, "-lm"])
    os.replace(tmp, lib_path)
    return lib_path


class _Problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("degree", C.c_int), ("n_loc", C.c_int),
                ("n", C.c_long), ("nnz", C.c_long), ("nb", C.c_long),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("cij", C.c_void_p),
                ("coloc", C.c_void_p), ("mi", C.c_void_p), ("MK", C.c_void_p),
                ("b_node", C.c_void_p), ("b_c", C.c_void_p), ("b_type", C.c_void_p),
                ("gamma", C.c_double), ("omega", C.c_double),
                ("order", C.c_int), ("limiter_passes", C.c_int), ("bounds_mode", C.c_int),
                ("c_k", C.c_double), ("p_k", C.c_double), ("c_ev", C.c_double),
                ("c_r", C.c_double), ("p_r", C.c_double),
                ("ls_tol", C.c_double), ("ls_maxit", C.c_int), ("relax_measure", C.c_int)]


_TRACE_FIELDS = ["dL", "dB", "dii", "UB", "ubar", "ubarB", "UL", "N", "dH", "dBH", "UH", "A", "AB",
                 "rho_min", "rho_max", "s_min", "l1", "l1B", "l2", "l2B", "U1"]


class _Trace(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in _TRACE_FIELDS]


_libs = {}


def lib(openmp: bool = False):
    L = _libs.get(openmp)
    if L is None:
        L = C.CDLL(build(openmp=openmp))
        L.orc_threads.restype = C.c_int
        L.orc_inoutflow_state.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_void_p]
        L.orc_line_search.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_int,
                                      C.c_double, C.c_double, C.c_int]
        L.orc_line_search.restype = C.c_double
        L.orc_lambda_max_batch.argtypes = [C.c_long, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                           C.c_void_p]
        L.orc_max_dt.argtypes = [C.POINTER(_Problem), C.c_void_p, C.c_void_p, C.c_double,
                                 C.POINTER(C.c_double)]
        L.orc_max_dt.restype = C.c_int
        L.orc_stage.argtypes = [C.POINTER(_Problem), C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                                C.c_void_p, C.c_void_p, C.POINTER(_Trace)]
        L.orc_stage.restype = C.c_int
        _libs[openmp] = L
    return L


def threads(openmp: bool = False) -> int:
    """Threads the stage's row loops use in that build (1 without OpenMP)."""
    return lib(openmp).orc_threads()


def default_params(degree: int) -> dict:
    """Parameters of the paper: c_k = 1, p_k = 1/2 (k even) or 0 (k odd) (Sec. 5.1); c_ev = 1, 0.5, 0.25
    for k = 1, 2, 3 (Sec. 5.2); c_r = 4, p_r = 1.5 (Sec. 5.4, eq. (ViscMinConst2)); two limiter passes
    (Sec. 6.1)."""
    return dict(order=LIMITED, limiter_passes=2, bounds_mode=0, c_k=1.0,
                p_k=0.5 if degree % 2 == 0 else 0.0,
                c_ev={1: 1.0, 2: 0.5}.get(degree, 0.25), c_r=4.0, p_r=1.5, ls_tol=1e-14, ls_maxit=50,
                relax_measure=0)


def _p(a):
    return a.ctypes.data if a is not None and a.size else None


@dataclass
class Oracle:
    """Holds one problem (arrays from paper_2402_04514_gb300.assembly.Problem or equivalent)."""

    problem: object
    gamma: float = 1.4
    params: dict = None
    openmp: bool = False  # the multi-core timing build (same results)

    def __post_init__(self):
        P = self.problem
        if not (1 <= P.dim <= 3 and 1 <= P.n_loc <= 32):
            raise ValueError("the oracle takes dim 1..3 and at most 32 nodes per element")
        self.params = {**default_params(P.degree), **(self.params or {})}
        self._keep = dict(
            row_ptr=np.ascontiguousarray(P.row_ptr, np.int64),
            col_idx=np.ascontiguousarray(P.col_idx, np.int32),
            cij=np.ascontiguousarray(P.cij, np.float64),
            coloc=np.ascontiguousarray(P.coloc, np.uint8),
            mi=np.ascontiguousarray(P.mi, np.float64),
            MK=np.ascontiguousarray(P.MK, np.float64),
            b_node=np.ascontiguousarray(P.b_node, np.int32),
            b_c=np.ascontiguousarray(P.b_c, np.float64),
            b_type=np.ascontiguousarray(P.b_type, np.int32))
        k = self._keep
        self.n, self.nnz, self.nb, self.m = int(P.n), int(k["col_idx"].size), int(k["b_node"].size), P.dim + 2
        pr = self.params
        self._c = _Problem(P.dim, P.degree, P.n_loc, self.n, self.nnz, self.nb,
                           _p(k["row_ptr"]), _p(k["col_idx"]), _p(k["cij"]), _p(k["coloc"]), _p(k["mi"]),
                           _p(k["MK"]), _p(k["b_node"]), _p(k["b_c"]), _p(k["b_type"]),
                           self.gamma, P.omega_measure, pr["order"], pr["limiter_passes"],
                           pr["bounds_mode"], pr["c_k"], pr["p_k"], pr["c_ev"], pr["c_r"], pr["p_r"],
                           pr["ls_tol"], pr["ls_maxit"], pr["relax_measure"])

    def set(self, **kw):
        for key, val in kw.items():
            self.params[key] = val
            setattr(self._c, key, val)

    def _bdata(self, bdata):
        if bdata is None:
            return None
        return np.ascontiguousarray(bdata, np.float64).reshape(self.m, self.nb)

    def max_dt(self, U, cfl, bdata=None) -> float:
        U = np.ascontiguousarray(U, np.float64)
        bd = self._bdata(bdata)
        tau = C.c_double()
        lib(self.openmp).orc_max_dt(C.byref(self._c), _p(U), _p(bd), cfl, C.byref(tau))
        return tau.value

    def stage(self, U_in, tau, U_base=None, alpha=0.0, bdata=None, trace=False):
        """Returns (U_out, flags[, trace dict])."""
        U_in = np.ascontiguousarray(U_in, np.float64)
        out = np.empty_like(U_in)
        ub = None if U_base is None else np.ascontiguousarray(U_base, np.float64)
        bd = self._bdata(bdata)
        tr = None
        arrays = {}
        if trace:
            m, n, nnz, nb = self.m, self.n, self.nnz, self.nb
            shapes = dict(dL=(nnz,), dB=(nb,), dii=(n,), UB=(m, nb), ubar=(m, nnz), ubarB=(m, nb), UL=(m, n),
                          N=(n,), dH=(nnz,), dBH=(nb,), UH=(m, n), A=(m, nnz), AB=(m, nb), rho_min=(n,),
                          rho_max=(n,), s_min=(n,), l1=(nnz,), l1B=(nb,), l2=(nnz,), l2B=(nb,), U1=(m, n))
            arrays = {f: np.zeros(shapes[f]) for f in _TRACE_FIELDS}
            tr = _Trace(*[_p(arrays[f]) for f in _TRACE_FIELDS])
        flags = lib(self.openmp).orc_stage(C.byref(self._c), _p(U_in), _p(ub), alpha, tau, _p(bd), _p(out),
                                C.byref(tr) if tr is not None else None)
        if trace:
            return out, flags, arrays
        return out, flags

    def ssprk54_step(self, U, dt, bdata_fn=None, t=0.0):
        """One SSPRK(5,4) step (oracle/ssprk.py) of size dt built from this oracle's limited forward-Euler
        stages; bdata_fn(t) gives Dirichlet data at a stage time."""
        from . import ssprk

        bd = (lambda s: None) if bdata_fn is None else bdata_fn
        U1, flags = ssprk.shu_osher_step(U, dt, lambda u, tau, ts: self.stage(u, tau, bdata=bd(ts)),
                                         ssprk.SSPRK54_ALPHA, ssprk.SSPRK54_BETA, t)
        f = 0
        for x in flags:
            f |= x
        return U1, f

    def ssprk3_step(self, U, tau, bdata_fn=None, t=0.0):
        """One Shu-Osher SSPRK3 step; bdata_fn(t) gives Dirichlet data [m][nb] at a stage time."""
        bd = (lambda s: None) if bdata_fn is None else bdata_fn
        flags = 0
        U1, f = self.stage(U, tau, bdata=bd(t)); flags |= f
        U2, f = self.stage(U1, tau, U_base=U, alpha=0.75, bdata=bd(t + tau)); flags |= f
        U3, f = self.stage(U2, tau, U_base=U, alpha=1.0 / 3.0, bdata=bd(t + 0.5 * tau)); flags |= f
        return U3, flags


def line_search(U0, Pv, rmin, rmax, smin, gamma=1.4, tol=1e-14, maxit=50):
    """The limiter's line search (orc_line_search) for one state U0 [m] and direction Pv [m]."""
    U0 = np.ascontiguousarray(U0, np.float64)
    Pv = np.ascontiguousarray(Pv, np.float64)
    return lib().orc_line_search(_p(U0), _p(Pv), rmin, rmax, smin, U0.shape[0] - 2, gamma, tol, maxit)


def inoutflow_state(Ui, Ud, nrm, gamma=1.4):
    """Boundary state of an in/outflow entry (orc_inoutflow_state) for one interior state Ui [m], data Ud
    [m] and outward unit normal nrm [d]."""
    Ui = np.ascontiguousarray(Ui, np.float64)
    Ud = np.ascontiguousarray(Ud, np.float64)
    nrm = np.ascontiguousarray(nrm, np.float64)
    out = np.empty_like(Ui)
    lib().orc_inoutflow_state(_p(Ui), _p(Ud), _p(nrm), nrm.shape[0], gamma, _p(out))
    return out


def lambda_max(UL, UR, nrm, gamma=1.4):
    """Vectorised lambda_max^+: UL, UR [count][m], nrm [count][d]."""
    UL = np.ascontiguousarray(UL, np.float64)
    UR = np.ascontiguousarray(UR, np.float64)
    nrm = np.ascontiguousarray(nrm, np.float64)
    out = np.empty(UL.shape[0])
    lib().orc_lambda_max_batch(UL.shape[0], _p(UL), _p(UR), _p(nrm), nrm.shape[1], gamma, _p(out))
    return out
