"""Python binding of the gdg C ABI (include/gdg.h): argument marshalling only.

Every computation of a stage runs in the CUDA kernels of libgdg.so; PyTorch provides device memory and
streams.  There is no CPU fallback: if the library is missing or the GPU is absent, construction fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

ORDER_LOW, ORDER_HIGH, ORDER_LIMITED = 0, 1, 2
KERNELS = ("prim", "maxdt", "low", "high", "limit2", "final", "edge", "lsfix", "tau", "clock", "axpy")  # GDG_K_*
BC_SLIP, BC_DIRICHLET, BC_INOUTFLOW = 0, 1, 2
FLAG_INADMISSIBLE, FLAG_CFL = 1, 2
PRECISION_FP64, PRECISION_MIXED = 0, 1
RELAX_NODE, RELAX_ELEMENT = 0, 1

_CODES = {0: "GDG_OK", 1: "GDG_EINVAL", 2: "GDG_ENOMEM", 3: "GDG_ECUDA", 4: "GDG_ESETUP", 5: "GDG_EADMISSIBLE",
          6: "GDG_ECFL", 7: "GDG_ETIMEOUT", 8: "GDG_ENOTSUP"}


class GdgError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {_CODES.get(code, code)}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("order", C.c_int32), ("limiter_passes", C.c_int32), ("bounds_mode", C.c_int32),
                ("c_k", C.c_double), ("p_k", C.c_double), ("c_ev", C.c_double), ("c_r", C.c_double),
                ("p_r", C.c_double), ("ls_tol", C.c_double), ("ls_maxit", C.c_int32), ("precision", C.c_int32),
                ("relax_measure", C.c_int32)]


class _Problem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("degree", C.c_int32), ("n_loc", C.c_int32),
                ("n", C.c_int64), ("nnz", C.c_int64), ("nb", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("cij", C.c_void_p), ("coloc", C.c_void_p),
                ("mi", C.c_void_p), ("MK", C.c_void_p), ("b_node", C.c_void_p), ("b_c", C.c_void_p),
                ("b_type", C.c_void_p), ("gamma", C.c_double), ("omega_measure", C.c_double),
                ("params", Params)]


class DevMesh(C.Structure):
    """gdg_dev_mesh: a mesh held in caller-owned device arrays (for gdg_max_dt_noalloc)."""

    _fields_ = [("dim", C.c_int32), ("n", C.c_int64), ("nnz", C.c_int64), ("nb", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("cij", C.c_void_p), ("mi", C.c_void_p),
                ("b_ptr", C.c_void_p), ("b_c", C.c_void_p), ("b_type", C.c_void_p), ("gamma", C.c_double)]


class _Info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("nb", C.c_int64), ("dim", C.c_int32), ("n_loc", C.c_int32),
                ("device_bytes", C.c_int64)]


class Schedule(C.Structure):
    """gdg_schedule: launch shapes (threads per block of the row kernels, element block cap, deferred
    line-search slots per thread, row order of the kernels with per-entry loops)."""

    _fields_ = [("prim_threads", C.c_int32), ("edge_threads", C.c_int32), ("tau_threads", C.c_int32),
                ("low_threads", C.c_int32), ("limit2_threads", C.c_int32), ("final_threads", C.c_int32),
                ("maxdt_threads", C.c_int32), ("high_block_cap", C.c_int32), ("lsfix_slots", C.c_int32),
                ("row_slices", C.c_int32)]


class RequestInfo(C.Structure):
    _fields_ = [("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double), ("t_final", C.c_double),
                ("steps", C.c_int64), ("status", C.c_int32), ("flags", C.c_int32), ("device_bytes", C.c_int64)]


class ServerInfo(C.Structure):
    _fields_ = [("queued", C.c_int64), ("active", C.c_int64), ("bytes_in_use", C.c_int64), ("budget", C.c_int64),
                ("iterations", C.c_int64), ("now", C.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libgdg.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libgdg.so not built ({path}); run __graft_entry__.build() or "
                               "python -m paper_2402_04514_gb300.build")
        _build.build()
    L = C.CDLL(path)
    vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    L.gdg_default_params.argtypes = [i32, C.POINTER(Params)]
    L.gdg_setup.argtypes = [C.POINTER(_Problem), C.POINTER(vp)]
    L.gdg_set_params.argtypes = [vp, C.POINTER(Params)]
    L.gdg_max_dt.argtypes = [vp, vp, vp, d, C.POINTER(d), vp]
    L.gdg_stage.argtypes = [vp, vp, vp, d, d, vp, vp, vp]
    L.gdg_ssprk3_step.argtypes = [vp, vp, vp, vp, vp, vp]
    L.gdg_ssprk54_step.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.gdg_ssprk3_step_host.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    L.gdg_batch_create.argtypes = [C.POINTER(vp), i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                   C.POINTER(vp)]
    L.gdg_batch_step.argtypes = [vp, vp]
    L.gdg_batch_set_persistent.argtypes = [vp, i32]
    L.gdg_batch_profile.argtypes = [vp, i32]
    L.gdg_batch_profile_read.argtypes = [vp, vp, vp]
    L.gdg_batch_destroy.argtypes = [vp]
    L.gdg_footprint.argtypes = [C.POINTER(_Problem), C.POINTER(i64)]
    L.gdg_autotune.argtypes = [vp, vp, vp, vp, vp, i32, vp]
    L.gdg_get_schedule.argtypes = [vp, C.POINTER(Schedule)]
    L.gdg_set_schedule.argtypes = [vp, C.POINTER(Schedule)]
    L.gdg_batch_autotune.argtypes = [vp, i32, vp]
    L.gdg_batch_get_schedule.argtypes = [vp, C.POINTER(Schedule)]
    L.gdg_batch_set_schedule.argtypes = [vp, C.POINTER(Schedule)]
    L.gdg_server_create.argtypes = [i64, C.POINTER(vp)]
    L.gdg_server_submit.argtypes = [vp, C.POINTER(_Problem), vp, vp, d, d, C.POINTER(i64)]
    L.gdg_server_wait.argtypes = [vp, i64, d, vp, C.POINTER(RequestInfo)]
    L.gdg_server_stats.argtypes = [vp, C.POINTER(ServerInfo)]
    L.gdg_server_destroy.argtypes = [vp]
    L.gdg_clock_set.argtypes = [vp, d, d, d, vp]
    L.gdg_clock_get.argtypes = [vp, C.POINTER(d), C.POINTER(d), C.POINTER(i64), vp]
    L.gdg_status.argtypes = [vp, C.POINTER(i32), i32, vp]
    L.gdg_debug_export.argtypes = [vp, C.c_char_p, vp, i64, vp]
    L.gdg_get_info.argtypes = [vp, C.POINTER(_Info)]
    L.gdg_profile.argtypes = [vp, i32]
    L.gdg_math_selftest.argtypes = [i32, i32, vp, vp, i64, vp]
    L.gdg_wave_speed_check.argtypes = [d, vp, vp, i64, vp]
    L.gdg_certificate_check.argtypes = [i32, d, vp, vp, i64, vp]
    L.gdg_fp64_throughput.argtypes = [i32, C.POINTER(d), vp]
    L.gdg_max_dt_noalloc.argtypes = [C.POINTER(DevMesh), vp, vp, d, vp, vp]
    L.gdg_profile_read.argtypes = [vp, vp, vp]
    L.gdg_destroy.argtypes = [vp]
    L.gdg_error_string.argtypes = [C.c_int]
    L.gdg_error_string.restype = C.c_char_p
    for f in ("gdg_setup", "gdg_set_params", "gdg_max_dt", "gdg_stage", "gdg_ssprk3_step", "gdg_ssprk54_step",
              "gdg_ssprk3_step_host",
              "gdg_clock_set",
              "gdg_clock_get", "gdg_batch_create", "gdg_batch_step", "gdg_batch_set_persistent", "gdg_batch_profile", "gdg_batch_profile_read",
              "gdg_footprint", "gdg_server_create", "gdg_server_submit", "gdg_server_wait", "gdg_server_stats",
              "gdg_autotune", "gdg_get_schedule", "gdg_set_schedule", "gdg_batch_autotune", "gdg_batch_get_schedule",
              "gdg_batch_set_schedule",
              "gdg_status", "gdg_debug_export",
              "gdg_get_info", "gdg_profile", "gdg_profile_read", "gdg_math_selftest", "gdg_fp64_throughput",
              "gdg_max_dt_noalloc", "gdg_wave_speed_check", "gdg_certificate_check"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _check(code, what):
    if code != 0:
        raise GdgError(code, what)


def default_params(degree: int) -> dict:
    p = Params()
    load().gdg_default_params(degree, C.byref(p))
    return {f: getattr(p, f) for f, _ in Params._fields_}


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def math_selftest(fn: int, q: int, x, stream=None):
    """Runs gdg_math_selftest on the device tensor x (float64) and returns the result tensor (for the
    binary functions 7..10, x holds pairs and the result has half its length)."""
    import torch

    n = x.numel() // 2 if fn >= 7 else x.numel()
    y = torch.empty(n, dtype=x.dtype, device=x.device)
    _check(load().gdg_math_selftest(fn, q, _ptr(x), _ptr(y), n, _stream(stream)), "gdg_math_selftest")
    return y


def wave_speed_check(gamma: float, states, stream=None):
    """gdg_wave_speed_check on the device tensor states [n, 6] (float64): returns [n, 4] with the FP64
    bound, the mixed-precision bound, the same without its margin, and the margin's scale."""
    import torch

    out = torch.empty((states.shape[0], 4), dtype=torch.float64, device=states.device)
    _check(load().gdg_wave_speed_check(gamma, _ptr(states), _ptr(out), states.shape[0], _stream(stream)),
           "gdg_wave_speed_check")
    return out


def certificate_check(dim: int, gamma: float, rows, stream=None):
    """gdg_certificate_check on the device tensor rows [n, 2m + 2] (float64): returns [n, 2] with 1/0
    (certified) and psi(s) in FP64."""
    import torch

    out = torch.empty((rows.shape[0], 2), dtype=torch.float64, device=rows.device)
    _check(load().gdg_certificate_check(dim, gamma, _ptr(rows), _ptr(out), rows.shape[0], _stream(stream)),
           "gdg_certificate_check")
    return out


def max_dt_noalloc(mesh: DevMesh, U, cfl: float, tau_out, bdata=None, stream=None) -> int:
    """gdg_max_dt_noalloc: writes tau into the device tensor tau_out (one float64) without allocating;
    returns the status code (0 on success)."""
    return load().gdg_max_dt_noalloc(C.byref(mesh), _ptr(U), _ptr(bdata), cfl, _ptr(tau_out), _stream(stream))


RATE_OPS = ("dfma", "ddiv", "dsqrt", "dpow", "ffma", "rcp64", "rootinv5", "f2f_pair", "dmul", "int_mul",
            "dmul_half_int", "dadd", "int_add", "dadd_quarter_int")


def fp64_throughput(stream=None) -> dict:
    """{operation: operations per second} measured on the current GPU (gdg_fp64_throughput)."""
    out = {}
    for i, name in enumerate(RATE_OPS):
        v = C.c_double()
        _check(load().gdg_fp64_throughput(i, C.byref(v), _stream(stream)), "gdg_fp64_throughput")
        out[name] = v.value
    return out


def _problem_struct(P, gamma, params):
    """gdg_problem for an assembled problem; returns it with the arrays it points into (keep them alive)."""
    prm = {**default_params(P.degree), **(params or {})}
    keep = dict(row_ptr=np.ascontiguousarray(P.row_ptr, np.int64), col_idx=np.ascontiguousarray(P.col_idx, np.int32),
                cij=np.ascontiguousarray(P.cij, np.float64), coloc=np.ascontiguousarray(P.coloc, np.uint8),
                mi=np.ascontiguousarray(P.mi, np.float64), MK=np.ascontiguousarray(P.MK, np.float64),
                b_node=np.ascontiguousarray(P.b_node, np.int32), b_c=np.ascontiguousarray(P.b_c, np.float64),
                b_type=np.ascontiguousarray(P.b_type, np.int32))

    def hp(a):
        return a.ctypes.data if a.size else None

    cp = _Problem(P.dim, P.degree, P.n_loc, int(P.n), int(P.col_idx.shape[0]), int(P.b_node.shape[0]),
                  hp(keep["row_ptr"]), hp(keep["col_idx"]), hp(keep["cij"]), hp(keep["coloc"]), hp(keep["mi"]),
                  hp(keep["MK"]), hp(keep["b_node"]), hp(keep["b_c"]), hp(keep["b_type"]), gamma, P.omega_measure,
                  Params(**prm))
    return cp, keep


def footprint(problem, gamma: float = 1.4, params: dict | None = None) -> int:
    """gdg_footprint: device bytes gdg_setup would allocate for the problem."""
    cp, keep = _problem_struct(problem, gamma, params)
    b = C.c_int64()
    _check(load().gdg_footprint(C.byref(cp), C.byref(b)), "gdg_footprint")
    return b.value


class Solver:
    """One mesh instance on the current CUDA device (a gdg handle)."""

    def __init__(self, problem, gamma: float = 1.4, params: dict | None = None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("gdg needs a CUDA device; there is no CPU fallback")
        L = load()
        P = problem
        self.dim, self.m, self.n = P.dim, P.dim + 2, int(P.n)
        self.nb = int(P.b_node.shape[0])
        self.nnz = int(P.col_idx.shape[0])
        self.gamma = gamma
        self.has_dirichlet = bool((np.asarray(P.b_type) != BC_SLIP).any())  # Dirichlet or in/outflow data
        cp, keep = _problem_struct(P, gamma, params)
        self._params = cp.params
        h = C.c_void_p()
        _check(L.gdg_setup(C.byref(cp), C.byref(h)), "gdg_setup")
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())

    @property
    def params(self) -> dict:
        return {f: getattr(self._params, f) for f, _ in Params._fields_}

    def set_params(self, **kw):
        p = Params(**{**self.params, **kw})
        _check(load().gdg_set_params(self._h, C.byref(p)), "gdg_set_params")
        self._params = p

    def _bdata(self, bdata):
        if bdata is None:
            if self.has_dirichlet:
                raise ValueError("Dirichlet boundary entries need bdata")
            return None
        assert bdata.is_cuda and bdata.dtype.itemsize == 8 and bdata.is_contiguous()
        assert tuple(bdata.shape) == (self.m, self.nb)
        return bdata

    def _check_state(self, U):
        assert U.is_cuda and U.is_contiguous() and tuple(U.shape) == (self.m, self.n), U.shape
        import torch
        assert U.dtype == torch.float64

    def max_dt(self, U, cfl: float, bdata=None, stream=None) -> float:
        self._check_state(U)
        bd = self._bdata(bdata)
        tau = C.c_double()
        _check(load().gdg_max_dt(self._h, _ptr(U), _ptr(bd), cfl, C.byref(tau), _stream(stream)), "gdg_max_dt")
        return tau.value

    def stage(self, U_in, tau: float, U_base=None, alpha: float = 0.0, bdata=None, out=None, stream=None):
        import torch

        self._check_state(U_in)
        if out is None:
            out = torch.empty_like(U_in)
        self._check_state(out)
        if U_base is not None:
            self._check_state(U_base)
        bd = self._bdata(bdata)
        _check(load().gdg_stage(self._h, _ptr(U_in), _ptr(U_base), alpha, tau, _ptr(bd), _ptr(out),
                                _stream(stream)), "gdg_stage")
        return out

    def status(self, clear: bool = False, stream=None) -> int:
        f = C.c_int32()
        _check(load().gdg_status(self._h, C.byref(f), 1 if clear else 0, _stream(stream)), "gdg_status")
        return f.value

    def export(self, name: str, stream=None) -> np.ndarray:
        m, n, nnz, nb = self.m, self.n, self.nnz, self.nb
        shapes = dict(dL=(nnz,), dB=(nb,), N=(n,), UL=(m, n), U1=(m, n), A=(m, nnz), rho_min=(n,), rho_max=(n,),
                      s_min=(n,), l1=(nnz,), l2=(nnz,), ls_deferred=(2,))
        out = np.empty(shapes[name])
        _check(load().gdg_debug_export(self._h, name.encode(), out.ctypes.data if out.size else None, out.size,
                                       _stream(stream)), f"gdg_debug_export({name})")
        return out

    def profile(self, enable: bool):
        """Bracket every kernel launch with CUDA events (on the launching stream) until disabled."""
        _check(load().gdg_profile(self._h, 1 if enable else 0), "gdg_profile")

    def profile_read(self) -> dict:
        """{kernel: (total_ms, launches)} accumulated since the last read; synchronises."""
        ms = np.zeros(len(KERNELS))
        cnt = np.zeros(len(KERNELS), np.int64)
        _check(load().gdg_profile_read(self._h, ms.ctypes.data, cnt.ctypes.data), "gdg_profile_read")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNELS)}

    def info(self) -> dict:
        i = _Info()
        _check(load().gdg_get_info(self._h, C.byref(i)), "gdg_get_info")
        return {f: getattr(i, f) for f, _ in _Info._fields_}

    def ssprk3_step(self, U, tau: float, bufs, out, bdata_fn=None, t: float = 0.0, stream=None):
        """Shu-Osher SSPRK3 step from U into out, with two scratch states bufs = (U1, U2).
        bdata_fn(time) returns the Dirichlet data (device [m][nb]) at a stage time."""
        bd = (lambda s: None) if bdata_fn is None else bdata_fn
        U1, U2 = bufs
        self.stage(U, tau, bdata=bd(t), out=U1, stream=stream)
        self.stage(U1, tau, U_base=U, alpha=0.75, bdata=bd(t + tau), out=U2, stream=stream)
        self.stage(U2, tau, U_base=U, alpha=1.0 / 3.0, bdata=bd(t + 0.5 * tau), out=out, stream=stream)
        return out

    def step(self, U, work, bdata=None, stream=None):
        """One fused step of U in place, the time step chosen on the device from the handle's clock
        (set_clock): gdg_ssprk3_step with work = (T1, T2), gdg_ssprk54_step with work = (T1, T2, T3)."""
        self._check_state(U)
        for T in work:
            self._check_state(T)
        bd = self._bdata(bdata)
        if len(work) == 2:
            _check(load().gdg_ssprk3_step(self._h, _ptr(U), _ptr(work[0]), _ptr(work[1]), _ptr(bd), _stream(stream)),
                   "gdg_ssprk3_step")
        elif len(work) == 3:
            _check(load().gdg_ssprk54_step(self._h, _ptr(U), _ptr(work[0]), _ptr(work[1]), _ptr(work[2]), _ptr(bd),
                                           _stream(stream)), "gdg_ssprk54_step")
        else:
            raise ValueError("work holds two (SSPRK3) or three (SSPRK(5,4)) scratch states")
        return U

    def _host_state(self, X, writable: bool):
        """Address of a host state [m][n] of float64: a CPU torch tensor (page-locked or not) or a numpy array."""
        if isinstance(X, np.ndarray):
            assert X.dtype == np.float64 and X.flags.c_contiguous and X.shape == (self.m, self.n), X.shape
            assert X.flags.writeable or not writable
            return C.c_void_p(X.ctypes.data)
        import torch

        assert isinstance(X, torch.Tensor) and not X.is_cuda and X.dtype == torch.float64
        assert X.is_contiguous() and tuple(X.shape) == (self.m, self.n), X.shape
        return C.c_void_p(X.data_ptr())

    def step_host(self, U_host_in, U_host_out, U, work, bdata=None, stream=None):
        """gdg_ssprk3_step_host: one fused SSP-RK3 step of a state in host memory (U_host_in -> U_host_out,
        which may be the same buffer), on the device in U and work = (T1, T2).  Asynchronous for
        page-locked buffers: synchronize the stream before reading U_host_out."""
        self._check_state(U)
        for T in work:
            self._check_state(T)
        T1, T2 = work
        bd = self._bdata(bdata)
        _check(load().gdg_ssprk3_step_host(self._h, self._host_state(U_host_in, False),
                                           self._host_state(U_host_out, True), _ptr(U), _ptr(T1), _ptr(T2),
                                           _ptr(bd), _stream(stream)), "gdg_ssprk3_step_host")
        return U_host_out

    def autotune(self, U, work, trials: int = 2, bdata=None, stream=None) -> dict:
        """gdg_autotune: picks the launch schedule by timing fused steps from U (restored afterwards)."""
        self._check_state(U)
        T1, T2 = work
        bd = self._bdata(bdata)
        _check(load().gdg_autotune(self._h, _ptr(U), _ptr(T1), _ptr(T2), _ptr(bd), trials, _stream(stream)),
               "gdg_autotune")
        return self.schedule()

    def schedule(self) -> dict:
        sc = Schedule()
        _check(load().gdg_get_schedule(self._h, C.byref(sc)), "gdg_get_schedule")
        return {f: getattr(sc, f) for f, _ in Schedule._fields_}

    def set_schedule(self, **kw):
        sc = Schedule(**{**self.schedule(), **kw})
        _check(load().gdg_set_schedule(self._h, C.byref(sc)), "gdg_set_schedule")

    def set_clock(self, t: float = 0.0, t_end: float = float("inf"), cfl: float = 0.5, stream=None):
        _check(load().gdg_clock_set(self._h, t, t_end, cfl, _stream(stream)), "gdg_clock_set")

    def clock(self, stream=None):
        """(t, tau of the last step, completed steps) of the fused step's clock; synchronises."""
        t, tau, n = C.c_double(), C.c_double(), C.c_int64()
        _check(load().gdg_clock_get(self._h, C.byref(t), C.byref(tau), C.byref(n), _stream(stream)), "gdg_clock_get")
        return t.value, tau.value, n.value

    def close(self):
        if getattr(self, "_h", None):
            load().gdg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """gdg_batch: instances (Solver objects) advanced by fused SSP-RK3 steps in shared kernel launches.
    states[k] is member k's state (updated in place), works[k] = (T1, T2) its workspace, bdatas[k] its
    Dirichlet data or None.  The solvers and tensors are kept alive by the batch."""

    def __init__(self, solvers, states, works, bdatas=None):
        n = len(solvers)
        if n == 0:
            raise ValueError("empty batch")
        bdatas = bdatas or [None] * n
        for S, U, (T1, T2), bd in zip(solvers, states, works, bdatas):
            S._check_state(U)
            S._check_state(T1)
            S._check_state(T2)
            S._bdata(bd)
        self._keep = (list(solvers), list(states), list(works), list(bdatas))
        arr = C.c_void_p * n
        h = arr(*[S._h.value for S in solvers])
        u = arr(*[U.data_ptr() for U in states])
        t1 = arr(*[w[0].data_ptr() for w in works])
        t2 = arr(*[w[1].data_ptr() for w in works])
        bd = arr(*[None if b is None else b.data_ptr() for b in bdatas])
        out = C.c_void_p()
        _check(load().gdg_batch_create(h, n, u, t1, t2, bd, C.byref(out)), "gdg_batch_create")
        self._b = out
        self.count = n

    def step(self, stream=None):
        _check(load().gdg_batch_step(self._b, _stream(stream)), "gdg_batch_step")

    def set_persistent(self, on: bool):
        """gdg_batch_set_persistent: one cooperative launch per stage instead of one launch per kernel."""
        _check(load().gdg_batch_set_persistent(self._b, 1 if on else 0), "gdg_batch_set_persistent")

    def profile(self, enable: bool):
        _check(load().gdg_batch_profile(self._b, 1 if enable else 0), "gdg_batch_profile")

    def autotune(self, trials: int = 2, stream=None) -> dict:
        """gdg_batch_autotune: picks the batch's launch schedule by timing steps (states restored)."""
        _check(load().gdg_batch_autotune(self._b, trials, _stream(stream)), "gdg_batch_autotune")
        return self.schedule()

    def schedule(self) -> dict:
        sc = Schedule()
        _check(load().gdg_batch_get_schedule(self._b, C.byref(sc)), "gdg_batch_get_schedule")
        return {f: getattr(sc, f) for f, _ in Schedule._fields_}

    def set_schedule(self, **kw):
        sc = Schedule(**{**self.schedule(), **kw})
        _check(load().gdg_batch_set_schedule(self._b, C.byref(sc)), "gdg_batch_set_schedule")

    def profile_read(self) -> dict:
        ms = np.zeros(len(KERNELS))
        cnt = np.zeros(len(KERNELS), np.int64)
        _check(load().gdg_batch_profile_read(self._b, ms.ctypes.data, cnt.ctypes.data), "gdg_batch_profile_read")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNELS)}

    def close(self):
        if getattr(self, "_b", None):
            load().gdg_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """gdg_server: continuous-batching request loop on the current device.  submit() returns an id at
    once; wait(id) returns (final state, info dict).  hbm_budget <= 0: 80% of the free device memory."""

    def __init__(self, hbm_budget: int = 0):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("gdg needs a CUDA device; there is no CPU fallback")
        out = C.c_void_p()
        _check(load().gdg_server_create(int(hbm_budget), C.byref(out)), "gdg_server_create")
        self._s = out
        self._shapes = {}

    def submit(self, problem, U0, t_end: float, cfl: float = 0.5, gamma: float = 1.4, params: dict | None = None,
               bdata=None) -> int:
        cp, keep = _problem_struct(problem, gamma, params)
        U0 = np.ascontiguousarray(U0, np.float64)
        assert U0.shape == (problem.dim + 2, problem.n)
        bd = None if bdata is None else np.ascontiguousarray(bdata, np.float64)
        rid = C.c_int64()
        _check(load().gdg_server_submit(self._s, C.byref(cp), U0.ctypes.data if U0.size else None,
                                        None if bd is None else bd.ctypes.data, t_end, cfl, C.byref(rid)),
               "gdg_server_submit")
        self._shapes[rid.value] = U0.shape
        return rid.value

    def wait(self, rid: int, timeout: float = -1.0):
        out = np.empty(self._shapes[rid])
        info = RequestInfo()
        rc = load().gdg_server_wait(self._s, rid, timeout, out.ctypes.data if out.size else None, C.byref(info))
        if rc == 7:
            raise TimeoutError(f"request {rid} not done after {timeout} s")
        del self._shapes[rid]
        _check(rc, f"request {rid}")
        return out, {f: getattr(info, f) for f, _ in RequestInfo._fields_}

    def stats(self) -> dict:
        i = ServerInfo()
        _check(load().gdg_server_stats(self._s, C.byref(i)), "gdg_server_stats")
        return {f: getattr(i, f) for f, _ in ServerInfo._fields_}

    def close(self):
        if getattr(self, "_s", None):
            load().gdg_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
