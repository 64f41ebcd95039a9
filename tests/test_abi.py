"""The C ABI on the CPU: the library loads, exports every function include/gdg.h declares, and
gdg_setup's validation (host code, before any CUDA call) rejects data that breaks a documented
requirement.  No compute call runs here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2402_04514_gb300 import assembly, gdg
from paper_2402_04514_gb300 import build as gbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return gdg.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "gdg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gdg_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_default_params_and_error_strings(lib):
    p1, p2, p3 = gdg.default_params(1), gdg.default_params(2), gdg.default_params(3)
    assert (p1["p_k"], p2["p_k"], p1["c_ev"], p2["c_ev"], p3["c_ev"]) == (0.0, 0.5, 1.0, 0.5, 0.25)
    assert p1["c_r"] == 4.0 and p1["p_r"] == 1.5 and p1["limiter_passes"] == 2
    for code in range(9):
        assert lib.gdg_error_string(code).startswith(b"GDG_")


def _setup(lib, P, gamma=1.4, params=None, **over):
    a = dict(row_ptr=np.ascontiguousarray(P.row_ptr, np.int64), col_idx=np.ascontiguousarray(P.col_idx, np.int32),
             cij=np.ascontiguousarray(P.cij), coloc=np.ascontiguousarray(P.coloc, np.uint8),
             mi=np.ascontiguousarray(P.mi), MK=np.ascontiguousarray(P.MK),
             b_node=np.ascontiguousarray(P.b_node, np.int32), b_c=np.ascontiguousarray(P.b_c),
             b_type=np.ascontiguousarray(P.b_type, np.int32))
    a.update(over)
    prm = gdg.Params(**{**gdg.default_params(P.degree), **(params or {})})
    keys = ["row_ptr", "col_idx", "cij", "coloc", "mi", "MK", "b_node", "b_c", "b_type"]
    cp = gdg._Problem(P.dim, P.degree, P.n_loc, P.n, len(a["col_idx"]), len(a["b_node"]),
                      *[a[k].ctypes.data if a[k].size else None for k in keys], gamma, P.omega_measure, prm)
    h = C.c_void_p()
    rc = lib.gdg_setup(C.byref(cp), C.byref(h))
    if rc == 0:
        lib.gdg_destroy(h)
    return rc


def _cuda_present():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_setup_validation(lib):
    P = assembly.assemble_2d(3, 3, 2)
    ok = 0 if _cuda_present() else 3  # valid data reaches the device allocation
    assert _setup(lib, P) == ok
    c = P.cij.copy()
    c[0, 0] *= 1.0 + 1e-15
    assert _setup(lib, P, cij=c) == 4  # skew symmetry must be exact
    co = P.coloc.copy()
    co[np.argmax(co)] = 0
    assert _setup(lib, P, coloc=co) == 4  # collocation flags symmetric
    mi = P.mi.copy()
    mi[5] *= 1.001
    assert _setup(lib, P, mi=mi) == 4  # consistent mass rows sum to m_i
    MK = P.MK.copy()
    MK[0, 0, 1] += 1e-3
    assert _setup(lib, P, MK=MK) == 4  # symmetric blocks
    bn = P.b_node.copy()
    bn[0] = P.n
    assert _setup(lib, P, b_node=bn) == 4
    bc = P.b_c.copy()
    bc[:, 0] *= 2.0
    assert _setup(lib, P, b_c=bc) == 4  # partition of unity
    col = P.col_idx.copy()
    col[0] = 0  # diagonal entry
    assert _setup(lib, P, col_idx=col) == 4
    assert _setup(lib, P, gamma=1.0) == 4
    assert _setup(lib, P, params=dict(limiter_passes=3)) == 1
    # relaxation r_h^- = 1 - c_r h^{p_r} must stay positive for the limited scheme
    assert _setup(lib, P, params=dict(c_r=40.0)) == 4
    assert _setup(lib, P, params=dict(c_r=40.0, order=0)) == ok


def test_rejects_unsupported(lib):
    P = assembly.assemble_2d(2, 2, 1)
    P.dim = 4
    assert _setup(lib, P) == 8


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(gdg, "_lib", None)
    monkeypatch.setattr(gdg._build, "LIB", "/nonexistent/libgdg.so")
    with pytest.raises(RuntimeError):
        gdg.load()
