"""gdg_max_dt_noalloc, the time-step entry point for callers that may not allocate device memory (for
instance code running under CUDA-graph stream capture, or a plug-in whose host application owns all
device memory through its own pool).  It must give the same tau as the handle-based gdg_max_dt and as the
oracle's time step (Sec. 3.3, eq. (MaxCFLdt)), on two calls in a row (its fixed device scratch keeps the
previous call's contents), and refuse meshes above its size limit.  Each test sets up its own data, so the
file passes alone in a fresh process as well as after the other tests; its name puts it last in
collection order."""
import numpy as np
import pytest

from paper_2402_04514_gb300 import assembly, workloads
from tests.helpers import dirichlet_vortex_problem, four_quadrant_problem

pytestmark = pytest.mark.gpu

MAX_NODES = 4194304  # GDG_NOALLOC_MAX_NODES


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04514_gb300 import build

    build.build()
    return torch


def _dev_mesh(torch, P, gamma):
    """Device copies (allocated here, by the test) of the mesh in the layout gdg_dev_mesh documents:
    boundary entries ordered by node with a per-node pointer array."""
    from paper_2402_04514_gb300.gdg import DevMesh

    # the structural rules the entry point trusts (the ones gdg_setup checks), checked here on the host
    rows = np.repeat(np.arange(P.n), np.diff(P.row_ptr))
    assert P.row_ptr[0] == 0 and P.row_ptr[-1] == P.nnz and (np.diff(P.row_ptr) >= 0).all()
    assert ((P.col_idx >= 0) & (P.col_idx < P.n)).all() and not (P.col_idx == rows).any()
    assert (P.mi > 0).all() and ((P.b_node >= 0) & (P.b_node < P.n)).all()
    order = np.argsort(P.b_node, kind="stable")
    b_ptr = np.zeros(P.n + 1, np.int32)
    np.add.at(b_ptr, P.b_node + 1, 1)
    b_ptr = np.cumsum(b_ptr).astype(np.int32)
    keep = dict(row_ptr=torch.from_numpy(P.row_ptr.astype(np.int32)).cuda(),
                col_idx=torch.from_numpy(P.col_idx.astype(np.int32)).cuda(),
                cij=torch.from_numpy(np.ascontiguousarray(P.cij)).cuda(),
                mi=torch.from_numpy(np.ascontiguousarray(P.mi)).cuda(),
                b_ptr=torch.from_numpy(b_ptr).cuda(),
                b_c=torch.from_numpy(np.ascontiguousarray(P.b_c[:, order])).cuda(),
                b_type=torch.from_numpy(np.ascontiguousarray(P.b_type[order].astype(np.int32))).cuda())

    def p(t):
        return t.data_ptr() if t.numel() else None

    mesh = DevMesh(P.dim, P.n, P.nnz, P.nb, p(keep["row_ptr"]), p(keep["col_idx"]), p(keep["cij"]), p(keep["mi"]),
                   p(keep["b_ptr"]), p(keep["b_c"]), p(keep["b_type"]), gamma)
    return mesh, keep, order


def _cases():
    P1, U1 = four_quadrant_problem(14, 2, seed=3)
    P2, U2, bd = dirichlet_vortex_problem(9, 1)
    P3 = assembly.assemble_1d(300, 1)
    U3 = workloads.sod(P3.x[0])
    P4 = assembly.assemble_1d(120, 2, bc=("inoutflow", "inoutflow"))
    U4 = workloads.sod(P4.x[0])
    return [("q2_four_quadrant_slip", P1, U1, None, 1.4), ("q1_vortex_dirichlet", P2, U2, bd(0.0), 5.0 / 3.0),
            ("sod_1d", P3, U3, None, 1.4), ("sod_1d_inoutflow", P4, U4, workloads.sod(P4.b_x[0]), 1.4)]


def _references(torch, P, U, bdata, gamma):
    """tau of the handle-based gdg_max_dt and of the oracle for the same mesh and state."""
    from oracle.oracle import Oracle
    from paper_2402_04514_gb300.gdg import Solver

    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    bd = None if bdata is None else torch.from_numpy(np.ascontiguousarray(bdata)).cuda()
    return Solver(P, gamma=gamma).max_dt(Ud, 0.5, bdata=bd), Oracle(P, gamma=gamma).max_dt(U, 0.5, bdata=bdata)


def _no_alloc(torch, P, U, bdata, gamma):
    from paper_2402_04514_gb300.gdg import max_dt_noalloc

    mesh, keep, order = _dev_mesh(torch, P, gamma)
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    bd_sorted = None if bdata is None else torch.from_numpy(np.ascontiguousarray(bdata[:, order])).cuda()
    tau = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    assert max_dt_noalloc(mesh, Ud, 0.5, tau, bdata=bd_sorted) == 0
    torch.cuda.synchronize()
    return float(tau.item())


@pytest.mark.parametrize("case", range(4))
def test_no_alloc_max_dt_matches_handle_max_dt(torch_cuda, case):
    """Two calls in a row on the same mesh: both equal gdg_max_dt and the oracle within 1e-13."""
    torch = torch_cuda
    name, P, U, bdata, gamma = _cases()[case]
    ref, orc = _references(torch, P, U, bdata, gamma)
    assert abs(ref - orc) <= 1e-13 * orc
    for call in range(2):
        got = _no_alloc(torch, P, U, bdata, gamma)
        assert abs(got - ref) <= 1e-13 * ref, (name, call, got, ref)
        assert abs(got - orc) <= 1e-13 * orc, (name, call, got, orc)


def test_no_alloc_reads_only_its_own_slots(torch_cuda):
    """A call on a large mesh (127 blocks of partial minima, small tau) and then one on a small mesh (one
    block, larger tau): the second result is the small mesh's own tau, so the final reduction reads only
    the slots its own call wrote, not the previous call's leftovers."""
    torch = torch_cuda
    Pb, Ub = four_quadrant_problem(60, 2, seed=1)
    Ps = assembly.assemble_1d(20, 1)
    Us = workloads.sod(Ps.x[0])
    big = _no_alloc(torch, Pb, Ub, None, 1.4)
    ref_b, orc_b = _references(torch, Pb, Ub, None, 1.4)
    small = _no_alloc(torch, Ps, Us, None, 1.4)
    ref_s, orc_s = _references(torch, Ps, Us, None, 1.4)
    assert (Pb.n + 255) // 256 == 127 and big < 0.5 * small
    assert abs(big - ref_b) <= 1e-13 * ref_b and abs(big - orc_b) <= 1e-13 * orc_b
    assert abs(small - ref_s) <= 1e-13 * ref_s and abs(small - orc_s) <= 1e-13 * orc_s


def test_no_alloc_without_dirichlet_data_gives_nan(torch_cuda):
    """A Dirichlet mesh called without its boundary data: tau is NaN (the entry reports a missing input in
    its result; gdg_max_dt, which has a handle, refuses such a call instead)."""
    torch = torch_cuda
    P, U, _ = dirichlet_vortex_problem(6, 1)
    got = _no_alloc(torch, P, U, None, 5.0 / 3.0)
    assert got != got


def test_no_alloc_rejects_meshes_above_its_limit(torch_cuda):
    from paper_2402_04514_gb300.gdg import DevMesh, max_dt_noalloc

    too_big = DevMesh(2, MAX_NODES + 1, 0, 0, None, None, None, None, None, None, None, 1.4)
    torch = torch_cuda
    tau = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert max_dt_noalloc(too_big, None, 0.5, tau) == 8  # GDG_ENOTSUP, nothing launched
    assert float(tau.item()) == 0.0
