"""gdg_max_dt_noalloc, the time-step entry point for callers that may not allocate device memory (for
instance code running under CUDA-graph stream capture, or a plug-in whose host application owns all
device memory through its own pool).  It must give the same tau as the handle-based gdg_max_dt, on two
calls in a row (its fixed device scratch keeps the previous call's contents), and refuse meshes above
its size limit.  This file sorts last so a failure here comes after every other GPU test has run."""
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


@pytest.mark.parametrize("case", range(4))
def test_no_alloc_max_dt_matches_handle_max_dt(torch_cuda, case):
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import Solver, max_dt_noalloc

    name, P, U, bdata, gamma = _cases()[case]
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    bd = None if bdata is None else torch.from_numpy(np.ascontiguousarray(bdata)).cuda()
    ref = Solver(P, gamma=gamma).max_dt(Ud, 0.5, bdata=bd)
    mesh, keep, order = _dev_mesh(torch, P, gamma)
    bd_sorted = None if bdata is None else torch.from_numpy(np.ascontiguousarray(bdata[:, order])).cuda()
    tau = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        tau.fill_(float("nan"))
        assert max_dt_noalloc(mesh, Ud, 0.5, tau, bdata=bd_sorted) == 0
        torch.cuda.synchronize()
        got = float(tau.item())
        assert abs(got - ref) <= 1e-13 * ref, (name, call, got, ref)


def test_no_alloc_rejects_meshes_above_its_limit(torch_cuda):
    from paper_2402_04514_gb300.gdg import DevMesh, max_dt_noalloc

    too_big = DevMesh(2, MAX_NODES + 1, 0, 0, None, None, None, None, None, None, None, 1.4)
    torch = torch_cuda
    tau = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert max_dt_noalloc(too_big, None, 0.5, tau) == 8  # GDG_ENOTSUP, nothing launched
    assert float(tau.item()) == 0.0
