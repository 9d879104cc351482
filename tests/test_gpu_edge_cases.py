"""Degenerate and boundary cases of the method on the GPU: one-level hierarchies (the cycle is the
coarse solve itself), a single element, a one-unknown FD grid, one-element-wide meshes, the
smallest smoothing order, meshes whose every node is a boundary node, and sizes beyond the
30-bit global-id limit (rejected before any allocation)."""
import numpy as np
import pytest

import workloads as W
from oracle import krylov as K
from oracle import multigrid as M
from oracle import problems as P
from oracle.sem import SemLevel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2210_03179_gb300 as cm  # noqa: E402
from gpu_util import N, T, relerr  # noqa: E402

F64 = cm.CHEBMG_F64


def test_fd_single_level_is_the_dense_solve():
    s = cm.Solver("fd2d", m=7, coarsening=2, coarsest=7)
    assert s.num_levels == 1
    H = P.fd_hierarchy(7, coarsest=7)
    b = W.fd_rhs(7)
    u = torch.zeros(49, dtype=torch.float64, device="cuda")
    code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, T(b), u, 1e-12, 10)
    assert code == cm.CHEBMG_OK and it == 1 and rel < 1e-12
    assert relerr(N(u), np.linalg.solve(H.levels[0].A.toarray(), b)) < 1e-12
    s.close()


def test_fd_one_unknown():
    s = cm.Solver("fd2d", m=1, coarsening=2, coarsest=1)
    assert s.num_levels == 1 and s.size(0) == 1
    u = torch.zeros(1, dtype=torch.float64, device="cuda")
    code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, T([2.0]), u, 1e-12, 5)
    # -Laplacian on one interior point of the unit square: 4 u / h^2 = b with h = 1/2
    assert code == cm.CHEBMG_OK and abs(float(u[0]) - 2.0 / 16.0) < 1e-15
    s.close()


def test_sem_single_level_is_the_coarse_cg():
    v = W.sem_box_vertices(3, 4, 5)
    L = SemLevel(v, 1)
    s = cm.Solver("sem", verts=v, orders=(1,))
    assert s.num_levels == 1
    b = W.sem_rhs(3, 4, 5, 1)
    u = torch.zeros(L.n, dtype=torch.float64, device="cuda")
    code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, T(b), u, 1e-8, 10)
    assert code == cm.CHEBMG_OK and it == 1          # the coarse CG solves to 1e-10 in one cycle
    assert np.linalg.norm(b - L.apply_A(N(u))) <= 1e-9 * np.linalg.norm(b)
    s.close()


@pytest.mark.parametrize("mesh", [(1, 1, 1), (1, 1, 4), (5, 1, 1)])
def test_thin_and_single_element_meshes(mesh):
    # one element, or one element across: every level has few free nodes, and (1,1,1) at N = 1 has
    # none at all (the coarsest problem is empty)
    v = W.sem_box_vertices(*mesh)
    H = P.sem_hierarchy(v, (7, 3, 1))
    s = cm.Solver("sem", verts=v, orders=(7, 3, 1), lmax=[L.lmax for L in H.levels[:-1]])
    L0 = H.levels[0]
    x = np.random.default_rng(0).uniform(-1, 1, L0.n)
    y = torch.zeros(L0.n, dtype=torch.float64, device="cuda")
    cm.chebmg_apply_A(s.ctx, 0, F64, T(x), y)
    assert relerr(N(y), L0.apply_A(x)) < 1e-12
    b = W.sem_rhs(*mesh, 7)
    _, it_ref, _ = K.fcg(L0.apply_A, lambda r: M.vcycle(H, r), b, 1e-8)
    u = torch.zeros(L0.n, dtype=torch.float64, device="cuda")
    code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, T(b), u, 1e-8, 100)
    assert code == cm.CHEBMG_OK and abs(it - it_ref) <= 1 and rel <= 1e-8
    s.close()


def test_order_one_smoother_everywhere():
    # k = 1: the optimized 4th kind is the 3/2-damped Jacobi iteration (Sec. 2.3)
    v = W.sem_box_vertices(2, 3, 2)
    H = P.sem_hierarchy(v, (4, 2, 1), kind="opt4th", k=1, sided="symmetric")
    s = cm.Solver("sem", verts=v, orders=(4, 2, 1), kind="opt4th", order=1, sided="symmetric",
                  lmax=[L.lmax for L in H.levels[:-1]])
    b = W.sem_rhs(2, 3, 2, 4)
    z = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    cm.chebmg_vcycle(s.ctx, T(b), z)
    assert relerr(N(z), M.vcycle(H, b)) < 1e-8
    s.close()


def test_sizes_beyond_the_id_limit_are_rejected():
    # 1025^3 > 2^30 global nodes: refused from the sizes alone (no vertices are read)
    opts = cm.chebmg_default_opts()
    verts = np.zeros((2, 2, 2, 3))
    ctx = cm.c_void_p()
    ords = (cm.c_int * 1)(7)
    code = cm.lib().chebmg_setup_sem(147, 147, 147, verts.ctypes.data_as(cm.POINTER(cm.c_double)), ords, 1,
                                     cm.byref(opts), cm.byref(ctx))
    assert code == cm.CHEBMG_EINVAL and not ctx.value
