"""The outer Krylov product in FP64-class arithmetic on FP32 pairs (CHEBMG_OUTER_F32X2).

The order-7 operator evaluated with every operation on (hi, lo) FP32 pairs must agree with the
FP64 oracle's operator (Sec. 1, Eq. 1.3) to 1e-12 per application -- the bar of the FP64 GPU
operator -- on random and smooth fields, on the box lattice and on a general mesh (map ids);
a mixed solve that uses it must take the oracle's iteration count within one and reach a true
(FP64) relative residual of 1e-8.
"""
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

MESH = (3, 4, 5)


@pytest.fixture(scope="module")
def verts():
    return W.sem_box_vertices(*MESH)


def fields(L, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, L.n)
    X = np.zeros(L.n)
    Y = np.zeros(L.n)
    Z = np.zeros(L.n)
    for c, Vv in zip(L.coords.reshape(-1, 3), L.gid.reshape(-1)):
        X[Vv], Y[Vv], Z[Vv] = c
    smooth = np.sin(np.pi * X) * np.cos(2 * Y) * (1 + Z ** 2)
    return [x, smooth]


def test_operator_matches_oracle_on_the_box(verts):
    L = SemLevel(verts, 7)
    s = cm.Solver("sem", verts=verts, orders=(7, 3, 1), prec="mixed", lmax=[1.0, 1.0])
    cm.chebmg_set_outer_operator(s.ctx, cm.CHEBMG_OUTER_F32X2)
    for x in fields(L, 3):
        x = np.where(L.dirichlet, 0.0, x)
        y = torch.zeros(L.n, dtype=torch.float64, device="cuda")
        cm.chebmg_apply_outer(s.ctx, T(x), y)
        ref = L.apply_A(x)
        assert relerr(N(y), ref) < 1e-12
        y64 = torch.zeros_like(y)
        cm.chebmg_apply_A(s.ctx, 0, cm.CHEBMG_F64, T(x), y64)
        assert relerr(N(y), N(y64)) < 1e-12
    # back to FP64: the native operator again (equal up to the atomics' summation order)
    cm.chebmg_set_outer_operator(s.ctx, cm.CHEBMG_OUTER_FP64)
    x = np.where(L.dirichlet, 0.0, fields(L, 4)[0])
    y = torch.zeros(L.n, dtype=torch.float64, device="cuda")
    y64 = torch.zeros_like(y)
    cm.chebmg_apply_outer(s.ctx, T(x), y)
    cm.chebmg_apply_A(s.ctx, 0, cm.CHEBMG_F64, T(x), y64)
    assert relerr(N(y), N(y64)) < 1e-14
    s.close()


def test_operator_on_a_general_mesh(verts):
    from test_gpu_mesh import general_mesh
    L, coords, gid, dirichlet, relabel = general_mesh(verts, 7, seed=5)
    s = cm.Solver("sem_mesh", coords=coords, gid=gid, n=L.n, dirichlet=dirichlet, orders=(7, 3, 1), prec="mixed",
                  lmax=[1.0, 1.0])
    cm.chebmg_set_outer_operator(s.ctx, cm.CHEBMG_OUTER_F32X2)
    u = np.random.default_rng(6).uniform(-1, 1, L.n)
    un = np.empty_like(u)
    un[relabel] = u
    y = torch.zeros(L.n, dtype=torch.float64, device="cuda")
    cm.chebmg_apply_outer(s.ctx, T(un), y)
    assert relerr(N(y)[relabel], L.apply_A(u)) < 1e-12
    s.close()


def test_mixed_solve_with_pair_arithmetic_outer_product(verts):
    H = P.sem_hierarchy(verts, (7, 3, 1), kind="opt4th", k=3, sided="one-sided")
    s = cm.Solver("sem", verts=verts, orders=(7, 3, 1), kind="opt4th", order=3, sided="one-sided", prec="mixed",
                  lmax=[L.lmax for L in H.levels[:-1]])
    cm.chebmg_set_outer_operator(s.ctx, cm.CHEBMG_OUTER_F32X2)
    b = W.sem_rhs(*MESH, 7)
    _, it_ref, _ = K.fcg(H.levels[0].apply_A, lambda r: M.vcycle(H, r), b, 1e-8)
    u = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, T(b), u, 1e-8, 100)
    assert code == cm.CHEBMG_OK and rel <= 1e-8 and abs(it - it_ref) <= 1, (it, it_ref)
    assert np.linalg.norm(b - H.levels[0].apply_A(N(u))) <= 1.01e-8 * np.linalg.norm(b)
    s.close()


def test_refused_where_it_does_not_apply(verts):
    f = cm.Solver("fd2d", m=15, coarsening=2, coarsest=7)
    with pytest.raises(cm.ChebmgError):
        cm.chebmg_set_outer_operator(f.ctx, cm.CHEBMG_OUTER_F32X2)
    f.close()
    s = cm.Solver("sem", verts=verts, orders=(5, 1), lmax=[1.0])
    with pytest.raises(cm.ChebmgError):
        cm.chebmg_set_outer_operator(s.ctx, cm.CHEBMG_OUTER_F32X2)
    with pytest.raises(cm.ChebmgError):
        cm.chebmg_set_outer_operator(s.ctx, 7)
    s.close()


def test_batched_solve_with_pair_arithmetic_outer_product(verts):
    H = P.sem_hierarchy(verts, (7, 3, 1), kind="opt4th", k=3, sided="one-sided")
    s = cm.Solver("sem", verts=verts, orders=(7, 3, 1), kind="opt4th", order=3, sided="one-sided", prec="mixed",
                  lmax=[L.lmax for L in H.levels[:-1]])
    cm.chebmg_set_outer_operator(s.ctx, cm.CHEBMG_OUTER_F32X2)
    A = H.levels[0].apply_A
    bs = [W.sem_rhs(*MESH, 7, seed=q) for q in range(5)]
    B = torch.tensor(np.stack(bs), device="cuda")
    for graph in (True, False):
        U = torch.zeros_like(B)
        code, its, rel = cm.chebmg_pcg_solve_batched(s.ctx, B, U, 1e-8, 100, graph=graph)
        assert code == cm.CHEBMG_OK and max(rel) <= 1e-8
        for q, b in enumerate(bs):
            _, it_ref, _ = K.fcg(A, lambda r: M.vcycle(H, r), b, 1e-8)
            assert abs(its[q] - it_ref) <= 1, (q, its[q], it_ref)
            assert np.linalg.norm(b - A(N(U[q]))) <= 1.01e-8 * np.linalg.norm(b)
    s.close()
