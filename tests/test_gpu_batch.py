"""Batches of right-hand sides and groups of meshes (Sec. 1: a sequence of Poisson problems
A u = b with one operator, setup amortised over them).

Each right-hand side of a batch must give what a separate solve gives: the batched operator
and V-cycle against the oracle element by element, the batched flexible CG against the
oracle's iteration count (within one) and the 1e-8 relative residual, and the same answer
with and without CUDA-graph replay.  Workloads: 64 right-hand sides (seeds 0..63) on
E = 8^3, N = 7, and the uneven group E in {4^3, 6^3, 8^3, 12^3} x N in {5, 7, 9}.
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

F64, F32 = cm.CHEBMG_F64, cm.CHEBMG_F32
MESH = (3, 4, 5)   # 60 elements: ragged last block for every elements-per-block choice


@pytest.fixture(scope="module")
def verts():
    return W.sem_box_vertices(*MESH)


def sem_solver(v, orders=(7, 3, 1), kind="opt4th", k=2, sided="one-sided", prec="fp64", lmax=None):
    return cm.Solver("sem", verts=v, orders=orders, kind=kind, order=k, sided=sided, prec=prec, lmax=lmax)


def rows(a):
    return T(np.ascontiguousarray(np.stack(a)))


def batch_variants():
    out = []
    for rb in (1, 3, 8):
        for eb in (1, 2, 4):
            for im in (0, 100):
                out.append(1000 * rb + im + eb)
    # right-hand sides taken in pairs through each line pass (odd counts leave a lone last one)
    for rb in (2, 3, 8):
        for eb in (11, 12):
            for im in (0, 100):
                out.append(1000 * rb + im + eb)
    # geometric factors held in registers across the block's right-hand sides
    for rb in (1, 3, 8):
        for eb in (21, 22):
            for im in (0, 100):
                out.append(1000 * rb + im + eb)
    return out


@pytest.mark.parametrize("variant", batch_variants())
def test_batched_order7_operator_every_variant(verts, variant):
    L = SemLevel(verts, 7)
    s = sem_solver(verts, (7, 3, 1), prec="mixed", lmax=[1.0, 1.0])
    nrhs = 7
    X = np.random.default_rng(variant).uniform(-1, 1, (nrhs, L.n))
    for dt in (F64, F32):
        try:
            cm.chebmg_set_batch_tile_choice(s.ctx, nrhs, 0, dt, variant)
        except cm.ChebmgError as e:
            assert e.code == cm.CHEBMG_EINVAL   # does not fit the shared-memory limit
            continue
        tdt = torch.float64 if dt == F64 else torch.float32
        Y = torch.zeros((nrhs, L.n), dtype=tdt, device="cuda")
        cm.chebmg_apply_A_batched(s.ctx, 0, dt, T(X, tdt), Y)
        for q in range(nrhs):
            xq = X[q] if dt == F64 else X[q].astype(np.float32).astype(np.float64)
            assert relerr(N(Y[q]), L.apply_A(xq)) < (1e-12 if dt == F64 else 1e-5)
    s.close()


@pytest.mark.parametrize("variant", [1002, 3004, 2102, 3012, 2112, 1022, 3122, 5021])
def test_batched_order7_operator_ragged_last_batch(variant):
    # 3 x 3 x 3 = 27 elements: a ragged last element batch for 2 and 4 elements per block
    v = W.sem_box_vertices(3, 3, 3)
    L = SemLevel(v, 7)
    s = sem_solver(v, (7, 3, 1), prec="mixed", lmax=[1.0, 1.0])
    nrhs = 5
    X = np.random.default_rng(variant).uniform(-1, 1, (nrhs, L.n))
    for dt in (F64, F32):
        try:
            cm.chebmg_set_batch_tile_choice(s.ctx, nrhs, 0, dt, variant)
        except cm.ChebmgError as e:
            assert e.code == cm.CHEBMG_EINVAL and dt == F64 and variant % 100 >= 20   # FP32-only form
            continue
        tdt = torch.float64 if dt == F64 else torch.float32
        Y = torch.zeros((nrhs, L.n), dtype=tdt, device="cuda")
        cm.chebmg_apply_A_batched(s.ctx, 0, dt, T(X, tdt), Y)
        for q in range(nrhs):
            xq = X[q] if dt == F64 else X[q].astype(np.float32).astype(np.float64)
            assert relerr(N(Y[q]), L.apply_A(xq)) < (1e-12 if dt == F64 else 1e-5), (variant, dt, q)
    s.close()


@pytest.mark.parametrize("orders", [(7, 3, 1), (9, 5, 2), (6, 1)])
def test_batched_operator_all_levels(verts, orders):
    levels = [SemLevel(verts, Nn) for Nn in orders]
    s = sem_solver(verts, orders, lmax=[1.0] * (len(orders) - 1))
    rng = np.random.default_rng(7)
    for j, L in enumerate(levels):
        X = rng.uniform(-1, 1, (5, L.n))
        Y = torch.zeros((5, L.n), dtype=torch.float64, device="cuda")
        cm.chebmg_apply_A_batched(s.ctx, j, F64, T(X), Y)
        for q in range(5):
            assert relerr(N(Y[q]), L.apply_A(X[q])) < 1e-12
    s.close()


@pytest.mark.parametrize("kind,k,sided", [("opt4th", 2, "one-sided"), ("1st", 2, "symmetric"),
                                          ("4th", 1, "symmetric")])
def test_batched_vcycle_sem(verts, kind, k, sided):
    H = P.sem_hierarchy(verts, (7, 3, 1), kind=kind, k=k, sided=sided)
    s = sem_solver(verts, kind=kind, k=k, sided=sided, lmax=[L.lmax for L in H.levels[:-1]])
    R = [W.sem_rhs(*MESH, 7, seed=q) for q in range(4)]
    Z = torch.zeros((4, len(R[0])), dtype=torch.float64, device="cuda")
    cm.chebmg_vcycle_batched(s.ctx, rows(R), Z)
    for q in range(4):
        # the coarse CG stops at 1e-10, so the cycles agree to about that level
        assert relerr(N(Z[q]), M.vcycle(H, R[q])) < 1e-8
    s.close()


@pytest.mark.parametrize("kind,k,sided", [("opt4th", 2, "one-sided"), ("1st", 2, "symmetric")])
def test_batched_vcycle_fd(kind, k, sided):
    H = P.fd_hierarchy(63, kind=kind, k=k, sided=sided)
    s = cm.Solver("fd2d", m=63, kind=kind, order=k, sided=sided, lmax=[L.lmax for L in H.levels[:-1]])
    R = [W.fd_rhs(63, seed=q) for q in range(5)]
    Z = torch.zeros((5, 3969), dtype=torch.float64, device="cuda")
    cm.chebmg_vcycle_batched(s.ctx, rows(R), Z)
    for q in range(5):
        assert relerr(N(Z[q]), M.vcycle(H, R[q])) < 1e-12
    s.close()


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_solve_sem_matches_oracle(verts, graph, prec):
    H = P.sem_hierarchy(verts, (7, 3, 1))
    s = sem_solver(verts, prec=prec, lmax=[L.lmax for L in H.levels[:-1]])
    A = H.levels[0].apply_A
    B = [W.sem_rhs(*MESH, 7, seed=q) for q in range(4)]
    B.append(np.zeros_like(B[0]))           # a zero right-hand side stops at once
    U = torch.full((5, len(B[0])), 7.0, dtype=torch.float64, device="cuda")
    code, its, rel = cm.chebmg_pcg_solve_batched(s.ctx, rows(B), U, 1e-8, 200, graph=graph)
    assert code == cm.CHEBMG_OK
    for q in range(4):
        _, it_ref, _ = K.fcg(A, lambda r: M.vcycle(H, r), B[q], 1e-8)
        assert abs(its[q] - it_ref) <= 1
        assert rel[q] <= 1e-8
        assert np.linalg.norm(B[q] - A(N(U[q]))) <= 1.01e-8 * np.linalg.norm(B[q])
    assert its[4] == 0 and rel[4] == 0.0 and float(U[4].abs().max()) == 0.0
    s.close()


def test_batched_equals_single_and_graph_equals_eager(verts):
    H = P.sem_hierarchy(verts, (7, 3, 1))
    s = sem_solver(verts, prec="mixed", lmax=[L.lmax for L in H.levels[:-1]])
    B = [W.sem_rhs(*MESH, 7, seed=10 + q) for q in range(6)]
    n = len(B[0])
    U1 = torch.zeros((6, n), dtype=torch.float64, device="cuda")
    U2 = torch.zeros_like(U1)
    _, its_g, _ = cm.chebmg_pcg_solve_batched(s.ctx, rows(B), U1, 1e-8, 200, graph=True)
    _, its_g2, _ = cm.chebmg_pcg_solve_batched(s.ctx, rows(B), U1, 1e-8, 200, graph=True)   # replayed graphs
    _, its_e, _ = cm.chebmg_pcg_solve_batched(s.ctx, rows(B), U2, 1e-8, 200, graph=False)
    assert its_g == its_e == its_g2
    assert relerr(N(U1), N(U2)) < 1e-9
    for q in (0, 5):
        u = torch.zeros(n, dtype=torch.float64, device="cuda")
        _, it, _, _ = cm.chebmg_pcg_solve(s.ctx, T(B[q]), u, 1e-8, 200)
        assert abs(it - its_g[q]) <= 1
        assert relerr(N(U1[q]), N(u)) < 1e-6
    s.close()


def test_batched_solve_fd_config():
    # 2-D FD, 63 x 63, order 2 symmetric and order 4 one-sided, 1st and 4th kind
    for kind, k, sided in [("1st", 2, "symmetric"), ("4th", 4, "one-sided"), ("opt4th", 2, "one-sided")]:
        H = P.fd_hierarchy(63, kind=kind, k=k, sided=sided)
        s = cm.Solver("fd2d", m=63, kind=kind, order=k, sided=sided, lmax=[L.lmax for L in H.levels[:-1]])
        B = [W.fd_rhs(63, seed=q) for q in range(6)]
        U = torch.zeros((6, 3969), dtype=torch.float64, device="cuda")
        code, its, rel = cm.chebmg_pcg_solve_batched(s.ctx, rows(B), U, 1e-8, 200)
        assert code == cm.CHEBMG_OK
        A = H.levels[0].apply_A
        for q in range(6):
            _, it_ref, _ = K.fcg(A, lambda r: M.vcycle(H, r), B[q], 1e-8)
            assert abs(its[q] - it_ref) <= 1 and rel[q] <= 1e-8
            assert np.linalg.norm(B[q] - A(N(U[q]))) <= 1.01e-8 * np.linalg.norm(B[q])
        s.close()


def test_batched_large_coarse_level_runs_per_rhs(verts):
    # coarsest level N = 4 on 3 x 4 x 5 elements has 4641 nodes: more than one thread block
    # holds, so each right-hand side's coarse solve is a separate persistent solve
    H = P.sem_hierarchy(verts, (7, 4))
    s = sem_solver(verts, (7, 4), lmax=[H.levels[0].lmax])
    B = [W.sem_rhs(*MESH, 7, seed=q) for q in range(3)]
    U = torch.zeros((3, len(B[0])), dtype=torch.float64, device="cuda")
    code, its, rel = cm.chebmg_pcg_solve_batched(s.ctx, rows(B), U, 1e-8, 200)
    assert code == cm.CHEBMG_OK
    A = H.levels[0].apply_A
    for q in range(3):
        _, it_ref, _ = K.fcg(A, lambda r: M.vcycle(H, r), B[q], 1e-8)
        assert abs(its[q] - it_ref) <= 1 and rel[q] <= 1e-8
    s.close()


def test_64_rhs_on_8cubed_mixed():
    ne = 8
    v = W.sem_box_vertices(ne, ne, ne)
    s = sem_solver(v, prec="mixed")
    n = s.size(0)
    assert n == 57 ** 3
    B = torch.tensor(np.stack([W.sem_rhs(ne, ne, ne, 7, seed=q) for q in range(64)]), device="cuda")
    U = torch.zeros_like(B)
    code, its, rel = cm.chebmg_pcg_solve_batched(s.ctx, B, U, 1e-8, 200)
    assert code == cm.CHEBMG_OK and max(rel) <= 1e-8
    variant, degree = cm.chebmg_batch_info(s.ctx, 64, 0, F32)
    assert variant // 1000 >= 1 and variant % 100 in (1, 2, 4, 11, 12, 21, 22) and degree in (1, 2, 4, 8, 12, 16)
    # true residuals with the FP64 operator (checked against the oracle above)
    AU = torch.zeros_like(U)
    cm.chebmg_apply_A_batched(s.ctx, 0, F64, U, AU)
    mask = torch.tensor(W.sem_boundary_mask(ne, ne, ne, 7), device="cuda")
    Bm = B.masked_fill(mask, 0.0)
    true_rel = (Bm - AU).norm(dim=1) / Bm.norm(dim=1)
    assert float(true_rel.max()) <= 1.01e-8
    # sampled right-hand sides against separate solves
    for q in (0, 37, 63):
        u = torch.zeros(n, dtype=torch.float64, device="cuda")
        _, it, _, _ = cm.chebmg_pcg_solve(s.ctx, B[q].contiguous(), u, 1e-8, 200)
        assert abs(it - its[q]) <= 1
    s.close()


def test_uneven_group_of_meshes():
    ctxs, solvers, Bs, shapes = [], [], [], []
    for ne in (4, 6, 8, 12):
        v = W.sem_box_vertices(ne, ne, ne)
        for Nn in (5, 7, 9):
            sv = sem_solver(v, (Nn, 3, 1), prec="mixed")
            solvers.append(sv)
            ctxs.append(sv.ctx)
            shapes.append((ne, Nn))
            Bs.append(T(W.sem_rhs(ne, ne, ne, Nn, seed=len(Bs))))
    g = cm.chebmg_group_create(ctxs)
    try:
        out = {}
        for graph in (True, False, True):
            Us = [torch.zeros_like(b) for b in Bs]
            code, its, rel = cm.chebmg_group_pcg_solve(g, ctxs, Bs, Us, 1e-8, 200, graph=graph)
            assert code == cm.CHEBMG_OK and max(rel) <= 1e-8
            out[graph] = (its, Us)
        assert out[True][0] == out[False][0]
        for k, sv in enumerate(solvers):
            u = torch.zeros_like(Bs[k])
            _, it, _, _ = cm.chebmg_pcg_solve(sv.ctx, Bs[k], u, 1e-8, 200)
            assert abs(it - out[True][0][k]) <= 1
            y = torch.zeros_like(u)
            cm.chebmg_apply_A(sv.ctx, 0, F64, out[True][1][k], y)
            ne, Nn = shapes[k]
            b = Bs[k].masked_fill(torch.tensor(W.sem_boundary_mask(ne, ne, ne, Nn), device="cuda"), 0.0)
            assert float((b - y).norm() / b.norm()) <= 1.01e-8
    finally:
        cm.chebmg_group_destroy(g)
        for sv in solvers:
            sv.close()


def test_smallest_group_member_matches_oracle():
    v = W.sem_box_vertices(4, 4, 4)
    H = P.sem_hierarchy(v, (5, 3, 1))
    s = sem_solver(v, (5, 3, 1), lmax=[L.lmax for L in H.levels[:-1]])
    b = W.sem_rhs(4, 4, 4, 5, seed=0)
    g = cm.chebmg_group_create([s.ctx])
    U = [torch.zeros(len(b), dtype=torch.float64, device="cuda")]
    code, its, rel = cm.chebmg_group_pcg_solve(g, [s.ctx], [T(b)], U, 1e-8, 200)
    cm.chebmg_group_destroy(g)
    _, it_ref, _ = K.fcg(H.levels[0].apply_A, lambda r: M.vcycle(H, r), b, 1e-8)
    assert code == cm.CHEBMG_OK and abs(its[0] - it_ref) <= 1 and rel[0] <= 1e-8
    s.close()


def test_batch_argument_errors(verts):
    s = sem_solver(verts, lmax=[1.0, 1.0])
    n = s.size(0)
    L = cm.lib()
    X = torch.zeros((2, n), dtype=torch.float64, device="cuda")
    import ctypes
    ptr = ctypes.c_void_p(X.data_ptr())
    assert L.chebmg_pcg_solve_batched(s.ctx, 0, ptr, ptr, 1e-8, 10, 0, None, None) == cm.CHEBMG_EINVAL
    assert L.chebmg_pcg_solve_batched(s.ctx, 2, ptr, ptr, 1e-8, 10, 8, None, None) == cm.CHEBMG_EINVAL
    assert L.chebmg_pcg_solve_batched(s.ctx, 2, None, ptr, 1e-8, 10, 0, None, None) == cm.CHEBMG_EINVAL
    with pytest.raises(cm.ChebmgError):
        cm.chebmg_set_batch_tile_choice(s.ctx, 4, 1, F64, 2002)     # level 1 is not order 7
    with pytest.raises(cm.ChebmgError):
        cm.chebmg_set_batch_tile_choice(s.ctx, 4, 0, F64, 2003)     # 3 elements per block
    with pytest.raises(cm.ChebmgError):
        cm.chebmg_group_create([s.ctx, s.ctx])
    # maxit reached: ENOTCONV with valid outputs
    B = rows([W.sem_rhs(*MESH, 7, seed=1), W.sem_rhs(*MESH, 7, seed=2)])
    code, its, rel = cm.chebmg_pcg_solve_batched(s.ctx, B, X, 1e-14, 2)
    assert code == cm.CHEBMG_ENOTCONV and its == [2, 2] and min(rel) > 1e-14
    s.close()
