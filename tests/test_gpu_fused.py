"""The fused order-7 smoother: every step of Algorithm 1 or 2 (element operator with gather-scatter,
Sec. 1 Eq. 1.3; Jacobi-scaled Chebyshev recurrence; residual update) and, inside a V-cycle, the
restriction residual r = b - A x of Eq. 2.2, in one persistent launch.  Held to the FP64 oracle at
1e-12 per smoother application on box meshes of one to nine element planes (the kernel's work
is cut by element plane) in FP64; the FP32 variant against the FP32 separate
kernels and the oracle; cycles and solves with the fused path forced on against the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import krylov as K
from oracle import multigrid as M
from oracle import problems as P
from oracle.chebyshev import smooth as oracle_smooth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2210_03179_gb300 as cm  # noqa: E402
from gpu_util import N, T, empty, relerr  # noqa: E402

F64, F32 = cm.CHEBMG_F64, cm.CHEBMG_F32

# element planes 7, 9, 2, 1, 5 (slabs of the fused kernel); ragged element counts per plane
MESHES = [(2, 3, 7), (1, 2, 9), (5, 3, 2), (1, 1, 1), (3, 4, 5)]


def solver(v, orders=(7, 3, 1), kind="opt4th", k=1, sided="symmetric", prec="fp64", lmax=None):
    return cm.Solver("sem", verts=v, orders=orders, kind=kind, order=k, sided=sided, prec=prec, lmax=lmax)


def _inputs(L, seed):
    rng = np.random.default_rng(seed)
    b = np.where(L.dirichlet, 0.0, rng.uniform(-1, 1, L.n))
    x0 = np.where(L.dirichlet, 0.0, rng.uniform(-1, 1, L.n))
    return b, x0


@pytest.mark.parametrize("mesh", MESHES, ids=lambda m: "x".join(map(str, m)))
@pytest.mark.parametrize("kind", ["1st", "4th", "opt4th"])
def test_fused_fp64_smoother_matches_oracle(mesh, kind):
    v = W.sem_box_vertices(*mesh)
    H = P.sem_hierarchy(v, (7, 3, 1), kind=kind, k=1, sided="symmetric")
    L = H.levels[0]
    s = solver(v, kind=kind, lmax=[Lv.lmax for Lv in H.levels[:-1]])
    b, x0 = _inputs(L, sum(mesh))
    for variant in (2,):
        cm.chebmg_set_fused_smoother(s.ctx, 0, F64, variant)
        assert cm.chebmg_fused_smoother(s.ctx, 0, F64) == variant
        for order in (1, 2, 3, 6):
            for x_zero in (True, False):
                ref = oracle_smooth(L, b, order, kind, L.lmax, 0.1, x0=None if x_zero else x0)
                x = empty(L.n) if x_zero else T(x0)
                cm.chebmg_smooth(s.ctx, 0, F64, T(b), x, order, x_zero)
                assert relerr(N(x), ref) < 1e-12, (variant, order, x_zero)
                assert np.all(N(x)[L.dirichlet] == 0.0)
    s.close()


@pytest.mark.parametrize("mesh", [(2, 3, 7), (3, 4, 5)], ids=lambda m: "x".join(map(str, m)))
@pytest.mark.parametrize("kind", ["1st", "opt4th"])
def test_fused_fp32_smoother_matches_separate_kernels_and_oracle(mesh, kind):
    v = W.sem_box_vertices(*mesh)
    H = P.sem_hierarchy(v, (7, 3, 1), kind=kind, k=1, sided="symmetric")
    L = H.levels[0]
    s = solver(v, kind=kind, prec="mixed", lmax=[Lv.lmax for Lv in H.levels[:-1]])
    b, x0 = _inputs(L, 3)
    b32 = b.astype(np.float32).astype(np.float64)
    x032 = x0.astype(np.float32).astype(np.float64)
    for order in (2, 5):
        for x_zero in (True, False):
            ref = oracle_smooth(L, b32, order, kind, L.lmax, 0.1, x0=None if x_zero else x032)
            out = {}
            for variant in (0, 1):
                cm.chebmg_set_fused_smoother(s.ctx, 0, F32, variant)
                x = empty(L.n, True) if x_zero else T(x0, torch.float32)
                cm.chebmg_smooth(s.ctx, 0, F32, T(b, torch.float32), x, order, x_zero)
                out[variant] = N(x)
            # the same FP32 arithmetic up to the order of the atomic sums
            assert relerr(out[1], out[0]) < 1e-5, (order, x_zero)
            # single-precision rounding against the FP64 oracle on the same (rounded) inputs
            assert relerr(out[1], ref) < 1e-4, (order, x_zero)
    s.close()


def test_fused_smoother_takes_misaligned_caller_vectors():
    # views that start 8 bytes into an allocation: the fused kernel's 16-byte accesses cannot
    # take them, so the call runs the separate kernels and still matches the oracle
    mesh = (2, 3, 7)
    v = W.sem_box_vertices(*mesh)
    H = P.sem_hierarchy(v, (7, 3, 1), kind="opt4th", k=1, sided="symmetric")
    L = H.levels[0]
    s = solver(v, lmax=[Lv.lmax for Lv in H.levels[:-1]])
    cm.chebmg_set_fused_smoother(s.ctx, 0, F64, 2)
    b, x0 = _inputs(L, 5)
    bb = T(np.concatenate([[0.0], b]))[1:]
    xx = T(np.concatenate([[0.0], x0]))[1:]
    ref = oracle_smooth(L, b, 4, "opt4th", L.lmax, 0.1, x0=x0)
    cm.chebmg_smooth(s.ctx, 0, F64, bb, xx, 4, False)
    assert relerr(N(xx), ref) < 1e-12
    s.close()


@pytest.mark.parametrize("kind,k,sided", [("opt4th", 3, "one-sided"), ("4th", 2, "symmetric"),
                                          ("1st", 2, "symmetric"), ("opt4th", 1, "one-sided")])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fused_vcycle_matches_oracle(kind, k, sided, prec):
    mesh = (3, 4, 5)
    v = W.sem_box_vertices(*mesh)
    H = P.sem_hierarchy(v, (7, 3, 1), kind=kind, k=k, sided=sided)
    s = solver(v, kind=kind, k=k, sided=sided, prec=prec, lmax=[Lv.lmax for Lv in H.levels[:-1]])
    dt = F32 if prec == "mixed" else F64
    r = W.sem_rhs(*mesh, 7, seed=6)
    z = {}
    for variant in (0, 1 if prec == "mixed" else 2):
        cm.chebmg_set_fused_smoother(s.ctx, 0, dt, variant)
        z[variant] = empty(len(r))
        cm.chebmg_vcycle(s.ctx, T(r), z[variant])
    zf = N(z[max(z)])
    ref = M.vcycle(H, r)
    if prec == "fp64":
        # the coarse CG stops at 1e-10, so cycles agree to about that level
        assert relerr(zf, ref) < 1e-8
        assert relerr(zf, N(z[0])) < 1e-8
    else:
        assert relerr(zf, N(z[0])) < 1e-5
        assert relerr(zf, ref) < 1e-4
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("sided", ["one-sided", "symmetric"])
def test_fused_solve_iterations_match_oracle(prec, sided):
    mesh = (2, 3, 7)
    v = W.sem_box_vertices(*mesh)
    H = P.sem_hierarchy(v, (7, 3, 1), kind="opt4th", k=2, sided=sided)
    s = solver(v, k=2, sided=sided, prec=prec, lmax=[Lv.lmax for Lv in H.levels[:-1]])
    cm.chebmg_set_fused_smoother(s.ctx, 0, F32 if prec == "mixed" else F64, 1 if prec == "mixed" else 2)
    b = W.sem_rhs(*mesh, 7)
    A = H.levels[0].apply_A
    x_ref, it_ref, _ = K.fcg(A, lambda q: M.vcycle(H, q), b, 1e-8)
    u = empty(len(b))
    code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, T(b), u, 1e-8, 200)
    assert code == cm.CHEBMG_OK and rel <= 1e-8 and abs(it - it_ref) <= 1, (it, it_ref)
    assert np.linalg.norm(b - A(N(u))) <= 1.01e-8 * np.linalg.norm(b)
    assert relerr(N(u), x_ref) < 1e-6
    s.close()


def test_fused_smoother_refused_where_it_does_not_apply():
    v = W.sem_box_vertices(2, 2, 2)
    s = solver(v, orders=(7, 3, 1), prec="mixed", lmax=[1.0, 1.0])
    for level, dt, variant in ((1, F64, 2), (2, F64, 2), (0, F64, 1), (0, F64, 3), (0, F32, 2)):
        with pytest.raises(cm.ChebmgError) as e:
            cm.chebmg_set_fused_smoother(s.ctx, level, dt, variant)
        assert e.value.code == cm.CHEBMG_EINVAL
    for level in (1, 2):
        assert cm.chebmg_fused_smoother(s.ctx, level, F64) == 0
    cm.chebmg_set_fused_smoother(s.ctx, 0, F64, 0)   # switching off is always allowed
    s.close()
    f = cm.Solver("fd2d", m=31, Lx=1.0, Ly=1.0, coarsening=2, coarsest=7, kind="opt4th", order=1,
                  sided="symmetric")
    with pytest.raises(cm.ChebmgError):
        cm.chebmg_set_fused_smoother(f.ctx, 0, F64, 2)
    f.close()


# ---- batches: a work item covers several right-hand sides (the geometric factors staged once) ----

def _rows(a):
    return T(np.ascontiguousarray(np.stack(a)))


@pytest.mark.parametrize("rhs_per_item", [1, 3, 8])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_fused_vcycle_matches_oracle(rhs_per_item, prec):
    mesh = (2, 3, 7)
    v = W.sem_box_vertices(*mesh)
    H = P.sem_hierarchy(v, (7, 3, 1), kind="opt4th", k=3, sided="one-sided")
    s = solver(v, k=3, sided="one-sided", prec=prec, lmax=[Lv.lmax for Lv in H.levels[:-1]])
    dt, var = (F32, 1) if prec == "mixed" else (F64, 2)
    nrhs = 7   # not a multiple of the group size: the last group is ragged
    R = [W.sem_rhs(*mesh, 7, seed=q) for q in range(nrhs)]
    Z = {}
    for v_ in (0, var):
        cm.chebmg_set_batch_fused_smoother(s.ctx, nrhs, 0, dt, v_, rhs_per_item)
        assert cm.chebmg_batch_fused_smoother(s.ctx, nrhs, 0, dt) == ((v_, rhs_per_item) if v_ else (0, 0))
        Z[v_] = torch.zeros((nrhs, len(R[0])), dtype=torch.float64, device="cuda")
        cm.chebmg_vcycle_batched(s.ctx, _rows(R), Z[v_])
    for q in range(nrhs):
        ref = M.vcycle(H, R[q])
        if prec == "fp64":
            assert relerr(N(Z[var][q]), ref) < 1e-8
            assert relerr(N(Z[var][q]), N(Z[0][q])) < 1e-8
        else:
            assert relerr(N(Z[var][q]), N(Z[0][q])) < 1e-5
            assert relerr(N(Z[var][q]), ref) < 1e-4
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_fused_solve_iterations_match_oracle(prec):
    mesh = (3, 4, 5)
    v = W.sem_box_vertices(*mesh)
    H = P.sem_hierarchy(v, (7, 3, 1), kind="opt4th", k=2, sided="one-sided")
    s = solver(v, k=2, sided="one-sided", prec=prec, lmax=[Lv.lmax for Lv in H.levels[:-1]])
    nrhs = 5
    cm.chebmg_set_batch_fused_smoother(s.ctx, nrhs, 0, F32 if prec == "mixed" else F64,
                                       1 if prec == "mixed" else 2, 4)
    A = H.levels[0].apply_A
    B = [W.sem_rhs(*mesh, 7, seed=q) for q in range(nrhs)]
    U = torch.zeros((nrhs, len(B[0])), dtype=torch.float64, device="cuda")
    code, its, rel = cm.chebmg_pcg_solve_batched(s.ctx, _rows(B), U, 1e-8, 200, graph=False)
    assert code == cm.CHEBMG_OK
    for q in range(nrhs):
        _, it_ref, _ = K.fcg(A, lambda r: M.vcycle(H, r), B[q], 1e-8)
        assert abs(its[q] - it_ref) <= 1 and rel[q] <= 1e-8
        assert np.linalg.norm(B[q] - A(N(U[q]))) <= 1.01e-8 * np.linalg.norm(B[q])
    s.close()
