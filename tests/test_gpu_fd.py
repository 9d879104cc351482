"""GPU-vs-oracle parity for the 2-D FD path (Sec. 3): stencil, transfers, smoothers, V-cycle, solve."""
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


def make(m=63, Lx=1.0, c=2, coarsest=7, kind="opt4th", k=2, sided="one-sided", prec="fp64"):
    H = P.fd_hierarchy(m, Lx=Lx, c=c, coarsest=coarsest, kind=kind, k=k, sided=sided)
    lmax = [L.lmax for L in H.levels[:-1]]
    s = cm.Solver("fd2d", m=m, Lx=Lx, coarsening=c, coarsest=coarsest, kind=kind, order=k, sided=sided,
                  prec=prec, lmax=lmax)
    return H, s


@pytest.mark.parametrize("m,Lx,c,coarsest", [(63, 1.0, 2, 7), (127, 8.0, 2, 1), (127, 64.0, 8, 1), (31, 1.0, 2, 3)])
def test_operator_transfers_and_diagonal(m, Lx, c, coarsest):
    H, s = make(m, Lx, c, coarsest)
    assert s.num_levels == len(H.levels)
    rng = np.random.default_rng(11)
    for j, L in enumerate(H.levels):
        assert s.size(j) == L.n
        x = rng.uniform(-1, 1, L.n)
        y = empty(L.n)
        cm.chebmg_apply_A(s.ctx, j, F64, T(x), y)
        assert relerr(N(y), L.apply_A(x)) < 1e-12
        d = empty(L.n)
        cm.chebmg_inv_diagonal(s.ctx, j, F64, d)
        assert relerr(N(d), L.invD) < 1e-13
    for j, Tr in enumerate(H.transfers):
        nf, nc = H.levels[j].n, H.levels[j + 1].n
        rf = rng.uniform(-1, 1, nf)
        rc = empty(nc)
        cm.chebmg_restrict(s.ctx, j, F64, T(rf), rc)
        assert relerr(N(rc), Tr.restrict(rf)) < 1e-13
        zc = rng.uniform(-1, 1, nc)
        zf = T(rng.uniform(-1, 1, nf))
        base = N(zf)
        cm.chebmg_prolong(s.ctx, j, F64, T(zc), zf, accumulate=True)
        assert relerr(N(zf), base + Tr.prolong(zc)) < 1e-13
        cm.chebmg_prolong(s.ctx, j, F64, T(zc), zf, accumulate=False)
        assert relerr(N(zf), Tr.prolong(zc)) < 1e-13
    s.close()


@pytest.mark.parametrize("kind", ["1st", "4th", "opt4th"])
@pytest.mark.parametrize("order", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("x_zero", [True, False])
def test_smoother_matches_algorithms(kind, order, x_zero):
    H, s = make(63, kind=kind)
    rng = np.random.default_rng(order)
    for j in range(len(H.levels) - 1):
        L = H.levels[j]
        b = rng.uniform(-1, 1, L.n)
        x0 = None if x_zero else rng.uniform(-1, 1, L.n)
        ref = oracle_smooth(L, b, order, kind, L.lmax, 0.1, x0=x0)
        x = empty(L.n) if x_zero else T(x0)
        cm.chebmg_smooth(s.ctx, j, F64, T(b), x, order, x_zero)
        assert relerr(N(x), ref) < 1e-12, (j, relerr(N(x), ref))
    s.close()


def test_coarse_solve_and_lanczos():
    H, s = make(63)
    Lc = H.levels[-1]
    r = np.random.default_rng(3).uniform(-1, 1, Lc.n)
    z = empty(Lc.n)
    cm.chebmg_coarse_solve(s.ctx, T(r), z)
    assert relerr(N(z), np.linalg.solve(Lc.A.toarray(), r)) < 1e-12
    s.close()
    # lambda_max by the library's own Lanczos (same SplitMix64 start vector, 30 steps)
    s = cm.Solver("fd2d", m=63, coarsening=2, coarsest=7, kind="opt4th", order=2, sided="one-sided")
    for j, L in enumerate(H.levels[:-1]):
        ref = K.lanczos_lmax(L.apply_A, L.invD, 30)
        assert abs(s.lambda_max(j) / ref - 1) < 1e-10
    assert abs(s.lambda_max(0) - 2 * np.sin(63 * np.pi / 128) ** 2) < 0.01
    s.close()


@pytest.mark.parametrize("kind", ["1st", "4th", "opt4th"])
@pytest.mark.parametrize("k,sided", [(1, "symmetric"), (2, "symmetric"), (2, "one-sided"), (4, "one-sided")])
def test_vcycle_matches_error_propagator(kind, k, sided):
    H, s = make(63, kind=kind, k=k, sided=sided)
    r = W.fd_rhs(63, seed=5)
    z = empty(len(r))
    cm.chebmg_vcycle(s.ctx, T(r), z)
    assert relerr(N(z), M.vcycle(H, r)) < 1e-12
    s.close()


@pytest.mark.parametrize("kind", ["1st", "4th", "opt4th"])
@pytest.mark.parametrize("k,sided", [(2, "symmetric"), (4, "one-sided"), (2, "one-sided")])
def test_pcg_solve_iterations_match(kind, k, sided):
    H, s = make(63, kind=kind, k=k, sided=sided)
    b = W.fd_rhs(63)
    A = H.levels[0].apply_A
    x_ref, it_ref, hist_ref = K.fcg(A, lambda r: M.vcycle(H, r), b, 1e-8)
    u = empty(len(b))
    code, it, rel, hist = cm.chebmg_pcg_solve(s.ctx, T(b), u, 1e-8, 200, history=True)
    assert code == cm.CHEBMG_OK
    assert abs(it - it_ref) <= 1
    assert rel <= 1e-8
    true_rel = np.linalg.norm(b - A(N(u))) / np.linalg.norm(b)
    assert true_rel <= 1.01e-8
    assert relerr(N(u), x_ref) < 1e-7
    n = min(len(hist), len(hist_ref))
    np.testing.assert_allclose(hist[:n], hist_ref[:n], rtol=1e-6)
    s.close()


def test_mixed_precision_fd_solve():
    H, s = make(63, prec="mixed")
    b = W.fd_rhs(63)
    _, it_ref, _ = K.fcg(H.levels[0].apply_A, lambda r: M.vcycle(H, r), b, 1e-8)
    u = empty(len(b))
    code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, T(b), u, 1e-8, 200)
    assert code == cm.CHEBMG_OK and rel <= 1e-8 and abs(it - it_ref) <= 1
    # FP32 operator against the FP64 oracle: single-precision rounding only
    L = H.levels[0]
    x = np.random.default_rng(1).uniform(-1, 1, L.n)
    y = empty(L.n, f32=True)
    cm.chebmg_apply_A(s.ctx, 0, F32, T(x, torch.float32), y)
    assert relerr(N(y), L.apply_A(x.astype(np.float32).astype(np.float64))) < 1e-5
    s.close()


def test_zero_rhs_and_errors():
    H, s = make(15, coarsest=3)
    b = empty(225)
    u = T(np.ones(225))
    code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, b, u, 1e-8, 10)
    assert code == cm.CHEBMG_OK and it == 0 and float(u.abs().max()) == 0.0
    code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, T(W.fd_rhs(15)), u, 1e-14, 1)
    assert code == cm.CHEBMG_ENOTCONV and it == 1 and rel > 1e-14
    nc = H.levels[-1].n
    with pytest.raises(cm.ChebmgError) as e:
        cm.chebmg_smooth(s.ctx, len(H.levels) - 1, F64, empty(nc), empty(nc), 2, True)   # not smoothed
    assert e.value.code == cm.CHEBMG_EINVAL
    with pytest.raises(cm.ChebmgError):
        cm.chebmg_apply_A(s.ctx, 0, F32, empty(225, True), empty(225, True))  # FP64-only context
    s.close()


def test_smoother_accepts_unaligned_caller_vectors():
    # caller vectors that are views at an odd offset take the scalar path of the update kernels
    H, s = make(63, kind="opt4th")
    L = H.levels[0]
    b = W.fd_rhs(63, seed=8)
    ref = oracle_smooth(L, b, 4, "opt4th", L.lmax, 0.1, x0=None)
    big = torch.zeros(L.n + 1, device="cuda:0", dtype=torch.float64)
    x = big[1:]
    assert x.data_ptr() % 16 != 0
    cm.chebmg_smooth(s.ctx, 0, F64, T(b), x, 4, True)
    assert relerr(N(x), ref) < 1e-12
    s.close()
