"""The 1st-kind smoother with the gamma^{-1}-optimal lambda_min (Sec. 2.4, Eq. 2.24) and the SEM
p-multigrid schedule 7 -> 5 -> 3 -> 1 (nekRS's, Sec. 4.1), against the oracle."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import workloads as W
from oracle import krylov as K
from oracle import multigrid as M
from oracle import problems as P
from oracle import theory as TH

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2210_03179_gb300 as cm  # noqa: E402
from gpu_util import N, T, relerr  # noqa: E402

MESH = (3, 4, 5)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 10])
def test_optimal_lambda_min_ratio(k):
    s = cm.Solver("fd2d", m=15, coarsest=3, kind="1st", order=1, sided="symmetric", lmin_ratio=0.0)
    ratio = cm.chebmg_lambda_min_ratio(s.ctx, k)
    res = minimize_scalar(lambda lm: -TH.gamma_inv("1st", k, lmin_ratio=lm), bounds=(1e-3, 0.6),
                          method="bounded", options={"xatol": 1e-7})
    # the library's ratio is the oracle's maximiser of gamma^{-1} (whose own sup evaluation is
    # accurate to a few 1e-6), and attains its optimal value
    assert abs(ratio - res.x) <= 1e-5 * res.x
    assert TH.gamma_inv("1st", k, lmin_ratio=ratio) >= -res.fun * (1 - 1e-5)
    # and follows the paper's correlation (Eq. 2.24) as closely as the oracle's optimum does
    ref = TH.lambda_min_opt_correlation(k)
    assert abs(ratio - ref) <= 0.01 * ref + 2e-3
    s.close()


def test_fixed_ratio_is_reported_unchanged():
    s = cm.Solver("fd2d", m=15, coarsest=3, kind="1st", order=2, sided="symmetric", lmin_ratio=0.1)
    assert cm.chebmg_lambda_min_ratio(s.ctx, 2) == 0.1
    s.close()


@pytest.mark.parametrize("k,sided", [(2, "symmetric"), (2, "one-sided"), (3, "symmetric")])
def test_fd_cycle_and_solve_with_optimal_lambda_min(k, sided):
    s0 = cm.Solver("fd2d", m=63, kind="1st", order=k, sided=sided, lmin_ratio=0.0, lmax=[1.0] * 3)
    pre = 2 * k if sided == "one-sided" else k
    ratio = cm.chebmg_lambda_min_ratio(s0.ctx, pre)
    s0.close()
    H = P.fd_hierarchy(63, kind="1st", k=k, sided=sided, lmin_ratio=ratio)
    s = cm.Solver("fd2d", m=63, kind="1st", order=k, sided=sided, lmin_ratio=0.0,
                  lmax=[L.lmax for L in H.levels[:-1]])
    r = W.fd_rhs(63, seed=3)
    z = torch.zeros(3969, dtype=torch.float64, device="cuda")
    cm.chebmg_vcycle(s.ctx, T(r), z)
    assert relerr(N(z), M.vcycle(H, r)) < 1e-12
    b = W.fd_rhs(63)
    _, it_ref, _ = K.fcg(H.levels[0].apply_A, lambda v: M.vcycle(H, v), b, 1e-8)
    u = torch.zeros_like(z)
    code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, T(b), u, 1e-8, 200)
    assert code == cm.CHEBMG_OK and abs(it - it_ref) <= 1 and rel <= 1e-8
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sem_schedule_7531(prec):
    v = W.sem_box_vertices(*MESH)
    H = P.sem_hierarchy(v, (7, 5, 3, 1), kind="opt4th", k=2, sided="one-sided")
    s = cm.Solver("sem", verts=v, orders=(7, 5, 3, 1), kind="opt4th", order=2, sided="one-sided", prec=prec,
                  lmax=[L.lmax for L in H.levels[:-1]])
    assert s.num_levels == 4
    r = W.sem_rhs(*MESH, 7, seed=6)
    z = torch.zeros(len(r), dtype=torch.float64, device="cuda")
    cm.chebmg_vcycle(s.ctx, T(r), z)
    assert relerr(N(z), M.vcycle(H, r)) < (1e-8 if prec == "fp64" else 1e-5)
    b = W.sem_rhs(*MESH, 7)
    A = H.levels[0].apply_A
    _, it_ref, _ = K.fcg(A, lambda q: M.vcycle(H, q), b, 1e-8)
    u = torch.zeros_like(z)
    code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, T(b), u, 1e-8, 200)
    assert code == cm.CHEBMG_OK and abs(it - it_ref) <= 1 and rel <= 1e-8
    assert np.linalg.norm(b - A(N(u))) <= 1.01e-8 * np.linalg.norm(b)
    s.close()
