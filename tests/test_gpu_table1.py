"""The paper's FD study on the GPU (Sec. 3, Table 1): n = 128 (127 x 127 unknowns),
Lx in {1, 8, 64, 128}, coarsening by 2 (down to one unknown, 7 levels) and by 8 (3 levels),
the smoother and (m, n) of each row, restarted flexible GMRES(20) to 1e-6.

Each row must take the oracle's iteration count (within one; same lambda_max passed to both),
and with the GPU's own Lanczos lambda_max the rows the oracle reproduces exactly must take
the printed count.  Weights for the orders 18 and 20 (not in Table 5) come from
tests/golden/optimal_betas.json.  GMRES itself is also checked on an SEM problem.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import krylov as K
from oracle import multigrid as M
from oracle import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2210_03179_gb300 as cm  # noqa: E402
from gpu_util import N, T  # noqa: E402

HERE = os.path.dirname(__file__)
ROWS = json.load(open(os.path.join(HERE, "golden", "fd_table1.json")))["rows"]
BETAS = {int(k): v["betas"] for k, v in
         json.load(open(os.path.join(HERE, "golden", "optimal_betas.json")))["orders"].items()}


def cycle_shape(row):
    if row["n"] == 0:
        return row["m"] // 2, "one-sided"
    assert row["m"] == row["n"]
    return row["m"], "symmetric"


def gpu_solver(row, lmax=None):
    k, sided = cycle_shape(row)
    order = row["m"] + row["n"]
    kind = row["kind"] if order <= 16 else "4th"
    s = cm.Solver("fd2d", m=127, Lx=row["Lx"], Ly=1.0, coarsening=row["coarsening"], coarsest=1, kind=kind,
                  order=k, sided=sided, lmax=lmax)
    if order > 16:
        cm.chebmg_set_smoother_weights(s.ctx, BETAS[order], 1.0)
    return s


def rhs(row, A):
    n, m, Lx = 128, 127, row["Lx"]
    x = np.arange(1, m + 1) * (Lx / n)
    y = np.arange(1, m + 1) / n
    X, Y = np.meshgrid(x, y)
    g = np.random.default_rng(0).uniform(-1, 1, m * m)
    return A @ ((np.sin(3 * np.pi * X / Lx) * np.sin(4 * np.pi * Y)).ravel() + g)


@pytest.mark.parametrize("row", ROWS, ids=lambda r: f"Lx{r['Lx']}-c{r['coarsening']}-{r['kind']}-{r['m']}-{r['n']}")
def test_table1_row_on_gpu(row):
    order = row["m"] + row["n"]
    kind = row["kind"] if order <= 16 else "4th"
    H = P.fd_hierarchy(127, Lx=row["Lx"], Ly=1.0, c=row["coarsening"], coarsest=1, kind=kind, k=1,
                       sided="symmetric", pre=row["m"], post=row["n"])
    if order > 16:
        H.betas = {order: np.array(BETAS[order])}
    A = H.levels[0].A
    b = rhs(row, A)
    _, it_ref, _ = K.gmres(lambda v: A @ v, lambda r: M.vcycle(H, r), b, rtol=1e-6, restart=20)
    s = gpu_solver(row, lmax=[L.lmax for L in H.levels[:-1]])
    assert s.num_levels == len(H.levels)
    u = torch.zeros(127 * 127, dtype=torch.float64, device="cuda")
    code, it, rel, hist = cm.chebmg_gmres_solve(s.ctx, T(b), u, 1e-6, 20, 200, history=True)
    assert code == cm.CHEBMG_OK and rel <= 1e-6
    assert abs(it - it_ref) <= 1
    assert np.linalg.norm(b - A @ N(u)) <= 1.0001e-6 * np.linalg.norm(b)
    s.close()
    # the GPU's own lambda_max (Lanczos) on the rows the oracle reproduces exactly
    exact = not (row["kind"] == "opt4th" and (row["coarsening"] == 8 or order > 16))
    if exact:
        s = gpu_solver(row)
        u.zero_()
        code, it, rel, _ = cm.chebmg_gmres_solve(s.ctx, T(b), u, 1e-6, 20, 200)
        assert code == cm.CHEBMG_OK and it == row["iterations"]
        assert it * (order + 1) == row["matvecs"]
        s.close()


def test_gmres_sem_matches_oracle():
    v = W.sem_box_vertices(3, 4, 5)
    H = P.sem_hierarchy(v, (7, 3, 1), kind="opt4th", k=2, sided="one-sided")
    s = cm.Solver("sem", verts=v, orders=(7, 3, 1), kind="opt4th", order=2, sided="one-sided",
                  lmax=[L.lmax for L in H.levels[:-1]])
    b = W.sem_rhs(3, 4, 5, 7)
    A = H.levels[0].apply_A
    _, it_ref, hist_ref = K.gmres(A, lambda r: M.vcycle(H, r), b, rtol=1e-8, restart=20)
    u = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    code, it, rel, hist = cm.chebmg_gmres_solve(s.ctx, T(b), u, 1e-8, 20, 200, history=True)
    assert code == cm.CHEBMG_OK and abs(it - it_ref) <= 1 and rel <= 1e-8
    n = min(len(hist), len(hist_ref))
    np.testing.assert_allclose(hist[:n], hist_ref[:n], rtol=1e-5)
    # restarts: GMRES(3) needs several cycles and still reaches the tolerance
    u.zero_()
    code, it3, rel3, _ = cm.chebmg_gmres_solve(s.ctx, T(b), u, 1e-8, 3, 500)
    _, it3_ref, _ = K.gmres(A, lambda r: M.vcycle(H, r), b, rtol=1e-8, restart=3)
    assert code == cm.CHEBMG_OK and abs(it3 - it3_ref) <= 1 and rel3 <= 1e-8
    # maxit reached
    u.zero_()
    code, it1, rel1, _ = cm.chebmg_gmres_solve(s.ctx, T(b), u, 1e-14, 20, 2)
    assert code == cm.CHEBMG_ENOTCONV and it1 == 2
    s.close()
