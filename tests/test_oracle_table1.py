"""Pin of the whole oracle pipeline (smoothers, V-cycles, Galerkin hierarchy down to one unknown)
against the paper's Table 1 (Sec. 3): fewest fine mat-vecs for the FD problem with n = 128,
GMRES(20) to a 1e-6 relative residual, u = sin(3 pi x / Lx) sin(4 pi y) + g.

All eight rows; for the smoothing orders 18 and 20, which Table 5 (which stops at 16) does
not list, the weights come from the oracle's gamma^{-1} maximisation (it reproduces Table 5).
The paper states neither lambda_max's estimator nor g; with the 30-step Lanczos estimate and
g = uniform[-1,1] from seed 0 the oracle gives the printed iteration counts for three rows
exactly; the aggressive-coarsening optimized row is sensitive to lambda_max (11 iterations with
an accurate estimate, 13 -- the paper's value -- with a 10-step estimate 1% low), so it is
held to within 2, as are the optimized rows of orders 18 and 20 (11, 11, 15, 12 against the
printed 12, 12, 17, 14).
"""
import json
import os

import numpy as np
import pytest

from oracle import krylov as K
from oracle import multigrid as M
from oracle import problems as P

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fd_table1.json")))
ROWS = GOLD["rows"]
# weights for the smoothing orders 18 and 20, which Table 5 does not list (written by
# tests/golden/make_optimal_betas.py from the oracle's gamma^{-1} maximisation)
BETAS = {int(k): np.array(v["betas"]) for k, v in
         json.load(open(os.path.join(os.path.dirname(__file__), "golden", "optimal_betas.json")))["orders"].items()}


@pytest.mark.parametrize("row", ROWS, ids=lambda r: f"Lx{r['Lx']}-c{r['coarsening']}-{r['kind']}-{r['m']}-{r['n']}")
def test_table1_iterations_and_matvecs(row):
    n = 128
    m = n - 1
    Lx, c = row["Lx"], row["coarsening"]
    order = row["m"] + row["n"]
    kind = row["kind"] if order <= 16 else "4th"
    H = P.fd_hierarchy(m, Lx=Lx, Ly=1.0, c=c, coarsest=1, kind=kind, k=1, sided="symmetric",
                       pre=row["m"], post=row["n"])
    if order > 16:
        H.betas = {order: BETAS[order]}
    assert abs(sum(L.nnz() for L in H.levels) / H.levels[0].nnz() - row["complexity"]) < 5e-4
    x = np.arange(1, m + 1) * (Lx / n)
    y = np.arange(1, m + 1) / n
    X, Y = np.meshgrid(x, y)
    A = H.levels[0].A
    g = np.random.default_rng(0).uniform(-1, 1, m * m)
    b = A @ ((np.sin(3 * np.pi * X / Lx) * np.sin(4 * np.pi * Y)).ravel() + g)
    _, it, hist = K.gmres(lambda v: A @ v, lambda r: M.vcycle(H, r), b, rtol=1e-6, restart=20)
    assert hist[-1] <= 1e-6
    matvecs = it * (row["m"] + row["n"] + 1)      # one V-cycle (m+n fine mat-vecs) + one GMRES product
    if row["kind"] == "opt4th" and (row["coarsening"] == 8 or order > 16):
        assert abs(it - row["iterations"]) <= 2
    else:
        assert it == row["iterations"] and matvecs == row["matvecs"]
