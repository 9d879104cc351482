"""Pins of the oracle's error-ratio gradient (the target of the GPU adjoint).

The gradient comes from forward-mode propagation through Algorithm 2 and Eq. 2.2; it is
checked against central finite differences (h = 1e-6) of the objective computed by separate
code (the plain smoother and V-cycle, themselves pinned against the paper elsewhere), and the
objective is checked against special cases that fix it exactly.
"""
import numpy as np
import pytest

import workloads as W
from oracle import problems as P
from oracle import sensitivity as SE
from oracle.chebyshev import optimized_betas


def fd_h(m=15, k=4, sided="symmetric", kind="opt4th"):
    return P.fd_hierarchy(m, coarsest=3, kind=kind, k=k, sided=sided)


def exact_coarse(H):
    Lc = H.levels[-1]
    live = ~Lc.dirichlet
    Ainv = np.linalg.inv(Lc.dense()[np.ix_(live, live)])

    def solve(r):
        z = np.zeros_like(r)
        z[live] = Ainv @ r[live]
        return z
    H.coarse_solve = solve
    return H


def central_fd(H, E0, betas, s, h=1e-6):
    p = np.concatenate([betas, [s]])
    g = np.zeros_like(p)
    for i in range(len(p)):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        g[i] = (SE.error_ratio(H, E0, pp[:-1], pp[-1]) - SE.error_ratio(H, E0, pm[:-1], pm[-1])) / (2 * h)
    return g


@pytest.mark.parametrize("k,sided,betas,s", [
    (4, "symmetric", None, 1.0),           # the paper's optimized weights (Table 5)
    (4, "symmetric", np.ones(4), 1.1),     # 4th kind, lambda_max over-estimated by 10%
    (2, "one-sided", None, 0.95),          # one-sided (4,0): four weights, lambda_max 5% low
])
def test_fd_gradient_matches_central_differences(k, sided, betas, s):
    H = fd_h(15, k=k, sided=sided)
    order = H.pre
    b = optimized_betas(order) if betas is None else np.asarray(betas, float)
    E0 = W.random_vectors(H.levels[0].n, 3, seed=5)
    f, g = SE.error_ratio_and_gradient(H, E0, b, s)
    assert f == pytest.approx(SE.error_ratio(H, E0, b, s), rel=1e-12)
    g_fd = central_fd(H, E0, b, s)
    assert np.abs(g - g_fd).max() <= 1e-6 * np.abs(g).max()
    assert len(g) == order + 1


def test_sem_gradient_matches_central_differences():
    v = W.sem_box_vertices(2, 2, 2)
    H = exact_coarse(P.sem_hierarchy(v, (4, 2, 1), kind="4th", k=3, sided="symmetric"))
    live = ~H.levels[0].dirichlet
    E0 = W.random_vectors(H.levels[0].n, 2, seed=9) * live[None, :]
    b = np.array([1.0, 1.1, 1.3])
    f, g = SE.error_ratio_and_gradient(H, E0, b, 1.05)
    assert f == pytest.approx(SE.error_ratio(H, E0, b, 1.05), rel=1e-12)
    g_fd = central_fd(H, E0, b, 1.05)
    assert np.abs(g - g_fd).max() <= 1e-6 * np.abs(g).max()


def test_zero_weights_leave_only_the_coarse_correction():
    # beta = 0: the smoothers do nothing, E = I - P A_c^{-1} P^T A at two levels; E is then an
    # A-orthogonal projector, so applying it three times equals applying it once, and the
    # derivative with respect to the lambda_max scale vanishes.
    H = P.fd_hierarchy(15, coarsest=7, kind="4th", k=2, sided="symmetric")
    assert len(H.levels) == 2
    E0 = W.random_vectors(H.levels[0].n, 2, seed=3)
    f1 = SE.error_ratio(H, E0, np.zeros(2), 1.0, steps=1)
    f3, g = SE.error_ratio_and_gradient(H, E0, np.zeros(2), 1.0, steps=3)
    assert f3 == pytest.approx(f1, rel=1e-10)
    assert abs(g[-1]) < 1e-12


def test_single_level_cycle_is_exact():
    # one level: the cycle is the exact coarse solve, B = A^{-1}, E = 0 for every weight
    H = P.fd_hierarchy(7, coarsest=7, kind="4th", k=2, sided="symmetric")
    assert len(H.levels) == 1
    E0 = W.random_vectors(H.levels[0].n, 2, seed=1)
    f, g = SE.error_ratio_and_gradient(H, E0, np.ones(2), 1.0, steps=1)
    assert f < 1e-24 and np.abs(g).max() < 1e-12


def test_ratio_is_invariant_to_the_size_of_e0():
    H = fd_h(15, k=2)
    E0 = W.random_vectors(H.levels[0].n, 2, seed=4)
    b = optimized_betas(2)
    assert SE.error_ratio(H, 7.0 * E0, b, 1.0) == pytest.approx(SE.error_ratio(H, E0, b, 1.0), rel=1e-12)


def test_rejects_weights_of_the_wrong_length():
    H = fd_h(15, k=2)
    with pytest.raises(ValueError):
        SE.error_ratio_and_gradient(H, W.random_vectors(H.levels[0].n, 1, seed=0), np.ones(3), 1.0)
