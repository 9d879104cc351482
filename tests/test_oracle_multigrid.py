"""Pins of the oracle's V-cycle against the dense error propagators of Sec. 2."""
import numpy as np
import pytest

import workloads as W
from oracle import krylov as K
from oracle import multigrid as M
from oracle import problems as Pr
from oracle import theory as T
from oracle.chebyshev import BETA_TABLE
from oracle.fd import fd_levels
from oracle.krylov import pcg_jacobi


def fourth_W(k, x):
    t = np.arccos(np.clip(x, -1, 1))
    return np.sin((k + 0.5) * t) / np.sin(t / 2)


def poly(kind, k, mu, lmin_ratio=0.1):
    """Closed-form smoothing polynomials (not the smoother code)."""
    if k == 0:
        return np.ones_like(mu)
    if kind == "1st":
        th, de = (1 + lmin_ratio) / 2, (1 - lmin_ratio) / 2
        return T.cheb_T(k, (th - mu) / de) / T.cheb_T(k, th / de)
    p = [np.ones_like(mu)] + [fourth_W(i, 1 - 2 * mu) / (2 * i + 1) for i in range(1, k + 1)]
    if kind == "4th":
        return p[k]
    beta = np.array(BETA_TABLE[k])
    return 1 - sum(beta[i - 1] * (p[i - 1] - p[i]) for i in range(1, k + 1))


def dense_smoother(A, S, lmax, kind, k):
    s = np.sqrt(S)
    Mm = (s[:, None] * A * s[None, :]) / lmax
    mu, U = np.linalg.eigh(Mm)
    return (s[:, None] * U) @ np.diag(poly(kind, k, mu)) @ (U.T / s[None, :])


def dense_cycle(levels, Ps, kind, m, n, j=0):
    """B_j from E_j = G'_j (I - P B_{j+1} P^T A_j) G_j (Eq. 2.2), B_l = A_l^{-1}."""
    A = levels[j].dense_A
    if j == len(levels) - 1:
        return np.linalg.inv(A)
    Bc = dense_cycle(levels, Ps, kind, m, n, j + 1)
    L = levels[j]
    G = dense_smoother(A, L.invD, L.lmax, kind, m)
    Gp = dense_smoother(A, L.invD, L.lmax, kind, n)
    P = Ps[j]
    E = Gp @ (np.eye(len(A)) - P @ Bc @ P.T @ A) @ G
    return (np.eye(len(A)) - E) @ np.linalg.inv(A)


def exact_lmax_fd(m, c, coarsest):
    levels, _ = fd_levels(m, 1.0, 1.0, c, coarsest)
    out = []
    for L in levels[:-1]:
        A = L.A.toarray()
        d = np.sqrt(np.diag(A))
        out.append(np.linalg.eigvalsh(A / d[:, None] / d[None, :]).max())
    return out


def cycle_matrix(H):
    n = H.levels[0].n
    return np.stack([M.vcycle(H, np.eye(n)[i]) for i in range(n)], axis=1)


@pytest.mark.parametrize("kind", ["1st", "4th", "opt4th"])
@pytest.mark.parametrize("k,sided", [(1, "symmetric"), (2, "symmetric"), (2, "one-sided"), (3, "one-sided")])
def test_fd_vcycle_equals_dense_error_propagator(kind, k, sided):
    # exact lambda_max keeps every mu = eig(SA)/lambda_max in (0, 1], where the closed forms hold
    H = Pr.fd_hierarchy(15, c=2, coarsest=3, kind=kind, k=k, sided=sided, lmax=exact_lmax_fd(15, 2, 3))
    for L in H.levels:
        L.dense_A = L.A.toarray()
    B = cycle_matrix(H)
    Bref = dense_cycle(H.levels, [T_.P.toarray() for T_ in H.transfers], kind, H.pre, H.post)
    assert np.abs(B - Bref).max() < 1e-11 * np.abs(Bref).max()
    if sided == "symmetric":
        assert np.abs(B - B.T).max() < 1e-13 * np.abs(B).max()
    else:
        assert np.abs(B - B.T).max() > 1e-6 * np.abs(B).max()


def test_sem_vcycle_equals_dense_error_propagator():
    v = W.sem_box_vertices(2, 2, 2)
    for kind, k, sided in [("opt4th", 2, "symmetric"), ("4th", 1, "one-sided"), ("1st", 2, "symmetric")]:
        H = Pr.sem_hierarchy(v, (4, 2, 1), kind=kind, k=k, sided=sided, lmax=[1.0, 1.0])
        for L in H.levels[:-1]:
            lv = ~L.dirichlet
            A = L.dense()[np.ix_(lv, lv)]
            d = np.sqrt(np.diag(A))
            L.lmax = np.linalg.eigvalsh(A / d[:, None] / d[None, :]).max()
        live = [~L.dirichlet for L in H.levels]
        for L, lv in zip(H.levels, live):
            L.dense_A = L.dense()[np.ix_(lv, lv)]
            L.invD = L.invD   # keep the full-length vector for the cycle
        # dense pieces on the live (non-Dirichlet) unknowns
        Ps = []
        for j, Tr in enumerate(H.transfers):
            nc = H.levels[j + 1].n
            P = np.stack([Tr.prolong(np.eye(nc)[g]) for g in range(nc)], axis=1)
            Ps.append(P[np.ix_(live[j], live[j + 1])])

        class Lv:
            pass
        red = []
        for L, lv in zip(H.levels, live):
            r = Lv()
            r.dense_A, r.invD, r.lmax = L.dense_A, L.invD[lv], getattr(L, "lmax", None)
            red.append(r)
        Bref = dense_cycle(red, Ps, kind, H.pre, H.post)
        n0 = H.levels[0].n
        idx = np.flatnonzero(live[0])
        B = np.stack([M.vcycle(H, np.eye(n0)[i])[idx] for i in idx], axis=1)
        assert np.abs(B - Bref).max() < 1e-10 * np.abs(Bref).max()
        if sided == "symmetric":
            assert np.abs(B - B.T).max() < 1e-12 * np.abs(B).max()


@pytest.mark.parametrize("kind", ["1st", "4th", "opt4th"])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_two_level_contraction_obeys_lemma_bound(kind, k):
    # Lemma 2.1 with one smoothed level: ||E_down||_A^2 <= C / (C + gamma^{-1}), S scaled so rho(SA) = 1,
    # C from Eq. 2.10 as a generalized eigenproblem, exact Galerkin coarse solve.
    levels, transfers = fd_levels(15, 1.0, 1.0, 2, 7)
    A = levels[0].A.toarray()
    P = transfers[0].P.toarray()
    Ac = levels[1].A.toarray()
    D = np.diag(A)
    lmax = np.linalg.eigvalsh(A / np.sqrt(D)[:, None] / np.sqrt(D)[None, :]).max()
    S = 1.0 / (D * lmax)
    Kc = np.linalg.inv(A) - P @ np.linalg.inv(Ac) @ P.T
    # Eq. 2.10: C = sup f^T K A K f / f^T S f with K A K = K for a Galerkin coarse space,
    # i.e. the largest eigenvalue of S^{-1/2} K S^{-1/2}
    s = np.sqrt(S)
    C = np.linalg.eigvalsh(Kc / s[:, None] / s[None, :]).max()
    G = dense_smoother(A, 1.0 / D, lmax, kind, k)
    E = (np.eye(len(A)) - P @ np.linalg.inv(Ac) @ P.T @ A) @ G
    Ah = np.linalg.cholesky(A).T                     # ||E||_A = ||Ah E Ah^{-1}||_2
    normA = np.linalg.norm(Ah @ E @ np.linalg.inv(Ah), 2)
    bound = C / (C + T.gamma_inv(kind, k))
    assert normA ** 2 <= bound * (1 + 1e-8)
    assert C > 1.0


def test_observed_rate_matches_spectral_radius():
    # Eq. 3.1 for MG as a stationary solver: rho_obs -> spectral radius of I - B A.
    H = Pr.fd_hierarchy(15, c=2, coarsest=3, kind="4th", k=1, sided="symmetric")
    A = H.levels[0].A.toarray()
    B = cycle_matrix(H)
    rho = np.abs(np.linalg.eigvals(np.eye(len(A)) - B @ A)).max()
    b = W.fd_rhs(15)
    x = np.zeros_like(b)
    r0 = np.linalg.norm(b)
    N = 40
    for _ in range(N):
        x = x + M.vcycle(H, b - A @ x)
    rN = np.linalg.norm(b - A @ x)
    rho_obs = np.exp(np.log(rN / r0) / N)
    assert abs(rho_obs - rho) < 0.1 * rho


@pytest.mark.parametrize("sided", ["symmetric", "one-sided"])
def test_fcg_solution_matches_direct_solve(sided):
    H = Pr.fd_hierarchy(31, c=2, coarsest=7, kind="opt4th", k=2, sided=sided)
    A = H.levels[0].A
    b = W.fd_rhs(31)
    x, it, hist = K.fcg(lambda v: A @ v, lambda r: M.vcycle(H, r), b, 1e-8)
    xd = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)
    assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
    assert 2 <= it <= 20 and len(hist) == it + 1
