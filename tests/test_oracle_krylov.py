"""Pins of the oracle's Krylov pieces: FCG, coarse PCG, GMRES, Lanczos, SplitMix64."""
import json
import os

import numpy as np
import pytest

from oracle import krylov as K
from oracle.fd import laplacian_5pt

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_outputs():
    gold = json.load(open(os.path.join(GOLD, "splitmix64.json")))
    got = [int(v) for v in K.splitmix64(gold["seed"], len(gold["outputs"]))]
    assert got == [int(v) for v in gold["outputs"]]
    u = K.splitmix64_uniform(42, 100000)
    assert u.min() >= -1 and u.max() < 1 and abs(u.mean()) < 0.01


def test_lanczos_on_known_spectrum():
    lam = np.linspace(0.1, 5.0, 400)
    got = K.lanczos_lmax(lambda v: lam * v, np.ones(400), steps=120)
    assert abs(got - 5.0) < 1e-6
    # S A with diagonal S: eigenvalues of diag(S) diag(a) are S*a
    a = np.linspace(1, 3, 300)
    S = 1 / np.linspace(1, 2, 300)
    assert abs(K.lanczos_lmax(lambda v: a * v, S, steps=150) - (a * S).max()) < 1e-8


def test_lanczos_fd_lambda_max_closed_form():
    m = 63
    A = laplacian_5pt(m, m, 1 / (m + 1), 1 / (m + 1))
    exact = 2 * np.sin(m * np.pi / (2 * (m + 1))) ** 2              # 1.998795456...
    S = 1 / A.diagonal()
    est30 = K.lanczos_lmax(lambda v: A @ v, S, steps=30)
    assert exact * 0.99 < est30 <= exact * (1 + 1e-12)
    est = K.lanczos_lmax(lambda v: A @ v, S, steps=300)
    assert abs(est - exact) < 1e-8


def test_pcg_jacobi_and_fcg_solve_spd():
    m = 20
    A = laplacian_5pt(m, m, 1 / (m + 1), 1 / (m + 1))
    b = np.random.default_rng(1).uniform(-1, 1, m * m)
    xd = np.linalg.solve(A.toarray(), b)
    x, it = K.pcg_jacobi(lambda v: A @ v, 1 / A.diagonal(), b, 1e-12)
    np.testing.assert_allclose(x, xd, rtol=1e-9, atol=1e-12)
    x2, it2, hist = K.fcg(lambda v: A @ v, lambda r: r / A.diagonal(), b, 1e-12)
    np.testing.assert_allclose(x2, xd, rtol=1e-9, atol=1e-12)
    assert abs(it2 - it) <= 1                      # FCG == PCG for a fixed SPD preconditioner
    assert hist[0] == 1.0 and hist[-1] <= 1e-12


def test_fcg_zero_rhs():
    x, it, hist = K.fcg(lambda v: v, lambda r: r, np.zeros(5))
    assert it == 0 and np.all(x == 0)


def test_gmres_matches_direct_solve_nonsymmetric():
    rng = np.random.default_rng(2)
    A = np.eye(60) * 4 + rng.uniform(-0.5, 0.5, (60, 60))
    b = rng.uniform(-1, 1, 60)
    x, it, hist = K.gmres(lambda v: A @ v, lambda r: r, b, rtol=1e-12, restart=20)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9)
    assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b) * 1.01


def test_not_converged_raises():
    A = laplacian_5pt(30, 30, 1 / 31, 1 / 31)
    with pytest.raises(K.NotConverged):
        K.pcg_jacobi(lambda v: A @ v, 1 / A.diagonal(), np.ones(900), 1e-12, maxit=3)


def test_polynomial_pcg_degree_one_is_jacobi_pcg_and_higher_degrees_cut_iterations():
    m = 31
    A = laplacian_5pt(m, m, 1 / (m + 1), 1 / (m + 1))
    S = 1 / A.diagonal()
    b = np.random.default_rng(5).uniform(-1, 1, m * m)
    lmax = K.lanczos_lmax(lambda v: A @ v, S, steps=60) * 1.01
    xj, itj = K.pcg_jacobi(lambda v: A @ v, S, b, 1e-10)
    x1, it1 = K.pcg_cheb4(lambda v: A @ v, S, b, lmax, 1, 1e-10)
    assert it1 == itj
    np.testing.assert_allclose(x1, xj, rtol=1e-8, atol=1e-12)
    xd = np.linalg.solve(A.toarray(), b)
    prev = itj
    for deg in (2, 4, 8):
        x, it = K.pcg_cheb4(lambda v: A @ v, S, b, lmax, deg, 1e-10)
        assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b) * 1.01
        np.testing.assert_allclose(x, xd, rtol=1e-7, atol=1e-10)
        assert it < prev
        prev = it
    # the degree-m preconditioner is SPD: its dense matrix is symmetric positive definite
    from oracle.chebyshev import chebyshev_4th
    n = 64
    A2 = laplacian_5pt(8, 8, 1 / 9, 1 / 9)
    S2 = 1 / A2.diagonal()
    l2 = K.lanczos_lmax(lambda v: A2 @ v, S2, steps=64)
    M = np.stack([chebyshev_4th(lambda v: A2 @ v, S2, np.eye(n)[i], 6, l2) for i in range(n)], axis=1)
    assert np.abs(M - M.T).max() < 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
