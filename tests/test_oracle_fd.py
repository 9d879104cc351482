"""Pins of the oracle's 2-D FD operator, transfers and Galerkin hierarchy (Sec. 3)."""
import json
import os

import numpy as np
import pytest

from oracle import theory as T
from oracle.chebyshev import BETA_TABLE, chebyshev_1st, chebyshev_4th
from oracle.fd import DenseCholeskySolve, fd_levels, laplacian_5pt

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def mode(m, i, j):
    x = np.arange(1, m + 1) / (m + 1)
    return np.outer(np.sin(j * np.pi * x), np.sin(i * np.pi * x)).ravel()   # [y, x], x fastest


@pytest.mark.parametrize("m,Lx", [(15, 1.0), (63, 1.0), (31, 8.0)])
def test_sine_modes_are_eigenvectors(m, Lx):
    hx, hy = Lx / (m + 1), 1.0 / (m + 1)
    A = laplacian_5pt(m, m, hx, hy)
    for (i, j) in [(1, 1), (3, 4), (m, m), (2, m - 1)]:
        v = mode(m, i, j)
        lam = 4 / hx ** 2 * np.sin(i * np.pi / (2 * (m + 1))) ** 2 + 4 / hy ** 2 * np.sin(j * np.pi / (2 * (m + 1))) ** 2
        np.testing.assert_allclose(A @ v, lam * v, atol=1e-9 * lam)


@pytest.mark.parametrize("kind,k", [("1st", 3), ("4th", 2), ("4th", 5), ("opt4th", 4)])
def test_one_smoother_application_scales_each_mode(kind, k):
    # D is constant, so S A has the sine modes as eigenvectors with mu = sin^2 + sin^2 and
    # one smoother application multiplies mode (i,j) by exactly p_k(mu / lambda_max).
    m = 31
    A = laplacian_5pt(m, m, 1 / (m + 1), 1 / (m + 1))
    S = 1.0 / A.diagonal()
    lmax = 2 * np.sin(m * np.pi / (2 * (m + 1))) ** 2
    for (i, j) in [(1, 1), (5, 9), (20, 3), (31, 31)]:
        e = mode(m, i, j)
        mu = np.sin(i * np.pi / (2 * (m + 1))) ** 2 + np.sin(j * np.pi / (2 * (m + 1))) ** 2
        b = A @ e
        if kind == "1st":
            x = chebyshev_1st(lambda v: A @ v, S, b, k, lmax, 0.1 * lmax)
        else:
            x = chebyshev_4th(lambda v: A @ v, S, b, k, lmax,
                              betas=np.array(BETA_TABLE[k]) if kind == "opt4th" else None)
        p = T.smoothing_polynomial(kind, k, np.array([mu / lmax]))[0]
        np.testing.assert_allclose(e - x, p * e, atol=1e-12)


def test_grid_complexity_matches_paper():
    gold = json.load(open(os.path.join(GOLD, "fd_grid_complexity.json")))
    n = gold["n"]
    for case in gold["cases"]:
        levels, _ = fd_levels(n - 1, 1.0, 1.0, case["coarsening"], 1)
        assert len(levels) == case["levels"]
        assert levels[-1].n == 1
        assert round(T.grid_complexity([L.nnz() for L in levels]), 3) == case["complexity"]


def test_galerkin_coarse_operator_is_symmetric_nine_point():
    levels, transfers = fd_levels(63, 1.0, 1.0, 2, 7)
    assert [L.mx for L in levels] == [63, 31, 15, 7]
    for L in levels[1:]:
        A = L.A.toarray()
        assert np.abs(A - A.T).max() < 1e-10 * np.abs(A).max()
        c = L.mx // 2
        row = A[c * L.mx + c].reshape(L.my, L.mx)
        nz = np.argwhere(np.abs(row) > 1e-12 * np.abs(row).max())
        assert len(nz) == 9 and np.all(np.abs(nz - c) <= 1)
        np.testing.assert_allclose(row.sum(), 0.0, atol=1e-10 * row[c, c])   # constants in the kernel
    # first Galerkin level: textbook stencil (3, -1/2, -1/4) / h_f^2 for bilinear P and R = P^T
    L = levels[1]
    c = L.mx // 2
    row = L.A.toarray()[c * L.mx + c].reshape(L.my, L.mx)
    np.testing.assert_allclose(row[c - 1:c + 2, c - 1:c + 2] / 64.0 ** 2,
                               [[-0.25, -0.5, -0.25], [-0.5, 3.0, -0.5], [-0.25, -0.5, -0.25]], atol=1e-12)


def test_dense_coarse_solve_is_exact():
    levels, _ = fd_levels(15, 1.0, 1.0, 2, 7)
    Ac = levels[-1].A
    b = np.random.default_rng(0).uniform(-1, 1, Ac.shape[0])
    x = DenseCholeskySolve(Ac)(b)
    np.testing.assert_allclose(Ac @ x, b, atol=1e-12)
