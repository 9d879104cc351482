"""Gauss-Lobatto-Legendre (GLL) basis for the spectral-element discretisation.

Test infrastructure only (see ``oracle/__init__``).

The SEM operator of the paper (Sec. 1, a_ij = int grad(phi_i).grad(phi_j) dV,
with the SEM details deferred to its reference on nekRS) uses tensor-product
Lagrange bases on the N+1 GLL points of [-1,1] and GLL quadrature.

* nodes: -1, +1 and the N-1 roots of P_N'(x), found by Newton's method from
  Chebyshev-Gauss-Lobatto guesses;
* weights: w_j = 2 / (N (N+1) P_N(x_j)^2);
* derivative matrix: D[i,j] = l_j'(x_i) from barycentric weights;
* interpolation matrix: J[a,b] = l_b(y_a) for Lagrange basis l_b on nodes x.
"""
from __future__ import annotations

import numpy as np


def legendre(N: int, x):
    """P_N(x) and P_N'(x) by the three-term recurrence (Bonnet) and its derivative."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if N == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for n in range(2, N + 1):
        p0, p1 = p1, ((2 * n - 1) * x * p1 - (n - 1) * p0) / n
    # (1 - x^2) P_N'(x) = N (P_{N-1}(x) - x P_N(x)); valid away from x = +-1
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = N * (p0 - x * p1) / (1.0 - x * x)
    end = np.abs(x) == 1.0
    if np.any(end):
        dp = np.where(end, np.sign(x) ** (N + 1) * N * (N + 1) / 2.0, dp)
    return p1, dp


def gll_nodes_weights(N: int):
    """GLL nodes (ascending) and weights for polynomial order N >= 1."""
    if N < 1:
        raise ValueError("N must be >= 1")
    x = -np.cos(np.pi * np.arange(N + 1) / N)
    for _ in range(100):
        inner = x[1:-1]
        p, dp = legendre(N, inner)
        # P_N'' from Legendre's ODE: (1-x^2) P'' - 2x P' + N(N+1) P = 0
        d2p = (2.0 * inner * dp - N * (N + 1) * p) / (1.0 - inner * inner)
        step = dp / d2p
        x[1:-1] = inner - step
        if np.max(np.abs(step), initial=0.0) < 1e-16:
            break
    x[0], x[-1] = -1.0, 1.0
    pN, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * pN * pN)
    return x, w


def barycentric_weights(x):
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    lam = np.ones(n)
    for j in range(n):
        for m in range(n):
            if m != j:
                lam[j] /= (x[j] - x[m])
    return lam


def derivative_matrix(x):
    """D[i, j] = l_j'(x_i) for the Lagrange basis on nodes x."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    lam = barycentric_weights(x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (lam[j] / lam[i]) / (x[i] - x[j])
        D[i, i] = -np.sum(D[i, :])
    return D


def interpolation_matrix(x, y):
    """J[a, b] = l_b(y_a): values at points y of the Lagrange basis on nodes x."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    J = np.ones((len(y), len(x)))
    for b in range(len(x)):
        for m in range(len(x)):
            if m != b:
                J[:, b] *= (y - x[m]) / (x[b] - x[m])
    return J
