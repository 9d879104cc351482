"""Pins of the oracle's GLL basis against library routines and exactness properties."""
import numpy as np
import pytest

from oracle.gll import derivative_matrix, gll_nodes_weights, interpolation_matrix

ORDERS = [1, 2, 3, 4, 5, 7, 9]


@pytest.mark.parametrize("N", ORDERS)
def test_nodes_are_endpoints_and_legendre_derivative_roots(N):
    x, w = gll_nodes_weights(N)
    assert x[0] == -1.0 and x[-1] == 1.0
    if N > 1:
        roots = np.sort(np.polynomial.legendre.Legendre.basis(N).deriv().roots().real)
        np.testing.assert_allclose(x[1:-1], roots, atol=1e-14)


@pytest.mark.parametrize("N", ORDERS)
def test_quadrature_exact_to_degree_2N_minus_1(N):
    x, w = gll_nodes_weights(N)
    for p in range(0, 2 * N):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(w @ x ** p - exact) < 1e-14
    if N >= 1:   # degree 2N is not integrated exactly (lumped mass)
        p = 2 * N
        assert abs(w @ x ** p - 2.0 / (p + 1)) > 1e-6


@pytest.mark.parametrize("N", ORDERS)
def test_derivative_matrix_exact_on_polynomials(N):
    x, _ = gll_nodes_weights(N)
    D = derivative_matrix(x)
    for p in range(0, N + 1):
        dp = p * x ** (p - 1) if p > 0 else np.zeros_like(x)
        np.testing.assert_allclose(D @ x ** p, dp, atol=1e-12 * max(1, N ** 2))
    # closed form of the GLL corner entries: D[0,0] = -N(N+1)/4
    assert abs(D[0, 0] + N * (N + 1) / 4.0) < 1e-12 * N * N


@pytest.mark.parametrize("Nf,Nc", [(7, 3), (3, 1), (7, 5), (9, 5), (5, 1)])
def test_interpolation_exact_and_nodal(Nf, Nc):
    xc, _ = gll_nodes_weights(Nc)
    xf, _ = gll_nodes_weights(Nf)
    J = interpolation_matrix(xc, xf)
    for p in range(Nc + 1):
        np.testing.assert_allclose(J @ xc ** p, xf ** p, atol=1e-13)
    np.testing.assert_array_equal(J[0], np.eye(Nc + 1)[0])
    np.testing.assert_array_equal(J[-1], np.eye(Nc + 1)[-1])
    np.testing.assert_allclose(J.sum(axis=1), 1.0, atol=1e-14)


@pytest.mark.parametrize("N", ORDERS)
def test_reflection_symmetry_of_nodes_weights_and_derivative(N):
    # x -> -x maps the GLL points onto themselves, so x[N-i] = -x[i], w[N-i] = w[i], and
    # differentiation anticommutes with the reflection: D[N-i][N-l] = -D[i][l]
    x, w = gll_nodes_weights(N)
    D = derivative_matrix(x)
    np.testing.assert_allclose(x[::-1], -x, atol=1e-15)
    np.testing.assert_allclose(w[::-1], w, rtol=1e-14)
    np.testing.assert_allclose(D[::-1, ::-1], -D, atol=1e-13 * max(1, N * N))
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-13 * max(1, N * N))


@pytest.mark.parametrize("N", [3, 5, 7, 9])
def test_even_odd_split_of_a_line_derivative(N):
    # the split a line pass can use: with e_l = u_l + u_{N-l}, o_l = u_l - u_{N-l} (l < (N+1)/2),
    # E_il = (D_il + D_i,N-l)/2 and O_il = (D_il - D_i,N-l)/2, (D u)_i = E_i.e + O_i.o and
    # (D u)_{N-i} = O_i.o - E_i.e for every u (odd N: an even number of points); also in the
    # form that continues the odd sum from the even one, (D u)_{N-i} = (D u)_i - 2 E_i.e
    x, _ = gll_nodes_weights(N)
    D = derivative_matrix(x)
    h = (N + 1) // 2
    E = 0.5 * (D[:h, :h] + D[:h, ::-1][:, :h])
    O = 0.5 * (D[:h, :h] - D[:h, ::-1][:, :h])
    rng = np.random.default_rng(N)
    for _ in range(4):
        u = rng.uniform(-1, 1, N + 1)
        e, o = u[:h] + u[::-1][:h], u[:h] - u[::-1][:h]
        du = D @ u
        np.testing.assert_allclose(E @ e + O @ o, du[:h], atol=1e-13 * N * N)
        np.testing.assert_allclose(O @ o - E @ e, du[::-1][:h], atol=1e-13 * N * N)
        np.testing.assert_allclose((E @ e + O @ o) - 2 * (E @ e), du[::-1][:h], atol=1e-13 * N * N)
    # transposed derivative: the same split with D^T
    Et = 0.5 * (D.T[:h, :h] + D.T[:h, ::-1][:, :h])
    Ot = 0.5 * (D.T[:h, :h] - D.T[:h, ::-1][:, :h])
    u = rng.uniform(-1, 1, N + 1)
    e, o = u[:h] + u[::-1][:h], u[:h] - u[::-1][:h]
    np.testing.assert_allclose(Et @ e + Ot @ o, (D.T @ u)[:h], atol=1e-13 * N * N)
    np.testing.assert_allclose(Ot @ o - Et @ e, (D.T @ u)[::-1][:h], atol=1e-13 * N * N)
