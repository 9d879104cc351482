"""Pins of Algorithms 1 and 2 (and the beta table) against closed forms of Sec. 2."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import theory as T
from oracle.chebyshev import BETA_TABLE, chebyshev_1st, chebyshev_4th

LAM = np.linspace(1e-3, 1.0, 997)


def fourth_kind_W(k, x):
    """W_k(cos t) = sin((k + 1/2) t) / sin(t/2) (Mason & Handscomb), independent of Eq. 2.12."""
    t = np.arccos(np.clip(x, -1, 1))
    return np.sin((k + 0.5) * t) / np.sin(t / 2)


@pytest.mark.parametrize("k", range(1, 9))
def test_algorithm2_is_fourth_kind_polynomial(k):
    p = T.smoothing_polynomial("4th", k, LAM)
    np.testing.assert_allclose(p, fourth_kind_W(k, 1 - 2 * LAM) / (2 * k + 1), atol=2e-14)


@pytest.mark.parametrize("k", range(1, 9))
@pytest.mark.parametrize("lmin", [0.1, 0.3, 1 / 30])
def test_algorithm1_is_shifted_scaled_first_kind(k, lmin):
    theta, delta = (1 + lmin) / 2, (1 - lmin) / 2
    ref = T.cheb_T(k, (theta - LAM) / delta) / T.cheb_T(k, theta / delta)
    np.testing.assert_allclose(T.smoothing_polynomial("1st", k, LAM, lmin_ratio=lmin), ref, atol=2e-14)


@pytest.mark.parametrize("k", range(1, 7))
def test_optimized_fourth_kind_is_beta_combination_of_fourth_kind(k):
    # x_k = sum_i beta_i d_{i-1} with d_{i-1} the standard increments, so
    # p_opt = 1 - sum_i beta_i (p_{i-1} - p_i) with p_i = W_i(1-2 lam)/(2i+1), p_0 = 1.
    beta = np.array(BETA_TABLE[k])
    p = [np.ones_like(LAM)] + [fourth_kind_W(i, 1 - 2 * LAM) / (2 * i + 1) for i in range(1, k + 1)]
    ref = 1 - sum(beta[i - 1] * (p[i - 1] - p[i]) for i in range(1, k + 1))
    np.testing.assert_allclose(T.smoothing_polynomial("opt4th", k, LAM), ref, atol=5e-14)


def test_optimized_k1_is_three_halves_richardson():
    # beta_1^{(1)} = 1.125 turns d_0 = (4/3) r_0 into the omega = 3/2 simple iteration (Eq. 2.3)
    np.testing.assert_allclose(T.smoothing_polynomial("opt4th", 1, LAM), 1 - 1.5 * LAM, atol=1e-15)
    np.testing.assert_allclose(T.smoothing_polynomial("simple", 3, LAM, omega=1.5), (1 - 1.5 * LAM) ** 3,
                               atol=1e-14)


def test_beta_table_shape():
    assert sorted(BETA_TABLE) == list(range(1, 17))
    for k, b in BETA_TABLE.items():
        assert len(b) == k
        assert all(1.0 < x < 1.52 for x in b)
        assert list(b) == sorted(b)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6])
def test_gamma_inverse_fourth_kind_closed_form(k):
    assert abs(T.gamma_inv("4th", k) / T.gamma_inv_4th(k) - 1) < 1e-5          # Eq. 2.19


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 8])
def test_gamma_inverse_optimized_fourth_kind(k):
    g = T.gamma_inv("opt4th", k)
    assert abs(g / T.gamma_inv_opt4th(k) - 1) < 0.01                         # Eq. 2.20 (approx.)
    assert g > T.gamma_inv("4th", k) * 1.05                                  # optimisation helps


@pytest.mark.parametrize("k", [2, 3, 4])
def test_beta_table_is_locally_optimal(k):
    base = np.array(BETA_TABLE[k])
    g0 = T.gamma_inv("opt4th", k)
    for i in range(k):
        for s in (-1, 1):
            b = base.copy()
            b[i] *= 1 + s * 3e-3
            assert T.gamma_inv("opt4th", k, betas=b) <= g0 * (1 + 1e-7)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_gamma_inverse_first_kind_closed_form(k):
    g = T.gamma_inv("1st", k, lmin_ratio=0.1)
    assert abs(g / T.gamma_inv_1st(k, 0.1, kstar=3) - 1) < 1e-5                # Eq. 2.21, k* = 3


def test_gamma_inverse_simple_closed_form():
    for k, om in [(1, 1.0), (3, 1.0), (2, 1.5), (5, 0.8)]:
        assert abs(T.gamma_inv("simple", k, omega=om) / T.gamma_inv_simple(k, om) - 1) < 1e-5


@pytest.mark.parametrize("k", [1, 2, 4, 10])
def test_optimal_lambda_min_correlation(k):
    res = minimize_scalar(lambda lm: -T.gamma_inv("1st", k, lmin_ratio=lm), bounds=(1e-3, 0.6),
                          method="bounded", options={"xatol": 1e-6})
    ref = T.lambda_min_opt_correlation(k)                                     # Eq. 2.24
    assert abs(res.x - ref) <= 0.01 * ref + 2e-3


@pytest.mark.parametrize("k", [1, 2, 3])
def test_critical_C_fourth_kind(k):
    gk, g2k = T.gamma_inv("4th", k), T.gamma_inv("4th", 2 * k)
    assert abs(T.critical_C_from_gamma(gk, g2k) / T.critical_C_4th(k) - 1) < 1e-4   # Eq. 2.25
    assert np.allclose([T.critical_C_4th(i) for i in (1, 2, 3)], [8 / 3, 6.0, 32 / 3])


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_critical_C_optimized_fourth_kind(k):
    # Eq. 2.26 substitutes the approximate Eq. 2.20 into Eq. 2.17
    gk, g2k = T.gamma_inv_opt4th(k), T.gamma_inv_opt4th(2 * k)
    assert abs(T.critical_C_from_gamma(gk, g2k) / T.critical_C_opt4th(k) - 1) < 1e-12
    num = T.critical_C_from_gamma(T.gamma_inv("opt4th", k), T.gamma_inv("opt4th", 2 * k))
    assert abs(num / T.critical_C_opt4th(k) - 1) < 0.1


def test_smoother_on_vectors_matches_scalar_polynomial():
    # Smoothing a diagonal system acts mode by mode: e_k = p_k(S A / lambda_max) e_0.
    rng = np.random.default_rng(0)
    d = rng.uniform(0.5, 2.0, 50)              # A = diag(d) * s, S = 1/d
    lam = rng.uniform(0.01, 1.0, 50)
    Adiag = lam * d * 3.0                      # S A = 3 lam, lambda_max = 3
    S = 1.0 / d
    e0 = rng.uniform(-1, 1, 50)
    b = Adiag * e0                             # exact solution e0, start from zero
    for kind, k in [("1st", 3), ("4th", 4), ("opt4th", 5)]:
        if kind == "1st":
            x = chebyshev_1st(lambda v: Adiag * v, S, b, k, 3.0, 0.3)
        else:
            bt = np.array(BETA_TABLE[k]) if kind == "opt4th" else None
            x = chebyshev_4th(lambda v: Adiag * v, S, b, k, 3.0, betas=bt)
        p = T.smoothing_polynomial(kind, k, lam)
        np.testing.assert_allclose(e0 - x, p * e0, atol=1e-13)


@pytest.mark.parametrize("k", [2, 4])
def test_gamma_maximising_weights_reproduce_table5(k):
    # the optimizer behind the weights of orders beyond Table 5 recovers the table's rows
    b, gi = T.optimal_betas(k, npts=4000, rounds=1)
    assert np.abs(b - np.array(BETA_TABLE[k])).max() < 2e-6
    assert gi == pytest.approx(T.gamma_inv("opt4th", k), rel=2e-6)


def test_stored_weights_beyond_table5_are_optimal():
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "optimal_betas.json")))
    for key, rec in gold["orders"].items():
        k = int(key)
        b = np.array(rec["betas"])
        assert len(b) == k
        g0 = T.gamma_inv("opt4th", k, betas=b)
        assert g0 == pytest.approx(rec["gamma_inv"], rel=1e-9)
        assert abs(g0 / T.gamma_inv_opt4th(k) - 1) < 0.01             # Eq. 2.20
        assert g0 > 1.2 * T.gamma_inv("4th", k)                        # above the 4th kind (ratio -> 12/pi^2)
        for i in (0, k // 2, k - 1):                                   # locally optimal
            for s in (-1, 1):
                bp = b.copy()
                bp[i] *= 1 + s * 3e-3
                assert T.gamma_inv("opt4th", k, betas=bp) <= g0 * (1 + 1e-7)
