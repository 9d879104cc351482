"""Smoothing-polynomial theory of Sec. 2 (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

The smoothers of ``oracle.chebyshev`` applied to the scalar problem A = lambda,
S = 1, lambda_max = 1, b = 1, x0 = 0 leave the error 1/lambda - x_k =
p_k(lambda) / lambda, so p_k(lambda) = 1 - lambda x_k is the smoothing
polynomial of each algorithm.  From it:

* gamma(k) = sup_{0<lambda<=1} lambda p_k^2 / (1 - p_k^2)   (Eq. 2.14), and gamma^{-1};
* the closed forms Eqs. 2.18-2.20 (simple, 4th kind, optimized 4th kind),
  Eq. 2.21 (1st kind, fixed lambda_min) and the correlation Eq. 2.24;
* the critical C above which (2k,0) beats (k,k) (Eqs. 2.17, 2.25-2.26);
* grid complexity (Eq. 3.2).
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import minimize_scalar

from .chebyshev import chebyshev_1st, chebyshev_4th, optimized_betas, simple


def smoothing_polynomial(kind: str, k: int, lam, lmin_ratio: float = 0.1, omega: float = 1.5,
                         betas=None):
    lam = np.atleast_1d(np.asarray(lam, dtype=np.float64))
    one = np.ones_like(lam)

    def apply(v):
        return lam * v

    if kind == "1st":
        x = chebyshev_1st(apply, one, one, k, 1.0, lmin_ratio)
    elif kind == "4th":
        x = chebyshev_4th(apply, one, one, k, 1.0, betas=betas)
    elif kind == "opt4th":
        x = chebyshev_4th(apply, one, one, k, 1.0,
                          betas=optimized_betas(k) if betas is None else betas)
    elif kind == "simple":
        x = simple(apply, one, one, k, omega, 1.0)
    else:
        raise ValueError(kind)
    return 1.0 - lam * x


def gamma(kind: str, k: int, **kw) -> float:
    """sup over (0,1] of lambda p^2 / (1 - p^2), by a dense grid then a local refinement."""
    def f(lam):
        p = smoothing_polynomial(kind, k, lam, **kw)
        return lam * p * p / (1.0 - p * p)

    lam = np.concatenate([np.geomspace(1e-7, 1e-2, 2000), np.linspace(1e-2, 1.0, 400001)])
    vals = f(lam)
    i = int(np.argmax(vals))
    best = float(vals[i])
    lo, hi = lam[max(i - 1, 0)], lam[min(i + 1, len(lam) - 1)]
    if hi > lo:
        res = minimize_scalar(lambda t: -float(f(t)[0]), bounds=(lo, hi), method="bounded",
                              options={"xatol": 1e-14})
        best = max(best, -float(res.fun))
    return best


def gamma_inv(kind: str, k: int, **kw) -> float:
    return 1.0 / gamma(kind, k, **kw)


def gamma_inv_simple(k, omega):            # Eq. 2.18
    return 2.0 * omega * k


def gamma_inv_4th(k):                      # Eq. 2.19
    return 4.0 / 3.0 * k * (k + 1)


def gamma_inv_opt4th(k):                   # Eq. 2.20 (approximate)
    return 4.0 / np.pi ** 2 * (2 * k + 1) ** 2 - 2.0 / 3.0


def cheb_T(k, x):
    return np.polynomial.chebyshev.chebval(x, [0] * k + [1])


def cheb_U(k, x):
    """Chebyshev polynomial of the 2nd kind U_k via U_k = (T_k x - T_{k+1}) / (1 - x^2) recurrence."""
    u0, u1 = 1.0, 2.0 * x
    if k == 0:
        return u0
    for _ in range(1, k):
        u0, u1 = u1, 2.0 * x * u1 - u0
    return u1


def gamma_inv_1st(k, lmin, kstar):         # Eq. 2.21 (lambda_max = 1)
    a = (lmin + 1.0) / (lmin - 1.0)
    if k <= kstar:
        return cheb_T(k, a) ** 2 - 1.0
    return 4.0 * k * cheb_U(k - 1, a) / ((lmin - 1.0) * cheb_T(k, a))


def lambda_min_opt_correlation(k):         # Eq. 2.24
    return 1.69 / (k ** 1.68 + 2.11 * k + 1.98)


def critical_C_from_gamma(gi_k, gi_2k):
    """C above which (2k,0) beats (k,k) in Eq. 2.17 (requires gi_2k > 2 gi_k)."""
    return gi_k ** 2 / (gi_2k - 2.0 * gi_k)


def critical_C_4th(k):                     # Eq. 2.25
    return 2.0 * (k + 1) ** 2 / 3.0


def critical_C_opt4th(k):                  # Eq. 2.26
    a = (2 * k + 1) ** 2
    return 2.0 * (6 * a - np.pi ** 2) ** 2 / (3 * np.pi ** 2 * (-12 * a + 6 * (4 * k + 1) ** 2 + np.pi ** 2))


def grid_complexity(nnz_per_level):        # Eq. 3.2
    nnz = np.asarray(nnz_per_level, dtype=np.float64)
    return float(nnz.sum() / nnz[0])


def _fourth_kind_directions(k: int, lam):
    """d_0 .. d_{k-1} of Algorithm 2 on the scalar problem (A = lambda, S = 1, lambda_max = 1,
    b = 1, x0 = 0), as columns: x_k = sum_i beta_i d_{i-1}, so p(lambda) = 1 - lambda x_k is
    affine in the weights."""
    r = np.ones_like(lam)
    d = (4.0 / 3.0) * r
    cols = [d.copy()]
    for i in range(1, k):
        r = r - lam * d
        d = (2.0 * i - 1.0) / (2.0 * i + 3.0) * d + (8.0 * i + 4.0) / (2.0 * i + 3.0) * r
        cols.append(d.copy())
    return np.stack(cols, axis=1)


def optimal_betas(k: int, npts: int = 8000, rounds: int = 2):
    """Weights beta_1..beta_k of Algorithm 2 that maximise gamma^{-1} (Eq. 2.14), the
    criterion of the optimized 4th kind (Sec. 2.3, Table 5).

    lambda p^2 / (1 - p^2) <= t is |p(lambda)| <= c_t = sqrt(t / (lambda + t)); as p is affine in
    the weights, for a fixed t the feasible weights on a set of lambda points form a polyhedron.
    Bisection on t with a linear-programming feasibility test (maximal common slack) gives the
    smallest feasible t, i.e. the largest gamma^{-1}.  The points are Chebyshev-spaced on (0, 1],
    then the local maxima of lambda p^2 / (1 - p^2) for the computed weights are added and the
    bisection is repeated.  Returns (betas, gamma^{-1})."""
    from scipy.optimize import linprog

    theta = np.linspace(0.0, np.pi, npts + 1)[1:]
    lam = 0.5 * (1.0 - np.cos(theta))

    def slack(G, lm, t):
        c = np.sqrt(t / (lm + t))
        lo, hi = 1.0 / ((lm + t) * (1.0 + c)), (1.0 + c) / lm   # (1 - c) / lambda without cancellation
        w = 0.5 * (hi - lo)
        A = np.vstack([np.hstack([-G, w[:, None]]), np.hstack([G, w[:, None]])])
        rhs = np.concatenate([-lo, hi])
        cost = np.zeros(k + 1)
        cost[-1] = -1.0
        res = linprog(cost, A_ub=A, b_ub=rhs, bounds=[(None, None)] * k + [(None, 1.0)], method="highs")
        return res.x[-1], res.x[:k]

    def solve(lm):
        G = _fourth_kind_directions(k, lm)
        g_est = 4.0 / np.pi ** 2 * (2 * k + 1) ** 2 - 2.0 / 3.0
        lo_t, hi_t = 0.25 / g_est, 4.0 / g_est
        for _ in range(80):
            mid = np.sqrt(lo_t * hi_t)
            if slack(G, lm, mid)[0] >= 0.0:
                hi_t = mid
            else:
                lo_t = mid
            if hi_t / lo_t - 1.0 < 1e-13:
                break
        return slack(G, lm, hi_t)[1]

    betas = solve(lam)
    for _ in range(rounds):
        fine = 0.5 * (1.0 - np.cos(np.linspace(0.0, np.pi, 40 * npts + 1)[1:]))
        x = _fourth_kind_directions(k, fine) @ betas
        p = 1.0 - fine * x
        f = p * p / (x * (1.0 + p))          # lambda p^2 / (1 - p^2) with 1 - p = lambda x
        peaks = np.where((f[1:-1] >= f[:-2]) & (f[1:-1] >= f[2:]))[0] + 1
        lam = np.unique(np.concatenate([lam, fine[peaks], fine[np.clip(peaks - 1, 0, None)],
                                        fine[np.clip(peaks + 1, None, len(fine) - 1)]]))
        betas = solve(lam)
    return betas, gamma_inv("opt4th", k, betas=betas)
