"""Sensitivity of the V-cycle's error reduction to the smoother weights (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

Objective.  With B one V-cycle (Eq. 2.2) and E = I - B A its error propagator, the
observed convergence of Sec. 3 (Eq. 3.1) after ``steps`` cycles from initial errors
e0_1 .. e0_J (the rows of E0) is measured by

    f = (1/J) sum_q ||E^steps e0_q||^2 / ||e0_q||^2 .

Parameters: the 4th-kind Chebyshev weights beta_1 .. beta_k of Algorithm 2 (one set,
used by every smoothing call of the cycle: k must equal the pre-smoothing order, and the
post-smoothing order if there is one) and a common scale s of the lambda_max values,
lambda_max_j = s * lmax_j.

Derivatives.  ``error_ratio_and_gradient`` propagates, next to every vector of the cycle,
its derivative with respect to each parameter (forward mode / tangent-linear): one
extra vector per parameter, updated by the product rule at each step of Algorithm 2, of
the residual/restriction/prolongation steps of Eq. 2.2 and of E.  The coarsest level is
solved with ``H.coarse_solve``, taken as linear (an exact solve, or an iterative one whose
tolerance is far below the differences being measured).
"""
from __future__ import annotations

import numpy as np


def _smooth_tangent(L, b, bt, order, lam, dlam, betas, x0=None, x0t=None):
    """Algorithm 2 with weights ``betas`` and lambda_max ``lam`` on level L.

    bt, x0t: tangents of b and x0, arrays of shape (P, n).  dlam: d lam / d param (P,).
    The weights are parameters 0..k-1.  Returns (x, xt)."""
    P = bt.shape[0]
    S = L.invD
    A = L.apply_A
    if x0 is None:
        x = np.zeros_like(b)
        xt = np.zeros_like(bt)
        r = b.copy()
        rt = bt.copy()
    else:
        x = x0.copy()
        xt = x0t.copy()
        r = b - A(x)
        rt = bt - np.stack([A(v) for v in xt])
    c = 4.0 / 3.0
    d = (c / lam) * (S * r)
    dt = (c / lam) * (S * rt) - (c * dlam / lam ** 2)[:, None] * (S * r)[None, :]
    for i in range(1, order):
        x = x + betas[i - 1] * d
        xt = xt + betas[i - 1] * dt
        xt[i - 1] += d
        Ad = A(d)
        r = r - Ad
        rt = rt - np.stack([A(v) for v in dt])
        c1 = (2.0 * i - 1.0) / (2.0 * i + 3.0)
        c2 = (8.0 * i + 4.0) / (2.0 * i + 3.0)
        d_new = c1 * d + (c2 / lam) * (S * r)
        dt = c1 * dt + (c2 / lam) * (S * rt) - (c2 * dlam / lam ** 2)[:, None] * (S * r)[None, :]
        d = d_new
    x = x + betas[order - 1] * d
    xt = xt + betas[order - 1] * dt
    xt[order - 1] += d
    assert xt.shape[0] == P
    return x, xt


def _vcycle_tangent(H, lams, dlams, betas, r, rt, j=0):
    """z = B r and its tangents (Eq. 2.2 with the 4th-kind smoother of weights ``betas``)."""
    if j == len(H.levels) - 1:
        return H.coarse_solve(r), np.stack([H.coarse_solve(v) for v in rt])
    L = H.levels[j]
    T = H.transfers[j]
    if H.pre > 0:
        z, zt = _smooth_tangent(L, r, rt, H.pre, lams[j], dlams[j], betas)
    else:
        z, zt = np.zeros_like(r), np.zeros_like(rt)
    res = r - L.apply_A(z)
    rest = rt - np.stack([L.apply_A(v) for v in zt])
    zc, zct = _vcycle_tangent(H, lams, dlams, betas, T.restrict(res), np.stack([T.restrict(v) for v in rest]),
                              j + 1)
    z = z + T.prolong(zc)
    zt = zt + np.stack([T.prolong(v) for v in zct])
    if H.post > 0:
        z, zt = _smooth_tangent(L, r, rt, H.post, lams[j], dlams[j], betas, x0=z, x0t=zt)
    return z, zt


def _check(H, betas):
    k = len(betas)
    if H.kind not in ("4th", "opt4th"):
        raise ValueError("the weights belong to Algorithm 2 (4th kind)")
    if H.pre != k or H.post not in (0, k):
        raise ValueError("one weight per smoothing step: k must equal the smoothing order")


def error_ratio_and_gradient(H, E0, betas, scale, steps: int = 3):
    """f and df/d(beta_1..beta_k, s) for the rows of E0 (shape (J, n)).

    H.levels[j].lmax are the unscaled lambda_max values; the cycle uses scale * lmax."""
    betas = np.asarray(betas, dtype=np.float64)
    _check(H, betas)
    k = len(betas)
    P = k + 1
    nlev = len(H.levels)
    lams = [scale * H.levels[j].lmax for j in range(nlev - 1)]
    dlams = []
    for j in range(nlev - 1):
        g = np.zeros(P)
        g[k] = H.levels[j].lmax          # d(s lmax_j)/ds
        dlams.append(g)
    A = H.levels[0].apply_A
    E0 = np.atleast_2d(np.asarray(E0, dtype=np.float64))
    J = E0.shape[0]
    f = 0.0
    grad = np.zeros(P)
    for q in range(J):
        e = E0[q].copy()
        et = np.zeros((P, e.size))
        n0 = e @ e
        for _ in range(steps):
            w = A(e)
            wt = np.stack([A(v) for v in et])
            z, zt = _vcycle_tangent(H, lams, dlams, betas, w, wt)
            e = e - z
            et = et - zt
        f += (e @ e) / n0 / J
        grad += 2.0 * (et @ e) / n0 / J
    return f, grad


def error_ratio(H, E0, betas, scale, steps: int = 3):
    """f alone for the rows of E0, by the plain smoother and cycle (no tangents)."""
    from .chebyshev import chebyshev_4th
    betas = np.asarray(betas, dtype=np.float64)
    _check(H, betas)
    nlev = len(H.levels)

    def cycle(r, j=0):
        if j == nlev - 1:
            return H.coarse_solve(r)
        L = H.levels[j]
        T = H.transfers[j]
        lam = scale * L.lmax
        z = chebyshev_4th(L.apply_A, L.invD, r, H.pre, lam, betas=betas)
        z = z + T.prolong(cycle(T.restrict(r - L.apply_A(z)), j + 1))
        if H.post > 0:
            z = chebyshev_4th(L.apply_A, L.invD, r, H.post, lam, betas=betas, x0=z)
        return z

    A = H.levels[0].apply_A
    E0 = np.atleast_2d(np.asarray(E0, dtype=np.float64))
    J = E0.shape[0]
    f = 0.0
    for q in range(J):
        e = E0[q].copy()
        n0 = e @ e
        for _ in range(steps):
            e = e - cycle(A(e))
        f += (e @ e) / n0 / J
    return f
