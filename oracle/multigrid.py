"""Multigrid V-cycle with Chebyshev smoothing (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

The V-cycle follows the recursive error propagator of Eq. 2.2,

    E_j = G'_j (I - P M_{j+1}^{-1} P^T A_j) G_j,   M_l^{-1} = A_l^{-1},

as a preconditioner z = M_0^{-1} r: pre-smooth from a zero guess with order m
(G_j), form the residual, restrict with P^T, recurse, add the interpolated
coarse correction, post-smooth with order n (G'_j).  The symmetric cycle is
(m, n) = (k, k) (G' = G); the one-sided cycle of Eq. 2.4 is (2k, 0) (G' = I).
Both cost 2k operator applications per level and cycle.
"""
from __future__ import annotations

import numpy as np

from .chebyshev import smooth


class Hierarchy:
    """Levels 0..l with transfers between j and j+1 and an exact/iterative coarse solve.

    Each level provides ``apply_A``, ``invD`` (Jacobi vector, 0 on Dirichlet
    nodes), ``n`` and ``lmax`` (lambda_max of S A, after any safety scaling).
    """

    def __init__(self, levels, transfers, coarse_solve, kind="opt4th", pre=2, post=0,
                 lmin_ratio=0.1, betas=None):
        if len(transfers) != len(levels) - 1:
            raise ValueError("need one transfer per level pair")
        self.levels = levels
        self.transfers = transfers
        self.coarse_solve = coarse_solve
        self.kind = kind
        self.pre = pre
        self.post = post
        self.lmin_ratio = lmin_ratio
        self.betas = betas            # optional override per order: {order: array}

    @staticmethod
    def orders(k: int, sided: str):
        """(m, n) for the symmetric (k,k) or one-sided (2k,0) cycle."""
        if sided == "symmetric":
            return k, k
        if sided == "one-sided":
            return 2 * k, 0
        raise ValueError(sided)

    def _smooth(self, j, b, order, x0):
        L = self.levels[j]
        bt = None if self.betas is None else self.betas.get(order)
        return smooth(L, b, order, self.kind, L.lmax, self.lmin_ratio, x0=x0, betas=bt)


def vcycle(H: Hierarchy, r, j: int = 0):
    """z = M_j^{-1} r by one V-cycle starting at level j."""
    if j == len(H.levels) - 1:
        return H.coarse_solve(r)
    L = H.levels[j]
    T = H.transfers[j]
    z = H._smooth(j, r, H.pre, None) if H.pre > 0 else np.zeros_like(r)
    res = r - L.apply_A(z)
    z = z + T.prolong(vcycle(H, T.restrict(res), j + 1))
    if H.post > 0:
        z = H._smooth(j, r, H.post, z)
    return z
