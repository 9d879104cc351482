"""Assembled FD and SEM multigrid hierarchies for the oracle.

Test infrastructure only (see ``oracle/__init__``).

lambda_max of S A on every smoothed level comes from ``krylov.lanczos_lmax``
(30 steps by default) times ``lmax_scale`` (1.0: the paper states no safety
factor), unless given explicitly.  The 1st-kind smoother uses
lambda_min = 0.1 lambda_max ("1st-Cheb", Sec. 2).
"""
from __future__ import annotations

from .fd import DenseCholeskySolve, fd_levels
from .krylov import lanczos_lmax, pcg_jacobi
from .multigrid import Hierarchy
from .sem import SemLevel, SemTransfer


def _set_lmax(levels, lmax, lanczos_steps, lmax_scale):
    for j, L in enumerate(levels[:-1]):
        if lmax is not None:
            L.lmax = float(lmax[j])
        else:
            L.lmax = lmax_scale * lanczos_lmax(L.apply_A, L.invD, lanczos_steps)


def fd_hierarchy(m=63, Lx=1.0, Ly=1.0, c=2, coarsest=7, kind="opt4th", k=2,
                 sided="one-sided", lmin_ratio=0.1, lmax=None, lanczos_steps=30,
                 lmax_scale=1.0, pre=None, post=None):
    levels, transfers = fd_levels(m, Lx, Ly, c, coarsest)
    for L in levels:
        L.invD = L.inv_diagonal()
    _set_lmax(levels, lmax, lanczos_steps, lmax_scale)
    mm, nn = Hierarchy.orders(k, sided)
    if pre is not None:
        mm, nn = pre, post
    coarse = DenseCholeskySolve(levels[-1].A)
    return Hierarchy(levels, transfers, coarse, kind, mm, nn, lmin_ratio)


def sem_hierarchy(verts, orders=(7, 3, 1), kind="opt4th", k=2, sided="one-sided",
                  lmin_ratio=0.1, lmax=None, lanczos_steps=30, lmax_scale=1.0,
                  coarse_rtol=1e-10, coarse_maxit=5000):
    levels = [SemLevel(verts, N) for N in orders]
    transfers = [SemTransfer(levels[j], levels[j + 1]) for j in range(len(levels) - 1)]
    for L in levels:
        L.invD = L.inv_diagonal()
    _set_lmax(levels, lmax, lanczos_steps, lmax_scale)
    mm, nn = Hierarchy.orders(k, sided)
    Lc = levels[-1]

    def coarse(r):
        return pcg_jacobi(Lc.apply_A, Lc.invD, r, coarse_rtol, coarse_maxit)[0]

    return Hierarchy(levels, transfers, coarse, kind, mm, nn, lmin_ratio)
