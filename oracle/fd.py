"""2-D finite-difference Poisson model problem with geometric multigrid (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

Sec. 3: -Laplace(u) = f on [0,Lx] x [0,Ly], u = 0 on the boundary, a grid of
(n+1) x (n+1) points, i.e. m = n-1 interior unknowns per direction, spacing
hx = Lx/n, hy = Ly/n.  The fine operator is the five-point stencil

    (A u)_ij = (2u_ij - u_{i-1,j} - u_{i+1,j}) / hx^2 + (2u_ij - u_{i,j-1} - u_{i,j+1}) / hy^2.

Coarse grids have n_c = n/c intervals (c = 2, or c = 8 for aggressive coarsening).
Interpolation is vertex-centred (bi)linear: coarse point I sits on fine point
c(I+1)-1 and fine point i receives weight max(0, 1 - |i - (c(I+1)-1)|/c).  The
coarse operators are Galerkin products A_{j+1} = P^T A_j P (Eq. 2.1); this
reading is pinned by the grid complexities 1.568 (c=2) and 1.023 (c=8) that
the paper prints for n = 128 (Eq. 3.2 and Table 1), which a rediscretised
five-point coarse operator does not reproduce.

Unknowns are ordered x fastest: index = j * mx + i.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def second_difference(m: int, h: float):
    """1-D Dirichlet second difference tridiag(-1, 2, -1) / h^2 on m interior points."""
    e = np.ones(m)
    return sp.diags([-e[:-1], 2.0 * e, -e[:-1]], [-1, 0, 1], format="csr") / (h * h)


def laplacian_5pt(mx: int, my: int, hx: float, hy: float):
    """Five-point operator as a sparse matrix (x fastest)."""
    return (sp.kron(sp.identity(my), second_difference(mx, hx))
            + sp.kron(second_difference(my, hy), sp.identity(mx))).tocsr()


def interpolation_1d(mf: int, c: int):
    """Linear interpolation from mc = (mf+1)/c - 1 coarse to mf fine interior points."""
    if (mf + 1) % c != 0:
        raise ValueError("fine size + 1 must be divisible by the coarsening factor")
    mc = (mf + 1) // c - 1
    P = np.zeros((mf, mc))
    i = np.arange(mf)
    for I in range(mc):
        P[:, I] = np.maximum(0.0, 1.0 - np.abs(i - (c * (I + 1) - 1)) / c)
    return sp.csr_matrix(P)


def bilinear_interpolation(mfx: int, mfy: int, c: int):
    return sp.kron(interpolation_1d(mfy, c), interpolation_1d(mfx, c)).tocsr()


class FdLevel:
    def __init__(self, A, mx: int, my: int):
        self.A = A.tocsr()
        self.A.eliminate_zeros()
        self.mx, self.my = mx, my
        self.n = mx * my
        self.dirichlet = np.zeros(self.n, dtype=bool)   # boundary is not in the unknowns
        self.lmax = None

    def apply_A(self, u):
        return self.A @ u

    def diagonal(self):
        return self.A.diagonal()

    def inv_diagonal(self):
        return 1.0 / self.A.diagonal()

    def nnz(self):
        return self.A.nnz


class FdTransfer:
    def __init__(self, P):
        self.P = P.tocsr()

    def prolong(self, zc):
        return self.P @ zc

    def restrict(self, rf):
        return self.P.T @ rf


def fd_levels(m: int, Lx: float = 1.0, Ly: float = 1.0, c: int = 2, coarsest: int = 7):
    """Galerkin hierarchy from an m x m interior grid down to ``coarsest`` x ``coarsest``."""
    hx, hy = Lx / (m + 1), Ly / (m + 1)
    levels = [FdLevel(laplacian_5pt(m, m, hx, hy), m, m)]
    transfers = []
    mf = m
    while mf > coarsest:
        P = bilinear_interpolation(mf, mf, c)
        mc = (mf + 1) // c - 1
        Ac = (P.T @ levels[-1].A @ P).tocsr()
        levels.append(FdLevel(Ac, mc, mc))
        transfers.append(FdTransfer(P))
        mf = mc
    return levels, transfers


class DenseCholeskySolve:
    """Exact coarsest-level solve M_l^{-1} = A_l^{-1} (Eq. 2.2) by a dense Cholesky factor."""

    def __init__(self, A):
        self.L = np.linalg.cholesky(np.asarray(A.todense() if sp.issparse(A) else A))

    def __call__(self, r):
        y = np.linalg.solve(self.L, r)
        return np.linalg.solve(self.L.T, y)
