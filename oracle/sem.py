"""Spectral-element Poisson operator on a box of trilinear hexahedra (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

Definition (Sec. 1, Eq. 1.3): a_ij = int_Omega grad(phi_i) . grad(phi_j) dV with
the phi_i tensor-product Lagrange polynomials of order N on GLL points, the
integral evaluated by GLL quadrature, and the elements assembled by direct
stiffness summation:

    A = M Q^T blockdiag(A_e) Q M,  A_e = sum_{m,n} Dhat_m^T G^e_mn Dhat_n,

with Q the global-to-local copy (gather), Q^T the scatter-add, M the mask that
removes Dirichlet nodes, Dhat_1 = I x I x D (r), Dhat_2 = I x D x I (s),
Dhat_3 = D x I x I (t) and

    G^e_mn(q) = w_i w_j w_k |J(q)| sum_l (dr_m/dx_l)(dr_n/dx_l)

the six geometric factors of each quadrature point (isoparametric: the
Jacobian is D applied to the GLL coordinates).

The p-multigrid hierarchy (Sec. 4.1) varies the order N on the same elements.
Interpolation from order Nc to Nf is P = W Q_f^T (J x J x J) Q_c with J the
Nc-basis evaluated at the Nf GLL points and W = diag(1/multiplicity); the
restriction is its exact transpose P^T = Q_c^T (J^T x J^T x J^T) Q_f W.

Local arrays are indexed ``[e, k, j, i]`` with i (the r direction) fastest;
element ``e = (ez*ney + ey)*nex + ex``; the global id of local node
(e, k, j, i) is ``((ez*N+k)*NY + ey*N+j)*NX + ex*N+i``.
"""
from __future__ import annotations

import numpy as np

from .gll import derivative_matrix, gll_nodes_weights, interpolation_matrix

# order of the six stored geometric factors
G_PAIRS = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def _along_i(M, u):
    """Apply matrix M along the i (fastest) axis of u[e, k, j, i]."""
    return np.matmul(u, M.T)


def _along_j(M, u):
    return np.matmul(M, u)


def _along_k(M, u):
    E, nk, nj, ni = u.shape
    return np.matmul(M, u.reshape(E, nk, nj * ni)).reshape(E, M.shape[0], nj, ni)


class SemLevel:
    """One order-N discretisation of the perturbed box (all or a subset of the elements)."""

    def __init__(self, verts: np.ndarray, N: int, elements=None):
        verts = np.asarray(verts, dtype=np.float64)
        self.verts = verts
        self.nez, self.ney, self.nex = (s - 1 for s in verts.shape[:3])
        self.N = N
        self.Nq = N + 1
        self.NX, self.NY, self.NZ = self.nex * N + 1, self.ney * N + 1, self.nez * N + 1
        self.n = self.NX * self.NY * self.NZ
        self.E_total = self.nex * self.ney * self.nez
        if elements is None:
            elements = np.arange(self.E_total)
        self.elements = np.asarray(elements, dtype=np.int64)
        self.E = len(self.elements)
        self.x, self.w = gll_nodes_weights(N)
        self.D = derivative_matrix(self.x)

        ex = self.elements % self.nex
        ey = (self.elements // self.nex) % self.ney
        ez = self.elements // (self.nex * self.ney)
        self.ex, self.ey, self.ez = ex, ey, ez
        q = np.arange(self.Nq)
        gx = ex[:, None, None, None] * N + q[None, None, None, :]
        gy = ey[:, None, None, None] * N + q[None, None, :, None]
        gz = ez[:, None, None, None] * N + q[None, :, None, None]
        self.gid = (gz * self.NY + gy) * self.NX + gx                     # [e,k,j,i]

        full = np.zeros((self.NZ, self.NY, self.NX), dtype=bool)
        full[0], full[-1] = True, True
        full[:, 0], full[:, -1] = True, True
        full[:, :, 0], full[:, :, -1] = True, True
        self.dirichlet = full.reshape(-1)

        self.coords = self._coordinates()
        self.G, self.jac = self._geometric_factors()

    # -- geometry -----------------------------------------------------------
    def _coordinates(self):
        """Trilinear map of each element's 8 vertices evaluated at the GLL points."""
        r = self.x
        phi = np.stack([(1.0 - r) / 2.0, (1.0 + r) / 2.0])                 # [a, i]
        X = np.zeros((self.E, self.Nq, self.Nq, self.Nq, 3))
        for c in (0, 1):
            for b in (0, 1):
                for a in (0, 1):
                    V = self.verts[self.ez + c, self.ey + b, self.ex + a]    # [e, 3]
                    shape = (phi[c][:, None, None] * phi[b][None, :, None] * phi[a][None, None, :])
                    X += shape[None, :, :, :, None] * V[:, None, None, None, :]
        return X

    def _geometric_factors(self):
        X = self.coords
        D = self.D
        dX = np.empty(X.shape + (3,))            # [e,k,j,i, a (x_a), b (r_b)]
        for a in range(3):
            dX[..., a, 0] = _along_i(D, X[..., a])
            dX[..., a, 1] = _along_j(D, X[..., a])
            dX[..., a, 2] = _along_k(D, X[..., a])
        jac = np.linalg.det(dX)
        if np.min(jac) <= 0.0:
            raise ValueError("mesh has a non-positive Jacobian")
        rx = np.linalg.inv(dX)                   # rx[..., m, l] = d r_m / d x_l
        w3 = self.w[:, None, None] * self.w[None, :, None] * self.w[None, None, :]
        wJ = w3[None] * jac
        G = np.empty((self.E, 6, self.Nq, self.Nq, self.Nq))
        for p, (m, nn) in enumerate(G_PAIRS):
            G[:, p] = wJ * np.sum(rx[..., m, :] * rx[..., nn, :], axis=-1)
        return G, jac

    # -- operator -------------------------------------------------------------
    def ax_local(self, uL):
        """Element-local A_e u_e for u_e given as [e, k, j, i]."""
        D = self.D
        ur = _along_i(D, uL)
        us = _along_j(D, uL)
        ut = _along_k(D, uL)
        G = self.G
        wr = G[:, 0] * ur + G[:, 1] * us + G[:, 2] * ut
        ws = G[:, 1] * ur + G[:, 3] * us + G[:, 4] * ut
        wt = G[:, 2] * ur + G[:, 4] * us + G[:, 5] * ut
        return _along_i(D.T, wr) + _along_j(D.T, ws) + _along_k(D.T, wt)

    def gather(self, u):
        """Q M u: local copies of the global vector, Dirichlet nodes read as 0."""
        u = np.where(self.dirichlet, 0.0, u)
        return u[self.gid]

    def scatter(self, yL):
        """M Q^T y_L: direct-stiffness sum of local contributions, masked."""
        y = np.bincount(self.gid.ravel(), weights=yL.ravel(), minlength=self.n)
        y[self.dirichlet] = 0.0
        return y

    def apply_A(self, u):
        return self.scatter(self.ax_local(self.gather(u)))

    def diag_local(self):
        """Diagonal of each A_e (GLL: only same-point cross terms survive)."""
        D = self.D
        D2 = D * D
        dd = np.diag(D)
        G = self.G
        di = dd[None, None, None, :]
        dj = dd[None, None, :, None]
        dk = dd[None, :, None, None]
        return (_along_i(D2.T, G[:, 0]) + _along_j(D2.T, G[:, 3]) + _along_k(D2.T, G[:, 5])
                + 2.0 * G[:, 1] * di * dj + 2.0 * G[:, 2] * di * dk + 2.0 * G[:, 4] * dj * dk)

    def diagonal(self):
        """Assembled diag(A), zero on Dirichlet nodes."""
        return self.scatter(self.diag_local())

    def inv_diagonal(self):
        """Jacobi S = diag(A)^{-1} (Sec. 2, Eq. 2.3 context), zero on Dirichlet nodes."""
        d = self.diagonal()
        out = np.zeros_like(d)
        live = ~self.dirichlet
        out[live] = 1.0 / d[live]
        return out

    def multiplicity(self):
        return np.bincount(self.gid.ravel(), minlength=self.n).astype(np.float64)

    def dense(self):
        """Dense assembled A (tiny meshes only): columns A e_g."""
        A = np.zeros((self.n, self.n))
        for g in range(self.n):
            e = np.zeros(self.n)
            e[g] = 1.0
            A[:, g] = self.apply_A(e)
        return A


class SemTransfer:
    """p-multigrid interpolation between two orders on the same elements (Sec. 4.1)."""

    def __init__(self, fine: SemLevel, coarse: SemLevel):
        self.fine, self.coarse = fine, coarse
        self.J = interpolation_matrix(coarse.x, fine.x)        # [fine point, coarse point]
        self.Wf = 1.0 / fine.multiplicity()

    def _interp_local(self, M, uL):
        return _along_k(M, _along_j(M, _along_i(M, uL)))

    def prolong(self, zc):
        """P z_c = W Q_f^T (J x J x J) Q_c z_c, masked."""
        zL = self._interp_local(self.J, self.coarse.gather(zc))
        z = np.bincount(self.fine.gid.ravel(), weights=zL.ravel(), minlength=self.fine.n) * self.Wf
        z[self.fine.dirichlet] = 0.0
        return z

    def restrict(self, rf):
        """P^T r_f = Q_c^T (J^T x J^T x J^T) Q_f W r_f, masked."""
        rL = self.fine.gather(rf * self.Wf)
        return self.coarse.scatter(self._interp_local(self.J.T, rL))
