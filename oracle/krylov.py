"""Outer Krylov solver, coarse Jacobi-PCG, Lanczos lambda_max, SplitMix64 (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

* ``fcg``: the outer solver.  The paper wraps one V-cycle in GMRES because the
  one-sided cycle is not symmetric (Sec. 6.1); here the outer loop is flexible
  CG with the Polak-Ribiere beta = (z_{k+1}, r_{k+1} - r_k) / (z_k, r_k), which
  equals PCG for a fixed symmetric preconditioner and tolerates the one-sided
  cycle and the inexact coarse solve.  Zero initial guess; stop when
  ||r||_2 / ||b||_2 <= rtol (the 1e-8 relative residual of Sec. 5.1).
  Iterations = number of x updates = number of preconditioner applications.
* ``pcg_jacobi``: Jacobi-preconditioned CG, used for the p = 1 coarse problem.
* ``pcg_cheb4``: CG preconditioned by one degree-m application of Algorithm 2 (the same
  coarse solver with a polynomial preconditioner; m = 1 reduces to Jacobi-PCG).
* ``lanczos_lmax``: lambda_max of S A (Sec. 2: lambda_max is the largest
  eigenvalue of S_j A_j; the paper does not say how it is estimated).  Plain
  Lanczos on the symmetric S^{1/2} A S^{1/2}, start vector from SplitMix64, the
  largest Ritz value of the tridiagonal matrix.
* ``splitmix64_uniform``: counter-based SplitMix64 (Steele, Lea & Flood 2014).
* ``gmres``: restarted GMRES(m) with classical Gram-Schmidt (Sec. 6.1), right
  preconditioned, for the paper's FD experiment (Sec. 3).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


class NotConverged(RuntimeError):
    pass


def fcg(apply_A, precond, b, rtol: float = 1e-8, maxit: int = 500):
    """Flexible CG.  Returns (x, iterations, history of ||r||/||b||)."""
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    hist = [1.0]
    if bnorm == 0.0:
        return x, 0, hist
    r = b.copy()
    z = precond(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = apply_A(p)
        alpha = rz / (p @ q)
        x = x + alpha * p
        r_new = r - alpha * q
        rel = np.linalg.norm(r_new) / bnorm
        hist.append(rel)
        if rel <= rtol:
            return x, it, hist
        z = precond(r_new)
        beta = (z @ (r_new - r)) / rz
        rz = r_new @ z
        p = z + beta * p
        r = r_new
    raise NotConverged(f"FCG did not reach {rtol} in {maxit} iterations (last {hist[-1]:.3e})")


def pcg_jacobi(apply_A, Sdiag, b, rtol: float = 1e-10, maxit: int = 2000):
    """Jacobi-PCG with zero initial guess to ||r||/||b|| <= rtol.  Returns (x, iterations)."""
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0
    r = b.copy()
    z = Sdiag * r
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = apply_A(p)
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        if np.linalg.norm(r) / bnorm <= rtol:
            return x, it
        z = Sdiag * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    raise NotConverged(f"coarse PCG did not reach {rtol} in {maxit} iterations")


def pcg_cheb4(apply_A, Sdiag, b, lmax: float, degree: int, rtol: float = 1e-10, maxit: int = 2000):
    """PCG whose preconditioner is one application of Algorithm 2 (4th kind, beta = 1) of the
    given degree from a zero guess: M^{-1} = q(S A) S with q(l) = (1 - W_m(1 - 2 l/lmax)/(2m+1)) / l,
    positive on (0, lmax], so M^{-1} is SPD.  degree = 1 is Jacobi-PCG (a scaled S).
    Returns (x, iterations)."""
    from .chebyshev import chebyshev_4th

    def precond(r):
        return chebyshev_4th(apply_A, Sdiag, r, degree, lmax)

    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0
    r = b.copy()
    z = precond(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = apply_A(p)
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        if np.linalg.norm(r) / bnorm <= rtol:
            return x, it
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    raise NotConverged(f"polynomial PCG did not reach {rtol} in {maxit} iterations")


_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First n outputs of SplitMix64 seeded with ``seed`` (as uint64)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + np.arange(1, n + 1, dtype=np.uint64) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """SplitMix64 outputs mapped to [-1, 1): 2 * (top 53 bits / 2^53) - 1."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


LANCZOS_SEED = 42


def lanczos_tridiagonal(apply_A, Sdiag, v0, steps: int = 30):
    """Plain Lanczos on S^{1/2} A S^{1/2}; returns the tridiagonal (alpha, beta)."""
    s = np.sqrt(Sdiag)
    v = v0 * (Sdiag > 0)
    v = v / np.linalg.norm(v)
    v_prev = np.zeros_like(v)
    beta = 0.0
    alphas, betas = [], []
    for _ in range(steps):
        w = s * apply_A(s * v)
        alpha = v @ w
        w = w - alpha * v - beta * v_prev
        alphas.append(alpha)
        beta = np.linalg.norm(w)
        if beta <= 1e-14 * abs(alpha):
            break
        betas.append(beta)
        v_prev, v = v, w / beta
    return np.array(alphas), np.array(betas[: len(alphas) - 1])


def lanczos_lmax(apply_A, Sdiag, steps: int = 30, seed: int = LANCZOS_SEED):
    """Largest Ritz value of S A after ``steps`` Lanczos steps from a SplitMix64 vector."""
    v0 = splitmix64_uniform(seed, len(Sdiag))
    a, b = lanczos_tridiagonal(apply_A, Sdiag, v0, steps)
    if len(a) == 1:
        return float(a[0])
    return float(sla.eigh_tridiagonal(a, b, eigvals_only=True)[-1])


def gmres(apply_A, precond, b, rtol: float = 1e-6, restart: int = 20, maxit: int = 1000):
    """Right-preconditioned restarted GMRES(m), classical Gram-Schmidt, x0 = 0.

    Returns (x, iterations, history).  One iteration = one Arnoldi step, i.e. one
    preconditioner application and one operator application.
    """
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    hist = [1.0]
    if bnorm == 0.0:
        return x, 0, hist
    its = 0
    r = b.copy()
    while its < maxit:
        beta = np.linalg.norm(r)
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        g = np.zeros(restart + 1)
        g[0] = beta
        j_done = 0
        for j in range(restart):
            z = precond(V[j])
            Z.append(z)
            w = apply_A(z)
            Vm = np.array(V)
            h = Vm @ w                        # classical Gram-Schmidt
            w = w - Vm.T @ h
            H[: j + 1, j] = h
            H[j + 1, j] = np.linalg.norm(w)
            its += 1
            j_done = j + 1
            y, res, *_ = np.linalg.lstsq(H[: j + 2, : j + 1], g[: j + 2], rcond=None)
            rel = np.linalg.norm(g[: j + 2] - H[: j + 2, : j + 1] @ y) / bnorm
            hist.append(rel)
            if rel <= rtol or H[j + 1, j] == 0.0 or its >= maxit:
                break
            V.append(w / H[j + 1, j])
        y = np.linalg.lstsq(H[: j_done + 1, :j_done], g[: j_done + 1], rcond=None)[0]
        x = x + np.array(Z[:j_done]).T @ y
        r = b - apply_A(x)
        if np.linalg.norm(r) / bnorm <= rtol:
            return x, its, hist
    raise NotConverged(f"GMRES did not reach {rtol} in {maxit} iterations")
