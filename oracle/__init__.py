"""Plain FP64 CPU oracle for Jacobi-Chebyshev multigrid (Phillips & Fischer, arXiv 2210.03179).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library never
imports, links or calls anything here, and nothing here imports the CUDA
library: the two share no code.  The only shared inputs come from the seeded
generators in ``workloads/``.

Everything is written for clarity, not speed: numpy/scipy FP64 with library
primitives (matmul, sparse products, dense factorisations) as the only
building blocks, following the paper's statement of each step.

Modules
-------
gll        GLL nodes/weights, derivative and interpolation matrices (SEM basis).
sem        spectral-element Poisson operator A = Q^T blockdiag(A_e) Q (Sec. 1, Eq. 1.3),
           Jacobi diagonal, p-multigrid transfers (Sec. 4.1).
fd         2-D five-point Poisson operator, bilinear interpolation and Galerkin
           coarse operators (Sec. 3, Eq. 2.1).
chebyshev  Algorithm 1 (1st kind) and Algorithm 2 ((optimized) 4th kind), the
           optimized-beta table (Table 5, Sec. 8.1) and the simple smoother (Eq. 2.3).
multigrid  V-cycle error propagator, symmetric (k,k) and one-sided (2k,0)
           (Eqs. 2.2, 2.4-2.6).
krylov     flexible CG, Jacobi-PCG coarse solve, Lanczos lambda_max, SplitMix64.
sensitivity  error reduction of three V-cycles and its gradient with respect to the
           4th-kind weights and the lambda_max scale (forward mode).
theory     gamma^{-1}(k) (Eq. 2.14), closed forms (Eqs. 2.18-2.24), critical C
           (Eqs. 2.25-2.28), grid complexity (Eq. 3.2).

Equation numbers follow the paper's per-section numbering (Sec. 2 starts at
Eq. 2.1, the Galerkin coarse operator).

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, library routines or values printed in the paper, except where a
module header says "parity unpinned".
"""
