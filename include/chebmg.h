/*
 * chebmg -- Jacobi-scaled Chebyshev smoothing in symmetric and one-sided
 * multigrid V-cycles, as a preconditioner for a flexible CG solve of the
 * Poisson problem A u = b (Phillips & Fischer, "Optimal Chebyshev Smoothers and
 * One-sided V-cycles", arXiv 2210.03179).
 *
 * C ABI.  Every pointer argument documented "device" is a caller-owned CUDA
 * device pointer; "host" pointers are caller-owned host memory.  The library
 * owns only its context and the workspace it allocates in a setup call; it
 * never frees or retains caller memory.  All work is issued on the stream in
 * chebmg_opts.stream (NULL = the legacy default stream); calls that return a
 * host scalar synchronise that stream.
 *
 * Errors: every int-returning call returns CHEBMG_OK (0) or a negative code;
 * chebmg_strerror() names it and chebmg_last_error() gives a one-line
 * description of the most recent failure in this thread.  No C++ exception
 * and no abort crosses the ABI.  A context is not thread-safe: calls on one
 * context must be serialised by the caller.
 *
 * Vector layout:
 *   SEM level of order N on an nex x ney x nez box: the global GLL lattice
 *     (NX, NY, NZ) = (nex N + 1, ney N + 1, nez N + 1), n = NX NY NZ, global id
 *     (gz NY + gy) NX + gx.  Nodes on the cube boundary are Dirichlet nodes: they
 *     are ignored on input and written 0 on output.
 *   FD level: the mx x my interior grid, x fastest (index j mx + i).
 * Precision: "dtype" arguments select FP64 (CHEBMG_F64, double*) or FP32
 * (CHEBMG_F32, float*) vectors.  FP32 level data exists only in a context set
 * up with prec = CHEBMG_FP32_SMOOTHER; vcycle/pcg_solve/coarse_solve vectors are
 * always FP64.
 */
#ifndef CHEBMG_H
#define CHEBMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define CHEBMG_OK 0
#define CHEBMG_EINVAL -1      /* bad argument (size, level, kind, dtype, pointer) */
#define CHEBMG_ECUDA -2       /* a CUDA runtime call failed */
#define CHEBMG_ENOTCONV -3    /* tolerance not reached within maxit; outputs valid */
#define CHEBMG_EBREAKDOWN -4  /* p^T A p <= 0, NaN/Inf residual, or Lanczos breakdown */
#define CHEBMG_ETIMEOUT -5    /* a bounded device wait gave up; context still usable, but
                                 every output of that call is undefined (a copy may still
                                 have landed late): re-run the call from its inputs.  The
                                 solvers zero u before returning it. */
#define CHEBMG_ENOMEM -6      /* device allocation failed */
#define CHEBMG_EMESH -7       /* mesh with a non-positive Jacobian */

/* ---- options ------------------------------------------------------------- */
typedef struct chebmg_ctx chebmg_ctx;

/* Smoother kinds (Sec. 2): Algorithm 1 with lambda_min = lmin_ratio lambda_max
 * ("1st-Cheb"), Algorithm 2 with beta_i = 1 (4th kind), Algorithm 2 with the
 * optimized beta_i of Table 5 (Sec. 8.1). */
enum { CHEBMG_CHEB_1ST = 1, CHEBMG_CHEB_4TH = 4, CHEBMG_CHEB_4TH_OPT = 5 };
/* V-cycle shape (Sec. 2, Eqs. 2.2 and 2.4): symmetric (k,k) or one-sided (2k,0). */
enum { CHEBMG_SYMMETRIC = 0, CHEBMG_ONE_SIDED = 1 };
/* Precision policy: all FP64, or FP32 smoother/Ax/transfers inside an FP64
 * outer solve (FP64 dots, Lanczos and coarse solve). */
enum { CHEBMG_FP64 = 0, CHEBMG_FP32_SMOOTHER = 1 };
enum { CHEBMG_F64 = 0, CHEBMG_F32 = 1 };

typedef struct {
  int kind;              /* CHEBMG_CHEB_1ST | CHEBMG_CHEB_4TH | CHEBMG_CHEB_4TH_OPT */
  int order;             /* k >= 1: (k,k) symmetric or (2k,0) one-sided */
  int sided;             /* CHEBMG_SYMMETRIC | CHEBMG_ONE_SIDED */
  int prec;              /* CHEBMG_FP64 | CHEBMG_FP32_SMOOTHER */
  double lmin_ratio;     /* 1st kind: lambda_min / lambda_max (0.1); <= 0: for each smoothing
                            order the ratio that maximises gamma^{-1} (Eq. 2.14; Eq. 2.24 fits it) */
  double lmax_scale;     /* multiplies the Lanczos estimate (1.0) */
  int lanczos_steps;     /* Lanczos steps per level (30) */
  const double* lmax_override; /* host, one per smoothed level, or NULL */
  double coarse_rtol;    /* SEM p=1 coarse CG relative tolerance (1e-10) */
  int coarse_maxit;      /* SEM coarse CG iteration cap (5000) */
  void* stream;          /* cudaStream_t, NULL = default stream */
} chebmg_opts;

/* Fill opts with the defaults listed above (kind 4th-opt, order 2, one-sided, FP64). */
void chebmg_default_opts(chebmg_opts* opts);

/* ---- setup ------------------------------------------------------------------ */

/* 2-D five-point Poisson problem of Sec. 3 on [0,Lx] x [0,Ly] with an m x m
 * interior grid (h = L/(m+1)); geometric coarsening by `coarsening` (2, or 8
 * for the aggressive n/8 hierarchy) while the grid is larger than `coarsest`;
 * Galerkin coarse operators A_{j+1} = P^T A_j P (Eq. 2.1) with bilinear P, and a
 * dense Cholesky solve on the coarsest grid.  Requires (m+1) divisible by the
 * coarsening factor at every level.  Returns EINVAL on bad sizes. */
int chebmg_setup_fd2d(int m, double Lx, double Ly, int coarsening, int coarsest,
                      const chebmg_opts* opts, chebmg_ctx** ctx);

/* 3-D spectral-element Poisson problem (Sec. 1, Eq. 1.3) with p-multigrid
 * (Sec. 4.1) on an nex x ney x nez box of trilinear hexahedra.
 * verts: host, (nez+1)(ney+1)(nex+1) x 3 doubles, [vz][vy][vx][xyz], copied.
 * orders: host, nlevels polynomial orders, strictly decreasing, each in 1..9
 *   (e.g. {7, 3, 1}); the last level is solved by FP64 Jacobi-PCG to coarse_rtol.
 * Returns EMESH if any quadrature point has a non-positive Jacobian. */
int chebmg_setup_sem(int nex, int ney, int nez, const double* verts, const int* orders,
                     int nlevels, const chebmg_opts* opts, chebmg_ctx** ctx);

/* SEM on a general conforming hexahedral mesh (the problem statement's A u = b on any mesh,
 * Sec. 1; the operator of Eq. 1.3 with isoparametric geometry).  Host arrays, copied:
 *   coords:    E * (N+1)^3 * 3 doubles, the GLL point coordinates of each element at order N,
 *              point (i, j, k) at index ((k (N+1) + j) (N+1) + i) * 3 (x, y, z); points shared
 *              by several elements must have the same coordinates in each;
 *   gid:       E * (N+1)^3 global ids in [0, n), every id used;
 *   dirichlet: n bytes, nonzero = Dirichlet node (removed from the system);
 *   orders:    decreasing, orders[0] = N (e.g. {7, 3, 1}).
 * Each element must be positively oriented (its GLL Jacobian determinant > 0 everywhere; EMESH
 * otherwise).  Coarser orders use the Lagrange interpolation of the coordinates and a numbering
 * derived from the mesh topology (shared vertices, edges and faces found through the ids of
 * their corner nodes); a coarse node is a Dirichlet node when every order-N node of its element
 * vertex, edge or face is one.  Vectors of level j are in that level's numbering (level 0:
 * the caller's gid).  Kernels that index through the box lattice are not used for such
 * contexts. */
int chebmg_setup_sem_mesh(int64_t E, int N, const double* coords, const int64_t* gid, int64_t n,
                          const uint8_t* dirichlet, const int* orders, int nlevels,
                          const chebmg_opts* opts, chebmg_ctx** ctx);

void chebmg_destroy(chebmg_ctx* ctx);

/* ---- queries ---------------------------------------------------------------- */
int chebmg_num_levels(const chebmg_ctx* ctx, int* nlevels);
/* Number of entries n of level-`level` vectors. */
int chebmg_level_size(const chebmg_ctx* ctx, int level, int64_t* n);
/* lambda_max of S A used by the smoother on `level` (after lmax_scale/override). */
int chebmg_lambda_max(const chebmg_ctx* ctx, int level, double* out);
/* Kernel launches issued by this library in this process (ctx unused; for accounting). */
int chebmg_launch_count(const chebmg_ctx* ctx, int64_t* count);
/* Variant chosen by the setup-time autotuner for the order-7 element operator on `level`
 * in `dtype`: 1, 2 or 4 elements per thread block, or 12 / 14 for the persistent pipelined
 * kernel with 2 / 4 elements per block, or 21 / 22 for 1 / 2 elements per block with the
 * geometric factors read from global memory where used (no shared-memory copy: more blocks
 * per SM), or 31 / 32 for the persistent kernel with 1 / 2 elements per block and one
 * geometric-factor buffer (refilled during the second half of each element batch: half the
 * shared memory, more blocks per SM); +100 when global ids are computed from the box lattice instead of read from the
 * element-to-global map.  Order-3 levels (N = 3): 40 for one thread per element point, 41
 * for line passes (16 threads per element, one 4-point line each, synchronised within the
 * warp), 141 for line passes with lattice ids.  0 for levels of other orders. */
int chebmg_tile_choice(const chebmg_ctx* ctx, int level, int dtype, int* elements_per_block);
/* Overrides that choice (same codes); EINVAL for other levels or codes. */
/* SEM coarse solver: PCG whose preconditioner is Algorithm 2 (4th kind, beta = 1) of
 * `degree` applied from zero with Jacobi scaling (degree 1 = Jacobi-PCG), chosen at setup
 * by timing; lmax = lambda_max of S A on the coarse level (FP64 Lanczos). */
int chebmg_coarse_info(const chebmg_ctx* ctx, int* degree, double* lmax);
/* Kernels of the SEM coarse CG (same method, same status words):
 *   CHEBMG_COARSE_GRID    one persistent cooperative launch over up to one block per SM;
 *                         products exchange rows through global memory as 64-bit words that
 *                         carry the value and its exchange tag together (no separate flag),
 *                         grid-wide reductions on an arrival counter (any coarse mesh);
 *   CHEBMG_COARSE_CLUSTER one thread-block cluster (up to 16 CTAs): box lattices at N = 1 with
 *                         the FP32 preconditioner; the operator's FP32 copy and the exchanged
 *                         vectors in shared memory, halos through distributed shared memory,
 *                         hardware cluster barriers;
 *   CHEBMG_COARSE_HOST    host-driven loop of kernels (cooperative launch unavailable). */
enum { CHEBMG_COARSE_HOST = 0, CHEBMG_COARSE_GRID = 1, CHEBMG_COARSE_CLUSTER = 2 };
/* Kernel chosen at setup (timed together with the degree), its thread blocks and the rows
 * each block owns (grid: a power of two times 256; cluster: planes x lattice plane). */
int chebmg_coarse_shape(const chebmg_ctx* ctx, int* kernel, int* blocks, int* rows_per_block);
/* Overrides the coarse kernel (GRID or CLUSTER); EINVAL where it does not apply. */
int chebmg_set_coarse_kernel(chebmg_ctx* ctx, int kernel);

/* Arithmetic of the outer Krylov product q = A p on the finest level (chebmg_pcg_solve;
 * the operator of Sec. 1, Eq. 1.3):
 *   CHEBMG_OUTER_FP64   FP64 (default);
 *   CHEBMG_OUTER_F32X2  the order-7 operator in FP64-class arithmetic on pairs of FP32 values
 *                       (value = hi + lo, about 48 significant bits; additions sum the high
 *                       parts exactly (TwoSum) and the low parts in FP32, products use the
 *                       fused-multiply-add error term), the
 *                       geometric factors kept as such pairs (8 bytes per value).  Relative
 *                       error near 1e-14 per application; FP32 exponent range (|values| well
 *                       inside 1e-30 .. 1e30).  GB300 executes FP32 at a large multiple of its
 *                       FP64 rate.  Opt-in: the first call converts the factors and times the
 *                       kernel variants.  EINVAL unless the finest level is SEM of order 7.
 * Everything else in the solve (residual update, dot products, preconditioner) is unchanged. */
enum { CHEBMG_OUTER_FP64 = 0, CHEBMG_OUTER_F32X2 = 1 };
int chebmg_set_outer_operator(chebmg_ctx* ctx, int kind);
/* y = A x on the finest level with the context's outer operator (FP64 device vectors). */
int chebmg_apply_outer(chebmg_ctx* ctx, const double* x, double* y);
int chebmg_set_coarse_degree(chebmg_ctx* ctx, int degree);
int chebmg_set_tile_choice(chebmg_ctx* ctx, int level, int dtype, int variant);

/* Fused smoother on order-7 box-lattice levels (Algorithms 1 and 2 with the operator of
 * Sec. 1, Eq. 1.3): every step of a smoother application -- element operator with
 * gather-scatter, Chebyshev recurrence with the Jacobi scaling, residual update -- and, in a
 * V-cycle, the restriction residual r = b - A x (Eq. 2.2) run in one persistent launch that
 * takes work items (elements of one element plane, or nodes of one plane range) in dependency
 * order, instead of two kernels per step.  Variant per level and dtype, chosen at setup by
 * timing against the separate kernels: 0 = separate kernels, 1 = FP32 (2 elements per work
 * item), 2 = FP64 (1 element per work item).  Batches have their own choice (below).  Same
 * results as the separate kernels up to the order of the atomic sums. */
int chebmg_fused_smoother(const chebmg_ctx* ctx, int level, int dtype, int* variant);
/* Overrides that choice; EINVAL on other levels (not order 7, not a box lattice, the
 * coarsest) or a variant that does not match dtype. */
int chebmg_set_fused_smoother(chebmg_ctx* ctx, int level, int dtype, int variant);
/* The same for batches of nrhs right-hand sides (allocating and tuning as the first batched
 * solve would): a work item of the fused kernel covers *rhs_per_item right-hand sides (the
 * geometric factors of its elements staged once for all of them); *variant 0 = separate
 * kernels (then *rhs_per_item = 0). */
int chebmg_batch_fused_smoother(chebmg_ctx* ctx, int nrhs, int level, int dtype, int* variant,
                                int* rhs_per_item);
/* Overrides that choice for batches of nrhs (variant 0, 1 for FP32 or 2 for FP64;
 * rhs_per_item 1..64); EINVAL as chebmg_set_fused_smoother. */
int chebmg_set_batch_fused_smoother(chebmg_ctx* ctx, int nrhs, int level, int dtype, int variant,
                                    int rhs_per_item);

/* ---- per-level operators (device vectors, dtype as above) ---------------- */

/* y = A x on `level`: SEM matrix-free element Ax with direct-stiffness
 * summation and Dirichlet mask (Eq. 1.3); FD five-point / Galerkin stencil. */
int chebmg_apply_A(chebmg_ctx* ctx, int level, int dtype, const void* x, void* y);

/* out = S = diag(A)^{-1} (Jacobi, Sec. 2), 0 on Dirichlet nodes. */
int chebmg_inv_diagonal(chebmg_ctx* ctx, int level, int dtype, void* out);

/* One smoother application of the context's kind and the given order on
 * `level` for A x = b: Algorithm 1 or 2 with x updated in place.  x_is_zero
 * skips the initial residual (x is then overwritten with the result). */
int chebmg_smooth(chebmg_ctx* ctx, int level, int dtype, const void* b, void* x, int order,
                  int x_is_zero);

/* rc = P^T rf from `level` to level+1 (SEM p-MG or FD bilinear restriction). */
int chebmg_restrict(chebmg_ctx* ctx, int level, int dtype, const void* rf, void* rc);

/* zf = P zc (accumulate = 0) or zf += P zc (accumulate = 1), level+1 -> level. */
int chebmg_prolong(chebmg_ctx* ctx, int level, int dtype, const void* zc, void* zf,
                   int accumulate);

/* z = A_l^{-1} r on the coarsest level: FD dense Cholesky; SEM preconditioned CG to
 * coarse_rtol (see chebmg_coarse_info; iters may be NULL).  FP64 device vectors. */
int chebmg_coarse_solve(chebmg_ctx* ctx, const double* r, double* z, int* iters);

/* ---- solver --------------------------------------------------------------- */

/* z = B r: one V-cycle (Eq. 2.2) from the finest level, FP64 device vectors. */
int chebmg_vcycle(chebmg_ctx* ctx, const double* r, double* z);

/* Flexible CG (x0 = 0) preconditioned by one V-cycle per iteration until
 * ||b - A u|| / ||b|| <= rtol (relative residual of Sec. 5.1).  b, u: FP64
 * device vectors.  iters, relres: host outputs (may be NULL).  history: host,
 * maxit+1 doubles of relative residuals, or NULL.  Returns ENOTCONV (u and
 * relres valid) if maxit is reached, EBREAKDOWN on p^T A p <= 0 or NaN. */
int chebmg_pcg_solve(chebmg_ctx* ctx, const double* b, double* u, double rtol, int maxit,
                     int* iters, double* relres, double* history);

/* Restarted flexible GMRES(restart) (x0 = 0), right preconditioned by one V-cycle per
 * iteration, classical Gram-Schmidt: the outer solver of the paper's experiments (Sec. 6.1) and
 * of its FD study (Table 1, Sec. 3).  Stops when the true relative residual ||b - A u|| / ||b||
 * <= rtol at the end of a restart cycle (a cycle ends early when the least-squares residual
 * estimate reaches rtol).  iters = Arnoldi steps = preconditioner applications.  history: host,
 * maxit+1 doubles of residual estimates, or NULL.  1 <= restart <= 64.  Returns ENOTCONV
 * (u and relres valid) after maxit steps. */
int chebmg_gmres_solve(chebmg_ctx* ctx, const double* b, double* u, double rtol, int restart,
                       int maxit, int* iters, double* relres, double* history);

/* Same as chebmg_pcg_solve with HOST b and u: copies b in and u out on the
 * context stream (end-to-end entry point). */
int chebmg_pcg_solve_host(chebmg_ctx* ctx, const double* b_host, double* u_host, double rtol,
                          int maxit, int* iters, double* relres);

/* ---- batches of right-hand sides ------------------------------------------------ */

/* The problem statement (Sec. 1) is a sequence of Poisson problems A u = b with one
 * operator: setup is amortised over many right-hand sides.  These calls solve several of
 * them at once. */
typedef struct chebmg_group chebmg_group;

/* flags: capture each Krylov half-iteration as a CUDA graph and replay it (needs a coarse
 * solve without host decisions: FD, or an SEM coarsest level of at most 3072 nodes;
 * otherwise the flag is ignored and the same kernels are launched one by one). */
#define CHEBMG_BATCH_GRAPH 1

/* nrhs independent chebmg_pcg_solve problems in one pass: every operator, transfer,
 * smoother and reduction kernel processes all right-hand sides in one launch (the order-7
 * operator stages each element's geometric factors once for several right-hand sides), each
 * right-hand side with its own FCG scalars and stopping test; one that has converged is
 * frozen while the others iterate, so iterations and results equal those of separate
 * solves up to rounding.  B, U: FP64 device arrays [nrhs][n] (right-hand side q at q*n).
 * iters, relres: host arrays of nrhs entries (may be NULL).  1 <= nrhs <= 65535.  The
 * first call for a batch size allocates nrhs copies of the work vectors and times the
 * batched kernel variants on the context's data (autotuning).  Returns the worst status
 * over the batch: EBREAKDOWN before ENOTCONV before OK; ETIMEOUT if a bounded device wait
 * gave up. */
int chebmg_pcg_solve_batched(chebmg_ctx* ctx, int nrhs, const double* B, double* U, double rtol,
                             int maxit, int flags, int* iters, double* relres);

/* Y = A X on `level` for nrhs vectors at once: X, Y device arrays [nrhs][n] of the dtype,
 * vector q at q*n.  Same kernels as the batched solve. */
int chebmg_apply_A_batched(chebmg_ctx* ctx, int level, int dtype, int nrhs, const void* X, void* Y);

/* Z = B R: one V-cycle (Eq. 2.2) for each of nrhs FP64 vectors, R, Z device arrays
 * [nrhs][n] of the finest level. */
int chebmg_vcycle_batched(chebmg_ctx* ctx, int nrhs, const double* R, double* Z);

/* Autotuned choices for batches of nrhs (allocating and tuning as the first batched solve
 * would): *variant = 1000 * right-hand sides per block + (100 if global ids come from the
 * box lattice) + elements per block of the batched order-7 operator on `level` (1, 2, 4; or
 * 11, 12 for 1 or 2 elements with the right-hand sides taken two at a time through every
 * line pass, at least 2 per block; or, FP32 only, 21, 22 for 1 or 2 elements with the geometric
 * factors held in registers across the block's right-hand sides instead of in shared memory)
 * (0 for other levels or nrhs = 1); *coarse_degree = degree of the Algorithm 2 preconditioner of the
 * per-right-hand-side coarse CG (0 if the coarsest level is not solved that way). */
int chebmg_batch_info(chebmg_ctx* ctx, int nrhs, int level, int dtype, int* variant,
                      int* coarse_degree);

/* Overrides the autotuned batched order-7 variant (encoding as in chebmg_batch_info) for
 * batches of nrhs >= 2 on `level`; EINVAL for other levels or a variant that does not fit. */
int chebmg_set_batch_tile_choice(chebmg_ctx* ctx, int nrhs, int level, int dtype, int variant);

/* A group of contexts on one device -- meshes of different sizes and polynomial orders --
 * each solving one right-hand side per chebmg_group_pcg_solve call.  Every context runs on
 * its own stream; with CHEBMG_BATCH_GRAPH each Krylov half-iteration of all of them is one
 * captured CUDA graph (fork/join over the streams), so the meshes' kernels overlap on the
 * GPU.  The contexts stay owned by the caller and must outlive the group; the group keeps
 * no reference to B or U.  Contexts must be distinct.  While a group call runs, its
 * contexts must not be used otherwise. */
int chebmg_group_create(chebmg_ctx* const* ctxs, int nctx, chebmg_group** group);
/* B[k], U[k]: FP64 device vectors of context k's finest level.  iters, relres: host arrays
 * of nctx entries (may be NULL).  Status as chebmg_pcg_solve_batched. */
int chebmg_group_pcg_solve(chebmg_group* group, const double* const* B, double* const* U,
                           double rtol, int maxit, int flags, int* iters, double* relres);
void chebmg_group_destroy(chebmg_group* group);

/* lambda_min / lambda_max that the 1st-kind smoother (Algorithm 1) of the given order uses in
 * this context: the fixed lmin_ratio, or the gamma^{-1}-optimal ratio (Sec. 2.4, Eq. 2.24)
 * when lmin_ratio <= 0 (computed on the host on first use, then cached). */
int chebmg_lambda_min_ratio(chebmg_ctx* ctx, int order, double* ratio);

/* Precision of the SEM coarse CG's polynomial preconditioner: CHEBMG_F64 (the default of an
 * FP64 context) or CHEBMG_F32 (the default of a CHEBMG_FP32_SMOOTHER context).  The CG itself -- iterate, residual, the products A p, the dot products and the
 * 1e-10 stopping test -- stays FP64 either way; with FP32 the preconditioner's products,
 * recurrence and neighbour exchanges use FP32 copies and the CG takes the flexible
 * (Polak-Ribiere) beta.  retune != 0 re-times the preconditioner degree for the new
 * precision.  EINVAL for contexts without an SEM coarse CG. */
int chebmg_set_coarse_precond_dtype(chebmg_ctx* ctx, int dtype, int retune);

/* ---- smoother weights and their gradient ----------------------------------------- */

/* Error reduction of `steps` V-cycles (Sec. 3, Eq. 3.1: observed convergence) and its
 * gradient.  With B one FP64 V-cycle (Eq. 2.2) whose Algorithm-2 smoother uses the weights
 * betas[0..nbeta-1] (beta_i of Sec. 2.3, for every smoothing call of the cycle) and
 * lambda_max_j = lmax_scale * (the context's lambda_max of level j), and E = I - B A:
 *   *f = (1/nrhs) sum_q ||E^steps e0_q||^2 / ||e0_q||^2 ,
 * and grad_betas[i] = df/dbeta_i, *grad_scale = df/dlmax_scale.  E0: FP64 device array
 * [nrhs][n] of the finest level (Dirichlet entries ignored).  f_each: host, nrhs values or
 * NULL.  The gradient is exact up to rounding: reverse mode through the cycle (A and S are
 * symmetric, so the adjoint is the transposed cycle), each cycle recomputed from its input
 * instead of being stored, all nrhs errors as one batch; the coarse solve is taken as the
 * linear map A_c^{-1} (its tolerance, coarse_rtol, bounds the error of that reading).
 * Needs a 4th-kind context (CHEBMG_CHEB_4TH or _4TH_OPT) with nbeta equal to the smoothing
 * order (pre, and post if nonzero).  The context's own weights are left unchanged.
 * grad_betas and grad_scale both NULL: the objective only (no adjoint pass). */
int chebmg_cycle_error_grad(chebmg_ctx* ctx, int nrhs, const double* E0, int steps,
                            const double* betas, int nbeta, double lmax_scale, double* f,
                            double* grad_betas, double* grad_scale, double* f_each);

/* Replaces the Algorithm-2 weights used by every later smoothing call of order nbeta (for
 * example weights tuned with chebmg_cycle_error_grad), and scales every level's lambda_max
 * by lmax_scale.  nbeta = 0 restores the defaults of the context's kind (lmax_scale still
 * applies). */
int chebmg_set_smoother_weights(chebmg_ctx* ctx, const double* betas, int nbeta, double lmax_scale);

/* ---- self-test -------------------------------------------------------------- */

/* Failure-path self-test of the persistent SEM coarse solver (not part of the paper's
 * method): launches it with one phantom block that never arrives at the grid barrier, so
 * every bounded wait runs out (after about a second), the kernel records a timeout and
 * returns instead of hanging.  *status receives the code the solver reports
 * (CHEBMG_ETIMEOUT expected); the context stays usable.  EINVAL if the context has no
 * persistent coarse solver. */
int chebmg_selftest_coarse_timeout(chebmg_ctx* ctx, int* status);

/* ---- allocation-free smoother ---------------------------------------------- */

/* The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory where they smooth (for example a plugin inside an application
 * whose device memory belongs entirely to that application's pool, or a real-time loop in
 * which cudaMalloc/cudaFree are forbidden because they may synchronise the device).
 *
 * Runs the same smoother as chebmg_smooth on level 0 of an FD context, without a context:
 * kind CHEBMG_CHEB_1ST (lambda_min = lmin_ratio * lmax), CHEBMG_CHEB_4TH or
 * CHEBMG_CHEB_4TH_OPT (order <= 16, the library's weight table) of the given order, on the
 * five-point operator of an m x m interior grid of [0,Lx] x [0,Ly] (spacing L/(m+1)), x
 * updated in place; lmax is lambda_max of S A supplied by the caller.  b, x: caller-owned
 * FP64 device vectors of m*m entries, x fastest.  No context, no device or host allocation:
 * the call makes no cudaMalloc, cudaFree or other allocating call.
 *
 * Limits and sharing: the work vectors live in one static device array of 4 x 262144
 * doubles (8 MiB) that every device which loads the library reserves until the process
 * exits; m*m > 262144 returns CHEBMG_EINVAL.  All calls on a device share that array and
 * each call overwrites what the previous one left there, so calls whose work may overlap
 * on the GPU (different streams, or host threads) race and must be serialised by the
 * caller.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, and looks it up again after the
 * device's context changes (a device reset); make that first call before any stream
 * capture.  Returns EINVAL on bad arguments, ECUDA on a CUDA error. */
int chebmg_fd_smooth_noalloc(int m, double Lx, double Ly, int kind, int order, double lmax,
                             double lmin_ratio, const double* b, double* x, int x_is_zero,
                             void* stream);

/* ---- utilities ----------------------------------------------------------------- */

/* out = in converted between CHEBMG_F32 and CHEBMG_F64 (or copied), n entries, device
 * vectors, on `stream` (NULL = default stream): the conversion kernel the mixed-precision solve
 * uses between its FP64 Krylov vectors and its FP32 V-cycle.  It converts in integer
 * arithmetic (GB300 issues hardware FP64 conversions at its small FP64 rate) and gives the
 * IEEE result: exact widening, narrowing rounded to nearest with ties to even.  EINVAL on bad
 * arguments. */
int chebmg_convert(const void* in, int in_dtype, void* out, int out_dtype, int64_t n, void* stream);

/* ---- errors ------------------------------------------------------------------ */
const char* chebmg_strerror(int code);
const char* chebmg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CHEBMG_H */
