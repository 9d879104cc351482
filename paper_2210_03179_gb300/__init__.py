"""Python binding of libchebmg: Jacobi-Chebyshev multigrid on GB300 (arXiv 2210.03179).

Argument marshalling only.  Every step of the smoother, the V-cycle and the
outer Krylov solve runs in the CUDA kernels of ``libchebmg.so`` behind the C ABI
declared in ``include/chebmg.h``; this module checks tensors, passes device
pointers and the current torch stream, and turns status codes into
exceptions.  There is no CPU fallback: if the shared library is missing the
first call raises.

The module-level functions carry the C names (``chebmg_apply_A`` ...);
``Solver`` is a small owner object around one context.
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, byref, c_double, c_int, c_int64, c_void_p
from pathlib import Path

import numpy as np

LIB_PATH = Path(__file__).resolve().parent / "libchebmg.so"

CHEBMG_OK = 0
CHEBMG_EINVAL = -1
CHEBMG_ECUDA = -2
CHEBMG_ENOTCONV = -3
CHEBMG_EBREAKDOWN = -4
CHEBMG_ETIMEOUT = -5
CHEBMG_ENOMEM = -6
CHEBMG_EMESH = -7

CHEBMG_CHEB_1ST = 1
CHEBMG_CHEB_4TH = 4
CHEBMG_CHEB_4TH_OPT = 5
CHEBMG_SYMMETRIC = 0
CHEBMG_ONE_SIDED = 1
CHEBMG_FP64 = 0
CHEBMG_FP32_SMOOTHER = 1
CHEBMG_F64 = 0
CHEBMG_F32 = 1
CHEBMG_COARSE_HOST = 0
CHEBMG_COARSE_GRID = 1
CHEBMG_COARSE_CLUSTER = 2
CHEBMG_OUTER_FP64 = 0
CHEBMG_OUTER_F32X2 = 1

KINDS = {"1st": CHEBMG_CHEB_1ST, "4th": CHEBMG_CHEB_4TH, "opt4th": CHEBMG_CHEB_4TH_OPT}
SIDED = {"symmetric": CHEBMG_SYMMETRIC, "one-sided": CHEBMG_ONE_SIDED}


class ChebmgError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {detail} (status {code})")
        self.code = code


class chebmg_opts(ctypes.Structure):
    _fields_ = [
        ("kind", c_int),
        ("order", c_int),
        ("sided", c_int),
        ("prec", c_int),
        ("lmin_ratio", c_double),
        ("lmax_scale", c_double),
        ("lanczos_steps", c_int),
        ("lmax_override", POINTER(c_double)),
        ("coarse_rtol", c_double),
        ("coarse_maxit", c_int),
        ("stream", c_void_p),
    ]


_lib = None

_SIGNATURES = {
    "chebmg_default_opts": (None, [POINTER(chebmg_opts)]),
    "chebmg_setup_fd2d": (c_int, [c_int, c_double, c_double, c_int, c_int, POINTER(chebmg_opts),
                                  POINTER(c_void_p)]),
    "chebmg_setup_sem": (c_int, [c_int, c_int, c_int, POINTER(c_double), POINTER(c_int), c_int,
                                 POINTER(chebmg_opts), POINTER(c_void_p)]),
    "chebmg_setup_sem_mesh": (c_int, [c_int64, c_int, POINTER(c_double), POINTER(c_int64), c_int64,
                                      POINTER(ctypes.c_uint8), POINTER(c_int), c_int, POINTER(chebmg_opts),
                                      POINTER(c_void_p)]),
    "chebmg_destroy": (None, [c_void_p]),
    "chebmg_num_levels": (c_int, [c_void_p, POINTER(c_int)]),
    "chebmg_level_size": (c_int, [c_void_p, c_int, POINTER(c_int64)]),
    "chebmg_lambda_max": (c_int, [c_void_p, c_int, POINTER(c_double)]),
    "chebmg_launch_count": (c_int, [c_void_p, POINTER(c_int64)]),
    "chebmg_tile_choice": (c_int, [c_void_p, c_int, c_int, POINTER(c_int)]),
    "chebmg_set_tile_choice": (c_int, [c_void_p, c_int, c_int, c_int]),
    "chebmg_fused_smoother": (c_int, [c_void_p, c_int, c_int, POINTER(c_int)]),
    "chebmg_set_fused_smoother": (c_int, [c_void_p, c_int, c_int, c_int]),
    "chebmg_convert": (c_int, [c_void_p, c_int, c_void_p, c_int, c_int64, c_void_p]),
    "chebmg_batch_fused_smoother": (c_int, [c_void_p, c_int, c_int, c_int, POINTER(c_int), POINTER(c_int)]),
    "chebmg_set_batch_fused_smoother": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int]),
    "chebmg_set_coarse_precond_dtype": (c_int, [c_void_p, c_int, c_int]),
    "chebmg_lambda_min_ratio": (c_int, [c_void_p, c_int, POINTER(c_double)]),
    "chebmg_coarse_info": (c_int, [c_void_p, POINTER(c_int), POINTER(c_double)]),
    "chebmg_coarse_shape": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    "chebmg_set_coarse_kernel": (c_int, [c_void_p, c_int]),
    "chebmg_set_outer_operator": (c_int, [c_void_p, c_int]),
    "chebmg_apply_outer": (c_int, [c_void_p, c_void_p, c_void_p]),
    "chebmg_set_coarse_degree": (c_int, [c_void_p, c_int]),
    "chebmg_apply_A": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "chebmg_inv_diagonal": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "chebmg_smooth": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_int, c_int]),
    "chebmg_restrict": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "chebmg_prolong": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_int]),
    "chebmg_coarse_solve": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(c_int)]),
    "chebmg_vcycle": (c_int, [c_void_p, c_void_p, c_void_p]),
    "chebmg_pcg_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int, POINTER(c_int),
                                 POINTER(c_double), POINTER(c_double)]),
    "chebmg_gmres_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int, c_int, POINTER(c_int),
                                   POINTER(c_double), POINTER(c_double)]),
    "chebmg_pcg_solve_host": (c_int, [c_void_p, POINTER(c_double), POINTER(c_double), c_double, c_int,
                                      POINTER(c_int), POINTER(c_double)]),
    "chebmg_fd_smooth_noalloc": (c_int, [c_int, c_double, c_double, c_int, c_int, c_double, c_double, c_void_p,
                                         c_void_p, c_int, c_void_p]),
    "chebmg_pcg_solve_batched": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_double, c_int, c_int,
                                         POINTER(c_int), POINTER(c_double)]),
    "chebmg_apply_A_batched": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]),
    "chebmg_vcycle_batched": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "chebmg_cycle_error_grad": (c_int, [c_void_p, c_int, c_void_p, c_int, POINTER(c_double), c_int, c_double,
                                        POINTER(c_double), POINTER(c_double), POINTER(c_double),
                                        POINTER(c_double)]),
    "chebmg_set_smoother_weights": (c_int, [c_void_p, POINTER(c_double), c_int, c_double]),
    "chebmg_batch_info": (c_int, [c_void_p, c_int, c_int, c_int, POINTER(c_int), POINTER(c_int)]),
    "chebmg_set_batch_tile_choice": (c_int, [c_void_p, c_int, c_int, c_int, c_int]),
    "chebmg_group_create": (c_int, [POINTER(c_void_p), c_int, POINTER(c_void_p)]),
    "chebmg_group_pcg_solve": (c_int, [c_void_p, POINTER(c_void_p), POINTER(c_void_p), c_double, c_int, c_int,
                                       POINTER(c_int), POINTER(c_double)]),
    "chebmg_group_destroy": (None, [c_void_p]),
    "chebmg_selftest_coarse_timeout": (c_int, [c_void_p, POINTER(c_int)]),
    "chebmg_strerror": (ctypes.c_char_p, [c_int]),
    "chebmg_last_error": (ctypes.c_char_p, []),
}


def lib():
    """Load libchebmg.so (built by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() first")
        handle = ctypes.CDLL(str(LIB_PATH))
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _check(code: int, where: str, allow=()):
    if code != CHEBMG_OK and code not in allow:
        L = lib()
        raise ChebmgError(code, where, f"{L.chebmg_strerror(code).decode()}: {L.chebmg_last_error().decode()}")
    return code


def _torch():
    import torch
    return torch


def _ptr(t, n: int, dtype: int, what: str):
    torch = _torch()
    want = torch.float64 if dtype == CHEBMG_F64 else torch.float32
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != want or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{what}: need a contiguous {want} tensor of {n} entries, got {t.dtype} {tuple(t.shape)}")
    return c_void_p(t.data_ptr())


def _stream_handle(stream=None):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return c_void_p(s.cuda_stream)


def chebmg_default_opts(kind="opt4th", order=2, sided="one-sided", prec="fp64", lmin_ratio=0.1,
                        lmax_scale=1.0, lanczos_steps=30, coarse_rtol=1e-10, coarse_maxit=5000,
                        stream=None) -> chebmg_opts:
    o = chebmg_opts()
    lib().chebmg_default_opts(byref(o))
    o.kind = KINDS[kind] if isinstance(kind, str) else int(kind)
    o.order = int(order)
    o.sided = SIDED[sided] if isinstance(sided, str) else int(sided)
    o.prec = {"fp64": CHEBMG_FP64, "mixed": CHEBMG_FP32_SMOOTHER}[prec] if isinstance(prec, str) else int(prec)
    o.lmin_ratio = lmin_ratio
    o.lmax_scale = lmax_scale
    o.lanczos_steps = lanczos_steps
    o.coarse_rtol = coarse_rtol
    o.coarse_maxit = coarse_maxit
    o.stream = _stream_handle(stream)
    return o


def chebmg_setup_fd2d(m, Lx, Ly, coarsening, coarsest, opts) -> c_void_p:
    ctx = c_void_p()
    _check(lib().chebmg_setup_fd2d(int(m), float(Lx), float(Ly), int(coarsening), int(coarsest), byref(opts),
                                   byref(ctx)), "chebmg_setup_fd2d")
    return ctx


def chebmg_setup_sem(nex, ney, nez, verts, orders, opts) -> c_void_p:
    verts = np.ascontiguousarray(verts, dtype=np.float64)
    if verts.shape != (nez + 1, ney + 1, nex + 1, 3):
        raise ValueError("verts must have shape (nez+1, ney+1, nex+1, 3)")
    ords = (c_int * len(orders))(*[int(o) for o in orders])
    ctx = c_void_p()
    _check(lib().chebmg_setup_sem(int(nex), int(ney), int(nez), verts.ctypes.data_as(POINTER(c_double)), ords,
                                  len(orders), byref(opts), byref(ctx)), "chebmg_setup_sem")
    return ctx


def chebmg_setup_sem_mesh(coords, gid, n, dirichlet, orders, opts) -> c_void_p:
    """coords: (E, (N+1)^3, 3) float64; gid: (E, (N+1)^3) int64 in [0, n); dirichlet: (n,) bool/uint8."""
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    gid = np.ascontiguousarray(gid, dtype=np.int64)
    dirichlet = np.ascontiguousarray(dirichlet, dtype=np.uint8)
    E, NP = gid.shape
    N = int(round(NP ** (1.0 / 3.0))) - 1
    if (N + 1) ** 3 != NP or coords.shape != (E, NP, 3) or dirichlet.shape != (int(n),):
        raise ValueError("coords (E, (N+1)^3, 3), gid (E, (N+1)^3), dirichlet (n,)")
    ords = (c_int * len(orders))(*[int(o) for o in orders])
    ctx = c_void_p()
    _check(lib().chebmg_setup_sem_mesh(E, N, coords.ctypes.data_as(POINTER(c_double)),
                                       gid.ctypes.data_as(POINTER(c_int64)), int(n),
                                       dirichlet.ctypes.data_as(POINTER(ctypes.c_uint8)), ords, len(orders),
                                       byref(opts), byref(ctx)), "chebmg_setup_sem_mesh")
    return ctx


def chebmg_destroy(ctx):
    lib().chebmg_destroy(ctx)


def chebmg_num_levels(ctx) -> int:
    v = c_int()
    _check(lib().chebmg_num_levels(ctx, byref(v)), "chebmg_num_levels")
    return v.value


def chebmg_level_size(ctx, level) -> int:
    v = c_int64()
    _check(lib().chebmg_level_size(ctx, int(level), byref(v)), "chebmg_level_size")
    return v.value


def chebmg_lambda_max(ctx, level) -> float:
    v = c_double()
    _check(lib().chebmg_lambda_max(ctx, int(level), byref(v)), "chebmg_lambda_max")
    return v.value


def chebmg_launch_count(ctx=None) -> int:
    v = c_int64()
    _check(lib().chebmg_launch_count(ctx, byref(v)), "chebmg_launch_count")
    return v.value


def chebmg_tile_choice(ctx, level, dtype) -> int:
    v = c_int()
    _check(lib().chebmg_tile_choice(ctx, int(level), int(dtype), byref(v)), "chebmg_tile_choice")
    return v.value


def chebmg_set_coarse_precond_dtype(ctx, dtype, retune=True):
    _check(lib().chebmg_set_coarse_precond_dtype(ctx, int(dtype), 1 if retune else 0),
           "chebmg_set_coarse_precond_dtype")


def chebmg_lambda_min_ratio(ctx, order) -> float:
    v = c_double()
    _check(lib().chebmg_lambda_min_ratio(ctx, int(order), byref(v)), "chebmg_lambda_min_ratio")
    return v.value


def chebmg_coarse_info(ctx):
    """(degree of the coarse CG's polynomial preconditioner, lambda_max of the coarse level)."""
    m, l = c_int(), c_double()
    _check(lib().chebmg_coarse_info(ctx, byref(m), byref(l)), "chebmg_coarse_info")
    return m.value, l.value


def chebmg_coarse_shape(ctx):
    """(kernel, thread blocks, rows per block) of the coarse CG (CHEBMG_COARSE_* kernels)."""
    k, g, r = c_int(), c_int(), c_int()
    _check(lib().chebmg_coarse_shape(ctx, byref(k), byref(g), byref(r)), "chebmg_coarse_shape")
    return k.value, g.value, r.value


def chebmg_set_coarse_kernel(ctx, kernel: int) -> None:
    _check(lib().chebmg_set_coarse_kernel(ctx, int(kernel)), "chebmg_set_coarse_kernel")


def chebmg_set_outer_operator(ctx, kind: int) -> None:
    _check(lib().chebmg_set_outer_operator(ctx, int(kind)), "chebmg_set_outer_operator")


def chebmg_apply_outer(ctx, x, y) -> None:
    n = chebmg_level_size(ctx, 0)
    _check(lib().chebmg_apply_outer(ctx, _ptr(x, n, CHEBMG_F64, "x"), _ptr(y, n, CHEBMG_F64, "y")),
           "chebmg_apply_outer")


def chebmg_set_coarse_degree(ctx, degree):
    _check(lib().chebmg_set_coarse_degree(ctx, int(degree)), "chebmg_set_coarse_degree")


def chebmg_set_tile_choice(ctx, level, dtype, variant):
    _check(lib().chebmg_set_tile_choice(ctx, int(level), int(dtype), int(variant)), "chebmg_set_tile_choice")


def chebmg_fused_smoother(ctx, level, dtype) -> int:
    """Fused-smoother variant of `level` in `dtype` (0: separate kernels)."""
    v = c_int()
    _check(lib().chebmg_fused_smoother(ctx, int(level), int(dtype), byref(v)), "chebmg_fused_smoother")
    return v.value


def chebmg_set_fused_smoother(ctx, level, dtype, variant):
    _check(lib().chebmg_set_fused_smoother(ctx, int(level), int(dtype), int(variant)), "chebmg_set_fused_smoother")


def chebmg_batch_fused_smoother(ctx, nrhs, level, dtype):
    """(variant, right-hand sides per work item) of the fused smoother for batches of nrhs."""
    v, g = c_int(), c_int()
    _check(lib().chebmg_batch_fused_smoother(ctx, int(nrhs), int(level), int(dtype), byref(v), byref(g)),
           "chebmg_batch_fused_smoother")
    return v.value, g.value


def chebmg_set_batch_fused_smoother(ctx, nrhs, level, dtype, variant, rhs_per_item=8):
    _check(lib().chebmg_set_batch_fused_smoother(ctx, int(nrhs), int(level), int(dtype), int(variant),
                                                 int(rhs_per_item)), "chebmg_set_batch_fused_smoother")


def chebmg_apply_A(ctx, level, dtype, x, y):
    n = chebmg_level_size(ctx, level)
    _check(lib().chebmg_apply_A(ctx, int(level), dtype, _ptr(x, n, dtype, "x"), _ptr(y, n, dtype, "y")),
           "chebmg_apply_A")


def chebmg_inv_diagonal(ctx, level, dtype, out):
    n = chebmg_level_size(ctx, level)
    _check(lib().chebmg_inv_diagonal(ctx, int(level), dtype, _ptr(out, n, dtype, "out")), "chebmg_inv_diagonal")


def chebmg_smooth(ctx, level, dtype, b, x, order, x_is_zero):
    n = chebmg_level_size(ctx, level)
    _check(lib().chebmg_smooth(ctx, int(level), dtype, _ptr(b, n, dtype, "b"), _ptr(x, n, dtype, "x"), int(order),
                               1 if x_is_zero else 0), "chebmg_smooth")


def chebmg_restrict(ctx, level, dtype, rf, rc):
    nf, nc = chebmg_level_size(ctx, level), chebmg_level_size(ctx, level + 1)
    _check(lib().chebmg_restrict(ctx, int(level), dtype, _ptr(rf, nf, dtype, "rf"), _ptr(rc, nc, dtype, "rc")),
           "chebmg_restrict")


def chebmg_prolong(ctx, level, dtype, zc, zf, accumulate=False):
    nf, nc = chebmg_level_size(ctx, level), chebmg_level_size(ctx, level + 1)
    _check(lib().chebmg_prolong(ctx, int(level), dtype, _ptr(zc, nc, dtype, "zc"), _ptr(zf, nf, dtype, "zf"),
                                1 if accumulate else 0), "chebmg_prolong")


def chebmg_coarse_solve(ctx, r, z) -> int:
    n = chebmg_level_size(ctx, chebmg_num_levels(ctx) - 1)
    it = c_int()
    _check(lib().chebmg_coarse_solve(ctx, _ptr(r, n, CHEBMG_F64, "r"), _ptr(z, n, CHEBMG_F64, "z"), byref(it)),
           "chebmg_coarse_solve", allow=(CHEBMG_ENOTCONV,))
    return it.value


def chebmg_vcycle(ctx, r, z):
    n = chebmg_level_size(ctx, 0)
    _check(lib().chebmg_vcycle(ctx, _ptr(r, n, CHEBMG_F64, "r"), _ptr(z, n, CHEBMG_F64, "z")), "chebmg_vcycle")


def chebmg_pcg_solve(ctx, b, u, rtol=1e-8, maxit=500, history=False):
    """Returns (status, iterations, relres, history-or-None); raises on errors other than ENOTCONV."""
    n = chebmg_level_size(ctx, 0)
    it, rel = c_int(), c_double()
    hist = (c_double * (maxit + 1))() if history else None
    code = _check(lib().chebmg_pcg_solve(ctx, _ptr(b, n, CHEBMG_F64, "b"), _ptr(u, n, CHEBMG_F64, "u"),
                                         float(rtol), int(maxit), byref(it), byref(rel), hist),
                  "chebmg_pcg_solve", allow=(CHEBMG_ENOTCONV,))
    h = list(hist)[: it.value + 1] if history else None
    return code, it.value, rel.value, h


def chebmg_gmres_solve(ctx, b, u, rtol=1e-6, restart=20, maxit=500, history=False):
    """Returns (status, iterations, relres, history-or-None); raises on errors other than ENOTCONV."""
    n = chebmg_level_size(ctx, 0)
    it, rel = c_int(), c_double()
    hist = (c_double * (maxit + 1))() if history else None
    code = _check(lib().chebmg_gmres_solve(ctx, _ptr(b, n, CHEBMG_F64, "b"), _ptr(u, n, CHEBMG_F64, "u"),
                                           float(rtol), int(restart), int(maxit), byref(it), byref(rel), hist),
                  "chebmg_gmres_solve", allow=(CHEBMG_ENOTCONV,))
    h = list(hist)[: it.value + 1] if history else None
    return code, it.value, rel.value, h


def chebmg_pcg_solve_host(ctx, b_host: np.ndarray, u_host: np.ndarray, rtol=1e-8, maxit=500):
    n = chebmg_level_size(ctx, 0)
    for a in (b_host, u_host):
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != n:
            raise ValueError("host vectors must be contiguous float64 of the fine-level size")
    it, rel = c_int(), c_double()
    code = _check(lib().chebmg_pcg_solve_host(ctx, b_host.ctypes.data_as(POINTER(c_double)),
                                              u_host.ctypes.data_as(POINTER(c_double)), float(rtol), int(maxit),
                                              byref(it), byref(rel)),
                  "chebmg_pcg_solve_host", allow=(CHEBMG_ENOTCONV,))
    return code, it.value, rel.value


CHEBMG_BATCH_GRAPH = 1


def chebmg_pcg_solve_batched(ctx, B, U, rtol=1e-8, maxit=500, graph=True):
    """B, U: contiguous FP64 CUDA tensors of shape (nrhs, n).  Returns (status, iterations[nrhs],
    relres[nrhs]); raises on errors other than ENOTCONV."""
    torch = _torch()
    n = chebmg_level_size(ctx, 0)
    if not isinstance(B, torch.Tensor) or B.dim() != 2 or B.shape[1] != n:
        raise ValueError(f"B must have shape (nrhs, {n})")
    nrhs = B.shape[0]
    its, rel = (c_int * nrhs)(), (c_double * nrhs)()
    code = _check(lib().chebmg_pcg_solve_batched(ctx, nrhs, _ptr(B, nrhs * n, CHEBMG_F64, "B"),
                                                 _ptr(U, nrhs * n, CHEBMG_F64, "U"), float(rtol), int(maxit),
                                                 CHEBMG_BATCH_GRAPH if graph else 0, its, rel),
                  "chebmg_pcg_solve_batched", allow=(CHEBMG_ENOTCONV,))
    return code, list(its), list(rel)


def chebmg_apply_A_batched(ctx, level, dtype, X, Y):
    """X, Y: contiguous CUDA tensors of shape (nrhs, n) of the dtype."""
    n = chebmg_level_size(ctx, level)
    if X.dim() != 2 or X.shape[1] != n:
        raise ValueError(f"X must have shape (nrhs, {n})")
    nrhs = X.shape[0]
    _check(lib().chebmg_apply_A_batched(ctx, int(level), int(dtype), nrhs, _ptr(X, nrhs * n, dtype, "X"),
                                        _ptr(Y, nrhs * n, dtype, "Y")), "chebmg_apply_A_batched")


def chebmg_vcycle_batched(ctx, R, Z):
    """R, Z: contiguous FP64 CUDA tensors of shape (nrhs, n)."""
    n = chebmg_level_size(ctx, 0)
    if R.dim() != 2 or R.shape[1] != n:
        raise ValueError(f"R must have shape (nrhs, {n})")
    nrhs = R.shape[0]
    _check(lib().chebmg_vcycle_batched(ctx, nrhs, _ptr(R, nrhs * n, CHEBMG_F64, "R"),
                                       _ptr(Z, nrhs * n, CHEBMG_F64, "Z")), "chebmg_vcycle_batched")


def chebmg_cycle_error_grad(ctx, E0, betas, lmax_scale=1.0, steps=3):
    """E0: contiguous FP64 CUDA tensor (nrhs, n).  Returns (f, grad_betas list, grad_scale, f_each list)."""
    n = chebmg_level_size(ctx, 0)
    if E0.dim() != 2 or E0.shape[1] != n:
        raise ValueError(f"E0 must have shape (nrhs, {n})")
    nrhs = E0.shape[0]
    k = len(betas)
    b = (c_double * k)(*[float(v) for v in betas])
    f, gs = c_double(), c_double()
    gb, fe = (c_double * k)(), (c_double * nrhs)()
    _check(lib().chebmg_cycle_error_grad(ctx, nrhs, _ptr(E0, nrhs * n, CHEBMG_F64, "E0"), int(steps), b, k,
                                         float(lmax_scale), byref(f), gb, byref(gs), fe), "chebmg_cycle_error_grad")
    return f.value, list(gb), gs.value, list(fe)


def chebmg_cycle_error(ctx, E0, betas, lmax_scale=1.0, steps=3):
    """The objective of chebmg_cycle_error_grad alone: (f, f_each list)."""
    n = chebmg_level_size(ctx, 0)
    if E0.dim() != 2 or E0.shape[1] != n:
        raise ValueError(f"E0 must have shape (nrhs, {n})")
    nrhs = E0.shape[0]
    k = len(betas)
    b = (c_double * k)(*[float(v) for v in betas])
    f, fe = c_double(), (c_double * nrhs)()
    _check(lib().chebmg_cycle_error_grad(ctx, nrhs, _ptr(E0, nrhs * n, CHEBMG_F64, "E0"), int(steps), b, k,
                                         float(lmax_scale), byref(f), None, None, fe), "chebmg_cycle_error_grad")
    return f.value, list(fe)


def chebmg_set_smoother_weights(ctx, betas=(), lmax_scale=1.0):
    k = len(betas)
    b = (c_double * max(k, 1))(*[float(v) for v in betas])
    _check(lib().chebmg_set_smoother_weights(ctx, b, k, float(lmax_scale)), "chebmg_set_smoother_weights")


def chebmg_batch_info(ctx, nrhs, level=0, dtype=CHEBMG_F64):
    """(batched order-7 variant, coarse preconditioner degree) autotuned for batches of nrhs."""
    v, m = c_int(), c_int()
    _check(lib().chebmg_batch_info(ctx, int(nrhs), int(level), int(dtype), byref(v), byref(m)), "chebmg_batch_info")
    return v.value, m.value


def chebmg_set_batch_tile_choice(ctx, nrhs, level, dtype, variant):
    _check(lib().chebmg_set_batch_tile_choice(ctx, int(nrhs), int(level), int(dtype), int(variant)),
           "chebmg_set_batch_tile_choice")


def chebmg_group_create(ctxs) -> c_void_p:
    arr = (c_void_p * len(ctxs))(*[c.value for c in ctxs])
    g = c_void_p()
    _check(lib().chebmg_group_create(arr, len(ctxs), byref(g)), "chebmg_group_create")
    return g


def chebmg_group_pcg_solve(group, ctxs, B, U, rtol=1e-8, maxit=500, graph=True):
    """One right-hand side per context: B[k], U[k] FP64 CUDA vectors of context k's fine size."""
    k = len(ctxs)
    if len(B) != k or len(U) != k:
        raise ValueError("one B and one U per context")
    bp = (c_void_p * k)(*[_ptr(B[q], chebmg_level_size(ctxs[q], 0), CHEBMG_F64, "B").value for q in range(k)])
    up = (c_void_p * k)(*[_ptr(U[q], chebmg_level_size(ctxs[q], 0), CHEBMG_F64, "U").value for q in range(k)])
    its, rel = (c_int * k)(), (c_double * k)()
    code = _check(lib().chebmg_group_pcg_solve(group, bp, up, float(rtol), int(maxit),
                                               CHEBMG_BATCH_GRAPH if graph else 0, its, rel),
                  "chebmg_group_pcg_solve", allow=(CHEBMG_ENOTCONV,))
    return code, list(its), list(rel)


def chebmg_group_destroy(group):
    lib().chebmg_group_destroy(group)


def chebmg_selftest_coarse_timeout(ctx) -> int:
    """Runs the persistent coarse solver with a barrier that can never complete; returns its status."""
    st = c_int()
    _check(lib().chebmg_selftest_coarse_timeout(ctx, byref(st)), "chebmg_selftest_coarse_timeout")
    return st.value


def chebmg_convert(x, y, stream=None):
    """y = x converted (FP32 <-> FP64) by the library's conversion kernel; x, y CUDA tensors."""
    import torch
    dt = {torch.float32: CHEBMG_F32, torch.float64: CHEBMG_F64}
    if x.dtype not in dt or y.dtype not in dt or x.numel() != y.numel():
        raise ValueError("x, y: float32/float64 CUDA tensors of the same length")
    if not (x.is_cuda and y.is_cuda and x.is_contiguous() and y.is_contiguous()):
        raise ValueError("x, y must be contiguous CUDA tensors")
    _check(lib().chebmg_convert(c_void_p(x.data_ptr()), dt[x.dtype], c_void_p(y.data_ptr()), dt[y.dtype],
                                x.numel(), _stream_handle(stream)), "chebmg_convert")


def chebmg_fd_smooth_noalloc(m, Lx, Ly, kind, order, lmax, lmin_ratio, b, x, x_is_zero, stream=None):
    """Context-free FD smoother that allocates nothing (see include/chebmg.h)."""
    n = int(m) * int(m)
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    _check(lib().chebmg_fd_smooth_noalloc(int(m), float(Lx), float(Ly), k, int(order), float(lmax),
                                          float(lmin_ratio), _ptr(b, n, CHEBMG_F64, "b"), _ptr(x, n, CHEBMG_F64, "x"),
                                          1 if x_is_zero else 0, _stream_handle(stream)),
           "chebmg_fd_smooth_noalloc")


class Solver:
    """Owns one chebmg context.  ``kind`` in {'1st','4th','opt4th'}, ``sided`` in
    {'symmetric','one-sided'}, ``prec`` in {'fp64','mixed'}."""

    def __init__(self, problem: str, *, lmax=None, **kw):
        setup = {k: kw.pop(k) for k in list(kw) if k in ("m", "Lx", "Ly", "coarsening", "coarsest",
                                                           "nex", "ney", "nez", "verts", "orders",
                                                           "coords", "gid", "n", "dirichlet")}
        self._lmax = None
        self.opts = chebmg_default_opts(**kw)
        if lmax is not None:
            self._lmax = (c_double * len(lmax))(*[float(v) for v in lmax])
            self.opts.lmax_override = ctypes.cast(self._lmax, POINTER(c_double))
        self.ctx = None
        if problem == "fd2d":
            self.ctx = chebmg_setup_fd2d(setup["m"], setup.get("Lx", 1.0), setup.get("Ly", 1.0),
                                         setup.get("coarsening", 2), setup.get("coarsest", 7), self.opts)
        elif problem == "sem":
            v = setup["verts"]
            self.ctx = chebmg_setup_sem(v.shape[2] - 1, v.shape[1] - 1, v.shape[0] - 1, v,
                                        setup.get("orders", (7, 3, 1)), self.opts)
        elif problem == "sem_mesh":
            self.ctx = chebmg_setup_sem_mesh(setup["coords"], setup["gid"], setup["n"], setup["dirichlet"],
                                             setup.get("orders", (7, 3, 1)), self.opts)
        else:
            raise ValueError(problem)
        self.mixed = self.opts.prec == CHEBMG_FP32_SMOOTHER

    @property
    def num_levels(self):
        return chebmg_num_levels(self.ctx)

    def size(self, level=0):
        return chebmg_level_size(self.ctx, level)

    def lambda_max(self, level):
        return chebmg_lambda_max(self.ctx, level)

    def close(self):
        if self.ctx is not None and self.ctx.value:
            chebmg_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
