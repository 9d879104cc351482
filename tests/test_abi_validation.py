"""Argument checks of the C ABI on the CPU: every malformed setup or option is refused with
CHEBMG_EINVAL and a message, before any device call (no GPU needed)."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def cm():
    import __graft_entry__ as g
    g.build()
    import paper_2210_03179_gb300 as m
    return m


def _opts(cm, **kw):
    o = cm.chebmg_opts()
    cm.lib().chebmg_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _fd(cm, o, m=63, Lx=1.0, Ly=1.0, c=2, coarsest=7):
    ctx = ctypes.c_void_p(1234)
    code = cm.lib().chebmg_setup_fd2d(m, Lx, Ly, c, coarsest, ctypes.byref(o), ctypes.byref(ctx))
    return code, ctx.value


def _einval(cm, code, ctx, fragment):
    assert code == cm.CHEBMG_EINVAL
    assert ctx is None                        # the output handle is cleared on failure
    assert fragment in cm.lib().chebmg_last_error().decode()


@pytest.mark.parametrize("field,value,fragment", [
    ("kind", 3, "kind"),
    ("order", 0, "order"),
    ("order", 9, "tabulated up to order 16"),           # one-sided (18, 0) of the optimized kind
    ("sided", 2, "sided"),
    ("prec", 7, "prec"),
    ("lmax_scale", 0.0, "lmax_scale"),
    ("lanczos_steps", 0, "lanczos_steps"),
    ("coarse_rtol", 0.0, "coarse"),
    ("coarse_maxit", 0, "coarse"),
])
def test_bad_options_are_refused(cm, field, value, fragment):
    code, ctx = _fd(cm, _opts(cm, **{field: value}))
    _einval(cm, code, ctx, fragment)


def test_first_kind_lambda_min_ratio_must_stay_below_one(cm):
    code, ctx = _fd(cm, _opts(cm, kind=cm.CHEBMG_CHEB_1ST, lmin_ratio=1.0))
    _einval(cm, code, ctx, "lmin_ratio")


@pytest.mark.parametrize("args,fragment", [
    (dict(m=0), "bad FD sizes"),
    (dict(Lx=0.0), "bad FD sizes"),
    (dict(Ly=-1.0), "bad FD sizes"),
    (dict(c=1), "bad FD sizes"),
    (dict(m=62), "not divisible"),
    (dict(m=63, c=8, coarsest=3), "below one unknown"),  # 63 -> 7 -> (7+1)/8 - 1 = 0 unknowns
    (dict(m=47, c=8, coarsest=3), "not divisible"),       # 48 / 8 = 6 -> 5, then 6 is not divisible by 8
])
def test_bad_fd_grids_are_refused(cm, args, fragment):
    code, ctx = _fd(cm, _opts(cm), **args)
    _einval(cm, code, ctx, fragment)


def _sem(cm, nex, ney, nez, orders, verts=True):
    v = np.zeros((nez + 1, ney + 1, nex + 1, 3)) if verts else None
    ords = (ctypes.c_int * len(orders))(*orders)
    ctx = ctypes.c_void_p(1234)
    o = _opts(cm)
    vp = v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if verts else None
    code = cm.lib().chebmg_setup_sem(nex, ney, nez, vp, ords, len(orders), ctypes.byref(o), ctypes.byref(ctx))
    return code, ctx.value


@pytest.mark.parametrize("mesh,orders,fragment", [
    ((2, 2, 2), (7, 3, 3), "decrease"),
    ((2, 2, 2), (3, 7, 1), "decrease"),
    ((2, 2, 2), (10, 3, 1), "1..9"),
    ((2, 2, 2), (7, 3, 0), "1..9"),
    ((0, 2, 2), (7, 3, 1), "bad SEM arguments"),
    ((147, 147, 147), (7, 3, 1), "30-bit"),                 # (147*7+1)^3 > 2^30 nodes
])
def test_bad_sem_boxes_are_refused(cm, mesh, orders, fragment):
    code, ctx = _sem(cm, *mesh, orders)
    _einval(cm, code, ctx, fragment)


def test_sem_box_without_vertices_is_refused(cm):
    code, ctx = _sem(cm, 2, 2, 2, (7, 3, 1), verts=False)
    _einval(cm, code, ctx, "bad SEM arguments")


def _mesh(cm, E, N, n, orders, gid_fill=0, bad_gid=None):
    NP = (N + 1) ** 3
    coords = np.zeros(E * NP * 3)
    gid = np.full(E * NP, gid_fill, dtype=np.int64)
    if bad_gid is not None:
        gid[-1] = bad_gid
    dirichlet = np.zeros(min(max(n, 1), 1 << 16), dtype=np.uint8)   # never read by the refused calls
    ords = (ctypes.c_int * len(orders))(*orders)
    ctx = ctypes.c_void_p(1234)
    o = _opts(cm)
    code = cm.lib().chebmg_setup_sem_mesh(
        E, N, coords.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        gid.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n,
        dirichlet.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), ords, len(orders), ctypes.byref(o),
        ctypes.byref(ctx))
    return code, ctx.value


@pytest.mark.parametrize("E,N,n,orders,bad_gid,fragment", [
    (1, 3, 64, (2, 1), None, "orders[0] must be the mesh order"),
    (1, 3, 64, (3, 3), None, "decrease"),
    (1, 3, 64, (3, 1), 64, "out of range"),
    (1, 3, 64, (3, 1), -1, "out of range"),
    (1, 10, 64, (10, 1), None, "bad SEM mesh arguments"),
    (0, 3, 64, (3, 1), None, "bad SEM mesh arguments"),
    (1, 3, 1 << 30, (3, 1), None, "30-bit"),
])
def test_bad_general_meshes_are_refused(cm, E, N, n, orders, bad_gid, fragment):
    code, ctx = _mesh(cm, E, N, n, orders, bad_gid=bad_gid)
    _einval(cm, code, ctx, fragment)


def test_calls_on_a_null_context_are_refused(cm):
    L = cm.lib()
    assert L.chebmg_apply_A(None, 0, 0, None, None) == cm.CHEBMG_EINVAL
    assert L.chebmg_vcycle(None, None, None) == cm.CHEBMG_EINVAL
    it, rel = ctypes.c_int(), ctypes.c_double()
    assert L.chebmg_pcg_solve(None, None, None, 1e-8, 10, ctypes.byref(it), ctypes.byref(rel), None) \
        == cm.CHEBMG_EINVAL
    assert "NULL" in L.chebmg_last_error().decode() or "ctx" in L.chebmg_last_error().decode()
