"""GPU-vs-oracle parity for the SEM path: element Ax + gather-scatter, Jacobi diagonal,
p-multigrid transfers, smoothers, coarse CG, V-cycle and flexible CG (Secs. 1, 2, 4.1)."""
import numpy as np
import pytest

import workloads as W
from oracle import krylov as K
from oracle import multigrid as M
from oracle import problems as P
from oracle.chebyshev import smooth as oracle_smooth
from oracle.sem import SemLevel, SemTransfer

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2210_03179_gb300 as cm  # noqa: E402
from gpu_util import N, T, empty, relerr  # noqa: E402

F64, F32 = cm.CHEBMG_F64, cm.CHEBMG_F32

# 3 x 4 x 5 = 60 elements: several thread blocks per level and a ragged last block
# (N = 1: 64 elements per block; N = 3: 8; N = 4: 8 -> 7 full + 4).
MESH = (3, 4, 5)


@pytest.fixture(scope="module")
def verts():
    return W.sem_box_vertices(*MESH)


def solver(v, orders, kind="opt4th", k=2, sided="one-sided", prec="fp64", lmax=None, **kw):
    return cm.Solver("sem", verts=v, orders=orders, kind=kind, order=k, sided=sided, prec=prec, lmax=lmax, **kw)


@pytest.mark.parametrize("orders", [(7, 3, 1), (7, 5, 3, 1), (9, 5, 2), (8, 4), (6, 1), (2, 1), (4, 3, 2, 1)])
def test_operator_diagonal_and_transfers(verts, orders):
    levels = [SemLevel(verts, Nn) for Nn in orders]
    s = solver(verts, orders, lmax=[1.0] * (len(orders) - 1))
    rng = np.random.default_rng(sum(orders))
    for j, L in enumerate(levels):
        assert s.size(j) == L.n
        x = rng.uniform(-1, 1, L.n)
        y = empty(L.n)
        cm.chebmg_apply_A(s.ctx, j, F64, T(x), y)
        ref = L.apply_A(x)
        assert relerr(N(y), ref) < 1e-12
        assert np.all(N(y)[L.dirichlet] == 0.0)
        d = empty(L.n)
        cm.chebmg_inv_diagonal(s.ctx, j, F64, d)
        assert relerr(N(d), L.inv_diagonal()) < 1e-12
    for j in range(len(levels) - 1):
        Tr = SemTransfer(levels[j], levels[j + 1])
        nf, nc = levels[j].n, levels[j + 1].n
        rf = rng.uniform(-1, 1, nf)
        rc = empty(nc)
        cm.chebmg_restrict(s.ctx, j, F64, T(rf), rc)
        assert relerr(N(rc), Tr.restrict(rf)) < 1e-12
        zc = rng.uniform(-1, 1, nc)
        zf = empty(nf)
        cm.chebmg_prolong(s.ctx, j, F64, T(zc), zf, accumulate=False)
        assert relerr(N(zf), Tr.prolong(zc)) < 1e-12
        base = rng.uniform(-1, 1, nf)
        base[levels[j].dirichlet] = 0
        zf = T(base)
        cm.chebmg_prolong(s.ctx, j, F64, T(zc), zf, accumulate=True)
        assert relerr(N(zf), base + Tr.prolong(zc)) < 1e-12
    s.close()


def test_dirichlet_inputs_are_ignored(verts):
    L = SemLevel(verts, 3)
    s = solver(verts, (3, 1), lmax=[1.0])
    x = np.random.default_rng(0).uniform(-1, 1, L.n)
    xz = x.copy()
    xz[L.dirichlet] = 0
    y1, y2 = empty(L.n), empty(L.n)
    cm.chebmg_apply_A(s.ctx, 0, F64, T(x), y1)
    cm.chebmg_apply_A(s.ctx, 0, F64, T(xz), y2)
    # FP64 atomics add element contributions in a run-dependent order: equal up to rounding
    assert relerr(N(y1), N(y2)) < 1e-14
    s.close()


@pytest.mark.parametrize("kind", ["1st", "4th", "opt4th"])
@pytest.mark.parametrize("order", [1, 2, 4, 6])
def test_smoother_matches_algorithms(verts, kind, order):
    H = P.sem_hierarchy(verts, (7, 3, 1), kind=kind, k=1, sided="symmetric")
    lmax = [L.lmax for L in H.levels[:-1]]
    s = solver(verts, (7, 3, 1), kind=kind, k=1, sided="symmetric", lmax=lmax)
    rng = np.random.default_rng(order)
    for j in range(2):
        L = H.levels[j]
        b = rng.uniform(-1, 1, L.n)
        b[L.dirichlet] = 0
        for x_zero in (True, False):
            x0 = None if x_zero else np.where(L.dirichlet, 0.0, rng.uniform(-1, 1, L.n))
            ref = oracle_smooth(L, b, order, kind, L.lmax, 0.1, x0=x0)
            x = empty(L.n) if x_zero else T(x0)
            cm.chebmg_smooth(s.ctx, j, F64, T(b), x, order, x_zero)
            assert relerr(N(x), ref) < 1e-12
    s.close()


def test_coarse_cg_and_lanczos(verts):
    H = P.sem_hierarchy(verts, (5, 3, 1))
    s = solver(verts, (5, 3, 1))
    for j, L in enumerate(H.levels[:-1]):
        assert abs(s.lambda_max(j) / L.lmax - 1) < 1e-10
    Lc = H.levels[-1]
    m, lc = cm.chebmg_coarse_info(s.ctx)
    assert 1 <= m <= 16
    assert abs(lc / K.lanczos_lmax(Lc.apply_A, Lc.invD, 30) - 1) < 1e-10
    r = np.random.default_rng(9).uniform(-1, 1, Lc.n)
    r[Lc.dirichlet] = 0
    # the autotuned degree, plain Jacobi (degree 1) and a high degree, each against the oracle
    for deg in (m, 1, 8):
        cm.chebmg_set_coarse_degree(s.ctx, deg)
        z = empty(Lc.n)
        iters = cm.chebmg_coarse_solve(s.ctx, T(r), z)
        zz = N(z)
        assert np.linalg.norm(r - Lc.apply_A(zz)) <= 1.01e-10 * np.linalg.norm(r)
        x_ref, it_ref = K.pcg_cheb4(Lc.apply_A, Lc.invD, r, lc, deg, 1e-10)
        assert abs(iters - it_ref) <= 1, (deg, iters, it_ref)
        assert relerr(zz, x_ref) < 1e-8
        if deg == 1:
            assert abs(iters - K.pcg_jacobi(Lc.apply_A, Lc.invD, r, 1e-10)[1]) <= 1
    # FP32 preconditioner (the mixed form's default): the FP64 CG still reaches 1e-10 and takes
    # the FP64 preconditioner's iteration count within one
    cm.chebmg_set_coarse_precond_dtype(s.ctx, F32, retune=False)
    for deg in (1, 8):
        cm.chebmg_set_coarse_degree(s.ctx, deg)
        z = empty(Lc.n)
        iters = cm.chebmg_coarse_solve(s.ctx, T(r), z)
        zz = N(z)
        assert np.linalg.norm(r - Lc.apply_A(zz)) <= 1.01e-10 * np.linalg.norm(r)
        x_ref, it_ref = K.pcg_cheb4(Lc.apply_A, Lc.invD, r, lc, deg, 1e-10)
        assert abs(iters - it_ref) <= 1, (deg, iters, it_ref)
        assert relerr(zz, x_ref) < 1e-8
    s.close()


@pytest.mark.parametrize("kind,k,sided", [("opt4th", 2, "one-sided"), ("4th", 2, "symmetric"),
                                          ("1st", 3, "symmetric"), ("opt4th", 1, "one-sided"),
                                          ("opt4th", 3, "one-sided")])
def test_vcycle(verts, kind, k, sided):
    H = P.sem_hierarchy(verts, (7, 3, 1), kind=kind, k=k, sided=sided)
    s = solver(verts, (7, 3, 1), kind=kind, k=k, sided=sided, lmax=[L.lmax for L in H.levels[:-1]])
    r = W.sem_rhs(*MESH, 7, seed=4)
    z = empty(len(r))
    cm.chebmg_vcycle(s.ctx, T(r), z)
    # the coarse CG stops at 1e-10, so the cycles agree to about that level
    assert relerr(N(z), M.vcycle(H, r)) < 1e-8
    s.close()


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("sided", ["one-sided", "symmetric"])
def test_pcg_solve_iterations_match(verts, k, sided):
    H = P.sem_hierarchy(verts, (7, 3, 1), kind="opt4th", k=k, sided=sided)
    s = solver(verts, (7, 3, 1), kind="opt4th", k=k, sided=sided, lmax=[L.lmax for L in H.levels[:-1]])
    b = W.sem_rhs(*MESH, 7)
    A = H.levels[0].apply_A
    x_ref, it_ref, hist_ref = K.fcg(A, lambda r: M.vcycle(H, r), b, 1e-8)
    u = empty(len(b))
    code, it, rel, hist = cm.chebmg_pcg_solve(s.ctx, T(b), u, 1e-8, 200, history=True)
    assert code == cm.CHEBMG_OK and rel <= 1e-8
    assert abs(it - it_ref) <= 1
    assert np.linalg.norm(b - A(N(u))) <= 1.01e-8 * np.linalg.norm(b)
    assert relerr(N(u), x_ref) < 1e-6
    s.close()


def test_mixed_precision_solve(verts):
    H = P.sem_hierarchy(verts, (7, 3, 1))
    lmax = [L.lmax for L in H.levels[:-1]]
    s64 = solver(verts, (7, 3, 1), lmax=lmax)
    s32 = solver(verts, (7, 3, 1), prec="mixed", lmax=lmax)
    b = W.sem_rhs(*MESH, 7)
    u64, u32 = empty(len(b)), empty(len(b))
    c64, it64, rel64, _ = cm.chebmg_pcg_solve(s64.ctx, T(b), u64, 1e-8, 200)
    c32, it32, rel32, _ = cm.chebmg_pcg_solve(s32.ctx, T(b), u32, 1e-8, 200)
    assert c64 == c32 == cm.CHEBMG_OK and rel32 <= 1e-8
    assert abs(it32 - it64) <= 1
    A = H.levels[0].apply_A
    x_ref, it_ref, _ = K.fcg(A, lambda r: M.vcycle(H, r), b, 1e-8)
    assert abs(it32 - it_ref) <= 1 and abs(it64 - it_ref) <= 1
    assert np.linalg.norm(b - A(N(u32))) <= 1.01e-8 * np.linalg.norm(b)
    # FP32 operator and smoother vs FP64 oracle: single-precision error only
    L = H.levels[0]
    x = np.where(L.dirichlet, 0, np.random.default_rng(2).uniform(-1, 1, L.n))
    y = empty(L.n, True)
    cm.chebmg_apply_A(s32.ctx, 0, F32, T(x, torch.float32), y)
    assert relerr(N(y), A(x.astype(np.float32).astype(np.float64))) < 2e-5
    s64.close()
    s32.close()


def test_host_entry_point(verts):
    H = P.sem_hierarchy(verts, (5, 3, 1))
    s = solver(verts, (5, 3, 1), lmax=[L.lmax for L in H.levels[:-1]])
    b = W.sem_rhs(*MESH, 5)
    u = np.zeros_like(b)
    code, it, rel = cm.chebmg_pcg_solve_host(s.ctx, b, u, 1e-8, 200)
    assert code == cm.CHEBMG_OK and rel <= 1e-8
    assert np.linalg.norm(b - H.levels[0].apply_A(u)) <= 1.01e-8 * np.linalg.norm(b)
    s.close()


def test_setup_rejects_bad_input():
    v = W.sem_box_vertices(2, 2, 2)
    with pytest.raises(cm.ChebmgError):
        solver(v, (3, 5))                       # orders must decrease
    bad = v.copy()
    bad[1, 1, 1] = bad[1, 1, 1] + 0.9           # fold an element
    with pytest.raises(cm.ChebmgError) as e:
        solver(bad, (3, 1))
    assert e.value.code == cm.CHEBMG_EMESH


def test_bounded_barrier_wait_reports_timeout_and_context_survives(verts):
    # The persistent coarse solver waits at a grid barrier with a bounded spin; with a
    # phantom block that never arrives every wait runs out and the kernel returns a
    # timeout status instead of hanging.  The same context must still solve correctly.
    import time
    H = P.sem_hierarchy(verts, (3, 1), kind="opt4th", k=1, sided="symmetric")
    s = solver(verts, (3, 1), kind="opt4th", k=1, sided="symmetric", lmax=[H.levels[0].lmax])
    t0 = time.time()
    st = cm.chebmg_selftest_coarse_timeout(s.ctx)
    assert st == cm.CHEBMG_ETIMEOUT
    assert time.time() - t0 < 30
    Lc = H.levels[-1]
    r = np.where(Lc.dirichlet, 0.0, np.random.default_rng(1).uniform(-1, 1, Lc.n))
    z = empty(Lc.n)
    cm.chebmg_coarse_solve(s.ctx, T(r), z)
    assert np.linalg.norm(r - Lc.apply_A(N(z))) <= 1.01e-10 * np.linalg.norm(r)
    s.close()


@pytest.mark.parametrize("variant", [1, 2, 4, 12, 14, 21, 22, 31, 32, 101, 102, 104, 112, 114, 121, 122, 131, 132])
def test_every_order7_kernel_variant(verts, variant):
    # the setup autotuner may pick any of these; each must match the oracle
    L = SemLevel(verts, 7)
    s = solver(verts, (7, 3, 1), prec="mixed", lmax=[1.0, 1.0])
    assert cm.chebmg_tile_choice(s.ctx, 0, F64) % 100 in (1, 2, 4, 12, 14, 21, 22, 31, 32)
    x = np.where(L.dirichlet, 0.0, np.random.default_rng(variant).uniform(-1, 1, L.n))
    ref = L.apply_A(x)
    for dt, tol in ((F64, 1e-12), (F32, 2e-5)):
        if dt == F64 and variant % 100 == 14:
            # needs 264 KB of shared memory in FP64: rejected, and never picked by the autotuner
            with pytest.raises(cm.ChebmgError):
                cm.chebmg_set_tile_choice(s.ctx, 0, dt, variant)
            continue
        cm.chebmg_set_tile_choice(s.ctx, 0, dt, variant)
        if dt == F64:
            xt, y = T(x), empty(L.n)
            ref_d = ref
        else:
            xt, y = T(x, torch.float32), empty(L.n, True)
            ref_d = L.apply_A(x.astype(np.float32).astype(np.float64))
        cm.chebmg_apply_A(s.ctx, 0, dt, xt, y)
        assert relerr(N(y), ref_d) < tol, (variant, dt)
    with pytest.raises(cm.ChebmgError):
        cm.chebmg_set_tile_choice(s.ctx, 1, F64, 2)   # level 1 is order 3
    s.close()


# 3 x 3 x 3 = 27 elements: a ragged last element batch for 2 and 4 elements per block (MESH
# divides by both)
@pytest.mark.parametrize("variant", [2, 4, 12, 14, 22, 32, 102, 104, 112, 114, 122, 132])
def test_order7_variants_ragged_last_batch(variant):
    v = W.sem_box_vertices(3, 3, 3)
    L = SemLevel(v, 7)
    s = solver(v, (7, 3, 1), prec="mixed", lmax=[1.0, 1.0])
    x = np.where(L.dirichlet, 0.0, np.random.default_rng(variant + 1).uniform(-1, 1, L.n))
    for dt, tol in ((F64, 1e-12), (F32, 2e-5)):
        try:
            cm.chebmg_set_tile_choice(s.ctx, 0, dt, variant)
        except cm.ChebmgError:
            assert dt == F64 and variant % 100 == 14   # 264 KB of shared memory in FP64
            continue
        if dt == F64:
            xt, y, ref = T(x), empty(L.n), L.apply_A(x)
        else:
            xt, y = T(x, torch.float32), empty(L.n, True)
            ref = L.apply_A(x.astype(np.float32).astype(np.float64))
        cm.chebmg_apply_A(s.ctx, 0, dt, xt, y)
        assert relerr(N(y), ref) < tol, (variant, dt)
        assert np.all(N(y)[L.dirichlet] == 0.0)
    s.close()


@pytest.mark.parametrize("mesh", [MESH, (3, 3, 3)])
@pytest.mark.parametrize("variant", [40, 41, 141])
def test_order3_operator_variants(mesh, variant):
    # the order-3 level of a (7, 3, 1) hierarchy: one thread per point (40) or line passes with
    # map (41) or lattice (141) ids; 16 elements per line-pass block, so both meshes end in a
    # ragged block (60 = 3 x 16 + 12, 27 = 16 + 11)
    v = W.sem_box_vertices(*mesh)
    L = SemLevel(v, 3)
    s = solver(v, (7, 3, 1), prec="mixed", lmax=[1.0, 1.0])
    assert cm.chebmg_tile_choice(s.ctx, 1, F64) in (40, 41, 141)
    rng = np.random.default_rng(variant)
    x = np.where(L.dirichlet, 0.0, rng.uniform(-1, 1, L.n))
    for dt, tol in ((F64, 1e-12), (F32, 2e-5)):
        cm.chebmg_set_tile_choice(s.ctx, 1, dt, variant)
        if dt == F64:
            xt, y, ref = T(x), empty(L.n), L.apply_A(x)
        else:
            xt, y = T(x, torch.float32), empty(L.n, True)
            ref = L.apply_A(x.astype(np.float32).astype(np.float64))
        cm.chebmg_apply_A(s.ctx, 1, dt, xt, y)
        assert relerr(N(y), ref) < tol, (variant, dt)
        assert np.all(N(y)[L.dirichlet] == 0.0)
    # a batch of three vectors through the same kernel (one grid row per vector)
    X = rng.uniform(-1, 1, (3, L.n))
    Y = torch.zeros((3, L.n), dtype=torch.float64, device="cuda")
    cm.chebmg_apply_A_batched(s.ctx, 1, F64, T(X), Y)
    for q in range(3):
        assert relerr(N(Y[q]), L.apply_A(X[q])) < 1e-12
    with pytest.raises(cm.ChebmgError):
        cm.chebmg_set_tile_choice(s.ctx, 1, F64, 42)
    s.close()


@pytest.fixture(scope="module")
def many_batches():
    # 13 x 11 x 11 = 1573 elements: more element batches than resident blocks of every
    # persistent variant, so each block walks several batches (and the geometric-factor buffers
    # are refilled), with a ragged last batch for 2 and 4 elements per block
    v = W.sem_box_vertices(13, 11, 11)
    L = SemLevel(v, 7)
    s = solver(v, (7, 3, 1), prec="mixed", lmax=[1.0, 1.0])
    yield L, s
    s.close()


@pytest.mark.parametrize("variant", [12, 14, 31, 32, 112, 114, 131, 132])
def test_persistent_variants_several_batches_per_block(many_batches, variant):
    L, s = many_batches
    x = np.where(L.dirichlet, 0.0, np.random.default_rng(variant + 2).uniform(-1, 1, L.n))
    for dt, tol in ((F64, 1e-12), (F32, 2e-5)):
        try:
            cm.chebmg_set_tile_choice(s.ctx, 0, dt, variant)
        except cm.ChebmgError:
            assert dt == F64 and variant % 100 == 14
            continue
        if dt == F64:
            xt, y, ref = T(x), empty(L.n), L.apply_A(x)
        else:
            xt, y = T(x, torch.float32), empty(L.n, True)
            ref = L.apply_A(x.astype(np.float32).astype(np.float64))
        for _ in range(2):   # a second application over the same (re-zeroed) output
            cm.chebmg_apply_A(s.ctx, 0, dt, xt, y)
        assert relerr(N(y), ref) < tol, (variant, dt)
