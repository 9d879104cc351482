"""The coarse CG on one thread-block cluster (box lattices at N = 1, FP32 preconditioner).

Interior lattice planes are split over up to 16 CTAs: one CTA, four CTAs with one plane each,
sixteen CTAs with an uneven split (two or three planes), and sixteen with two planes each.
Each case against the oracle's polynomial-preconditioned CG (Algorithm 2 of degree m inside
CG, Sec. 4.1): the 1e-10 residual, the oracle's iteration count within one, the solution to
1e-8; and against the grid-wide kernel on the same context.
"""
import numpy as np
import pytest

import workloads as W
from oracle import krylov as K
from oracle.sem import SemLevel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2210_03179_gb300 as cm  # noqa: E402
from gpu_util import N, T, empty, relerr  # noqa: E402

F32 = cm.CHEBMG_F32

# (elements per direction) -> lattice (ex+1) x (ey+1) x (ez+1), interior planes ez-1
MESHES = [(2, 3, 2),      # 1 interior plane: a cluster of one CTA
          (3, 4, 5),      # 4 planes, 4 CTAs
          (4, 3, 20),     # 19 planes over 16 CTAs: three CTAs hold two planes
          (6, 5, 40),     # 39 planes over 16 CTAs: seven hold three planes
          (5, 5, 33)]     # 32 planes, two per CTA


@pytest.mark.parametrize("mesh", MESHES)
def test_cluster_coarse_cg_matches_oracle(mesh):
    v = W.sem_box_vertices(*mesh)
    s = cm.Solver("sem", verts=v, orders=(2, 1), prec="mixed", lmax=[1.0])
    Lc = SemLevel(v, 1)
    Lc.invD = Lc.inv_diagonal()
    cm.chebmg_set_coarse_kernel(s.ctx, cm.CHEBMG_COARSE_CLUSTER)
    kern, blocks, rows = cm.chebmg_coarse_shape(s.ctx)
    planes = mesh[2] - 1
    assert kern == cm.CHEBMG_COARSE_CLUSTER and blocks == min(16, planes)
    assert rows == -(-planes // blocks) * (mesh[0] + 1) * (mesh[1] + 1)
    _, lc = cm.chebmg_coarse_info(s.ctx)
    r = np.random.default_rng(11).uniform(-1, 1, Lc.n)
    r[Lc.dirichlet] = 0
    for deg in (1, 4, 12):
        cm.chebmg_set_coarse_degree(s.ctx, deg)
        z = empty(Lc.n)
        z.fill_(np.nan)        # every entry, Dirichlet planes included, must be written
        iters = cm.chebmg_coarse_solve(s.ctx, T(r), z)
        zz = N(z)
        assert np.isfinite(zz).all()
        assert np.all(zz[Lc.dirichlet] == 0.0)
        assert np.linalg.norm(r - Lc.apply_A(zz)) <= 1.01e-10 * np.linalg.norm(r)
        x_ref, it_ref = K.pcg_cheb4(Lc.apply_A, Lc.invD, r, lc, deg, 1e-10)
        assert abs(iters - it_ref) <= 1, (mesh, deg, iters, it_ref)
        assert relerr(zz, x_ref) < 1e-8
        # the grid-wide kernel on the same context: same method, same iterations within one
        cm.chebmg_set_coarse_kernel(s.ctx, cm.CHEBMG_COARSE_GRID)
        z2 = empty(Lc.n)
        it2 = cm.chebmg_coarse_solve(s.ctx, T(r), z2)
        assert abs(it2 - iters) <= 1 and relerr(N(z2), zz) < 1e-8
        cm.chebmg_set_coarse_kernel(s.ctx, cm.CHEBMG_COARSE_CLUSTER)
    s.close()


def test_cluster_kernel_zero_rhs_and_refusals():
    v = W.sem_box_vertices(3, 4, 5)
    s = cm.Solver("sem", verts=v, orders=(2, 1), prec="mixed", lmax=[1.0])
    cm.chebmg_set_coarse_kernel(s.ctx, cm.CHEBMG_COARSE_CLUSTER)
    n = SemLevel(v, 1).n
    z = empty(n)
    z.fill_(1.0)
    assert cm.chebmg_coarse_solve(s.ctx, T(np.zeros(n)), z) == 0
    assert float(z.abs().max()) == 0.0
    # an FP64 preconditioner falls back to the grid-wide kernel; the cluster kernel is refused
    cm.chebmg_set_coarse_precond_dtype(s.ctx, cm.CHEBMG_F64, retune=False)
    assert cm.chebmg_coarse_shape(s.ctx)[0] == cm.CHEBMG_COARSE_GRID
    with pytest.raises(cm.ChebmgError):
        cm.chebmg_set_coarse_kernel(s.ctx, cm.CHEBMG_COARSE_CLUSTER)
    s.close()
    # general (non-box) meshes have no lattice: refused
    from test_gpu_mesh import general_mesh
    L, coords, gid, dirichlet, _ = general_mesh(v, 2, seed=3)
    g = cm.Solver("sem_mesh", coords=coords, gid=gid, n=L.n, dirichlet=dirichlet, orders=(2, 1), prec="mixed",
                  lmax=[1.0])
    with pytest.raises(cm.ChebmgError):
        cm.chebmg_set_coarse_kernel(g.ctx, cm.CHEBMG_COARSE_CLUSTER)
    g.close()


def test_mixed_solve_through_the_cluster_kernel():
    # the benchmark's cycle at a small size with the coarse CG forced onto the cluster kernel
    from oracle import multigrid as M
    from oracle import problems as P
    mesh = (4, 4, 6)
    v = W.sem_box_vertices(*mesh)
    H = P.sem_hierarchy(v, (7, 3, 1), kind="opt4th", k=3, sided="one-sided")
    s = cm.Solver("sem", verts=v, orders=(7, 3, 1), kind="opt4th", order=3, sided="one-sided", prec="mixed",
                  lmax=[L.lmax for L in H.levels[:-1]])
    cm.chebmg_set_coarse_kernel(s.ctx, cm.CHEBMG_COARSE_CLUSTER)
    b = W.sem_rhs(*mesh, 7)
    _, it_ref, _ = K.fcg(H.levels[0].apply_A, lambda r: M.vcycle(H, r), b, 1e-8)
    u = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, T(b), u, 1e-8, 100)
    assert code == cm.CHEBMG_OK and rel <= 1e-8 and abs(it - it_ref) <= 1, (it, it_ref)
    assert np.linalg.norm(b - H.levels[0].apply_A(N(u))) <= 1.01e-8 * np.linalg.norm(b)
    s.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_grid_kernel_on_a_many_block_lattice(prec):
    # E = 16^3 at N = 1: 17^3 nodes over 20 blocks, the coarse operator in lattice slot order.
    # Every degree must reach 1e-10 within one iteration of the oracle, repeatedly (a block that
    # ran two exchanges ahead of a neighbour would show up as a timeout or a wrong count).
    v = W.sem_box_vertices(16, 16, 16)
    s = cm.Solver("sem", verts=v, orders=(2, 1), prec=prec, lmax=[1.0])
    cm.chebmg_set_coarse_kernel(s.ctx, cm.CHEBMG_COARSE_GRID)
    kern, blocks, _ = cm.chebmg_coarse_shape(s.ctx)
    assert kern == cm.CHEBMG_COARSE_GRID and blocks > 1
    Lc = SemLevel(v, 1)
    Lc.invD = Lc.inv_diagonal()
    _, lc = cm.chebmg_coarse_info(s.ctx)
    rng = np.random.default_rng(5)
    for deg in (1, 8, 16):
        cm.chebmg_set_coarse_degree(s.ctx, deg)
        r = rng.uniform(-1, 1, Lc.n)      # Dirichlet entries included: the solver ignores them
        _, it_ref = K.pcg_cheb4(Lc.apply_A, Lc.invD, np.where(Lc.dirichlet, 0.0, r), lc, deg, 1e-10)
        for rep in range(3):
            z = empty(Lc.n)
            iters = cm.chebmg_coarse_solve(s.ctx, T(r), z)
            rr = np.where(Lc.dirichlet, 0.0, r)
            assert np.linalg.norm(rr - Lc.apply_A(N(z))) <= 1.01e-10 * np.linalg.norm(rr)
            assert abs(iters - it_ref) <= 1, (prec, deg, iters, it_ref)
    s.close()
