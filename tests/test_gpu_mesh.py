"""SEM on a general conforming hexahedral mesh (chebmg_setup_sem_mesh).

The perturbed box is handed over as a general mesh -- elements in a random order, global ids
randomly relabelled, and every element's reference axes turned by a random proper rotation --
so the library must find shared vertices, edges and faces, and orient coarse-level nodes on them,
from the topology alone.  Everything must then agree with the box: the finest operator and
diagonal through the relabelling (1e-12), the coarse levels' spectra (permutation invariant),
and the solve's iteration count and solution.
"""
import numpy as np
import pytest

import workloads as W
from oracle import problems as P
from oracle.sem import SemLevel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2210_03179_gb300 as cm  # noqa: E402
from gpu_util import N, T, relerr  # noqa: E402

F64 = cm.CHEBMG_F64
MESH = (3, 4, 5)


def rotate(a, rots):
    """Apply proper rotations (np.rot90 in the given axis pairs) to an element array [k, j, i, ...]."""
    for axes in rots:
        a = np.rot90(a, 1, axes=axes)
    return a


def general_mesh(v, Nn, seed):
    L = SemLevel(v, Nn)
    E, Q = L.E, Nn + 1
    rng = np.random.default_rng(seed)
    order = rng.permutation(E)
    relabel = rng.permutation(L.n)           # new id of box id g
    X = L.coords                             # [e, k, j, i, 3]
    G = L.gid                                # [e, k, j, i]
    coords = np.empty((E, Q ** 3, 3))
    gid = np.empty((E, Q ** 3), dtype=np.int64)
    pairs = [(0, 1), (1, 2), (0, 2)]
    for new_e, old_e in enumerate(order):
        rots = [pairs[q] for q in rng.integers(0, 3, size=rng.integers(0, 4))]
        coords[new_e] = np.ascontiguousarray(rotate(X[old_e], rots)).reshape(-1, 3)
        gid[new_e] = relabel[np.ascontiguousarray(rotate(G[old_e], rots)).reshape(-1)]
    dirichlet = np.zeros(L.n, dtype=np.uint8)
    dirichlet[relabel[np.nonzero(L.dirichlet)[0]]] = 1
    return L, coords, gid, dirichlet, relabel


@pytest.fixture(scope="module")
def verts():
    return W.sem_box_vertices(*MESH)


def test_finest_operator_through_the_relabelling(verts):
    L, coords, gid, dirichlet, relabel = general_mesh(verts, 7, seed=1)
    s = cm.Solver("sem_mesh", coords=coords, gid=gid, n=L.n, dirichlet=dirichlet, orders=(7, 3, 1),
                  lmax=[1.0, 1.0])
    assert s.size(0) == L.n and s.num_levels == 3
    u = np.random.default_rng(2).uniform(-1, 1, L.n)
    un = np.empty_like(u)
    un[relabel] = u
    y = torch.zeros(L.n, dtype=torch.float64, device="cuda")
    cm.chebmg_apply_A(s.ctx, 0, F64, T(un), y)
    assert relerr(N(y)[relabel], L.apply_A(u)) < 1e-12
    d = torch.zeros_like(y)
    cm.chebmg_inv_diagonal(s.ctx, 0, F64, d)
    assert relerr(N(d)[relabel], L.inv_diagonal()) < 1e-12
    s.close()


@pytest.mark.parametrize("orders", [(7, 3, 1), (5, 2), (4, 3, 2, 1)])
def test_coarse_levels_match_the_box_spectrally(verts, orders):
    _, coords, gid, dirichlet, _ = general_mesh(verts, orders[0], seed=3)
    levels = [SemLevel(verts, Nn) for Nn in orders]
    s = cm.Solver("sem_mesh", coords=coords, gid=gid, n=levels[0].n, dirichlet=dirichlet, orders=orders,
                  lmax=[1.0] * (len(orders) - 1))
    for j in range(1, len(orders)):
        Lj = levels[j]
        assert s.size(j) == Lj.n
        live = ~Lj.dirichlet
        if Lj.n > 2500:
            continue
        # dense operator of the general mesh's level j, column by column (batched apply)
        Id = torch.eye(Lj.n, dtype=torch.float64, device="cuda")
        Y = torch.zeros_like(Id)
        cm.chebmg_apply_A_batched(s.ctx, j, F64, Id, Y)
        A = N(Y).T
        dvec = torch.zeros(Lj.n, dtype=torch.float64, device="cuda")
        cm.chebmg_inv_diagonal(s.ctx, j, F64, dvec)
        mask = N(dvec) != 0
        assert mask.sum() == live.sum()                          # same number of free nodes
        ev = np.linalg.eigvalsh(A[np.ix_(mask, mask)])
        ev_ref = np.linalg.eigvalsh(Lj.dense()[np.ix_(live, live)])
        assert np.abs(ev - ev_ref).max() <= 1e-10 * ev_ref.max()
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_matches_the_box(verts, prec):
    L, coords, gid, dirichlet, relabel = general_mesh(verts, 7, seed=4)
    H = P.sem_hierarchy(verts, (7, 3, 1))
    lmax = [Lv.lmax for Lv in H.levels[:-1]]
    box = cm.Solver("sem", verts=verts, orders=(7, 3, 1), prec=prec, lmax=lmax)
    gen = cm.Solver("sem_mesh", coords=coords, gid=gid, n=L.n, dirichlet=dirichlet, orders=(7, 3, 1),
                    prec=prec, lmax=lmax)
    b = W.sem_rhs(*MESH, 7)
    bn = np.empty_like(b)
    bn[relabel] = b
    u1 = torch.zeros(L.n, dtype=torch.float64, device="cuda")
    u2 = torch.zeros_like(u1)
    c1, it1, rel1, _ = cm.chebmg_pcg_solve(box.ctx, T(b), u1, 1e-8, 200)
    c2, it2, rel2, _ = cm.chebmg_pcg_solve(gen.ctx, T(bn), u2, 1e-8, 200)
    assert c1 == c2 == cm.CHEBMG_OK and rel2 <= 1e-8
    assert abs(it1 - it2) <= 1
    assert relerr(N(u2)[relabel], N(u1)) < 1e-7
    A = H.levels[0].apply_A
    assert np.linalg.norm(b - A(N(u2)[relabel])) <= 1.01e-8 * np.linalg.norm(b)
    box.close()
    gen.close()


def test_batched_solve_on_a_general_mesh(verts):
    L, coords, gid, dirichlet, relabel = general_mesh(verts, 7, seed=6)
    gen = cm.Solver("sem_mesh", coords=coords, gid=gid, n=L.n, dirichlet=dirichlet, orders=(7, 3, 1),
                    prec="mixed")
    B = torch.tensor(np.stack([W.sem_rhs(*MESH, 7, seed=q)[np.argsort(relabel)] for q in range(4)]),
                     device="cuda")
    U = torch.zeros_like(B)
    code, its, rel = cm.chebmg_pcg_solve_batched(gen.ctx, B, U, 1e-8, 200)
    assert code == cm.CHEBMG_OK and max(rel) <= 1e-8
    gen.close()


def test_invalid_meshes_are_rejected(verts):
    L, coords, gid, dirichlet, _ = general_mesh(verts, 3, seed=7)
    opts = cm.chebmg_default_opts(lanczos_steps=10)
    # a reflected element has a negative Jacobian
    bad = coords.copy().reshape(L.E, 4, 4, 4, 3)
    bad[0] = bad[0][:, :, ::-1]
    g2 = gid.copy().reshape(L.E, 4, 4, 4)
    g2[0] = g2[0][:, :, ::-1]
    with pytest.raises(cm.ChebmgError) as e:
        cm.chebmg_setup_sem_mesh(bad.reshape(L.E, 64, 3), g2.reshape(L.E, 64), L.n, dirichlet, (3, 1), opts)
    assert e.value.code == cm.CHEBMG_EMESH
    with pytest.raises(cm.ChebmgError) as e:                   # id out of range
        g3 = gid.copy()
        g3[0, 0] = L.n
        cm.chebmg_setup_sem_mesh(coords, g3, L.n, dirichlet, (3, 1), opts)
    assert e.value.code == cm.CHEBMG_EINVAL
    with pytest.raises(cm.ChebmgError) as e:                   # an unused id
        cm.chebmg_setup_sem_mesh(coords, gid, L.n + 1, np.append(dirichlet, 0), (3, 1), opts)
    assert e.value.code == cm.CHEBMG_EINVAL
    with pytest.raises(cm.ChebmgError) as e:                   # orders[0] != N
        cm.chebmg_setup_sem_mesh(coords, gid, L.n, dirichlet, (2, 1), opts)
    assert e.value.code == cm.CHEBMG_EINVAL
