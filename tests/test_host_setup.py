"""The library's host setup (csrc/setup_host.cpp) against the oracle, on the CPU.

The setup routines run once per context on the host (Sec. 1: setup is amortised over many
right-hand sides) and everything the kernels read comes from them: GLL points, weights and the
derivative matrix, the element-to-global ids with their Dirichlet and owner bits, the six
geometric factors per point (Sec. 1, Eq. 1.3), the assembled diagonal (the Jacobi scaling of
Sec. 2), the FD Galerkin stencils (Sec. 3) and the optimal 1st-kind lambda_min (Sec. 2.4).  A
small driver (tests/host_setup_dump.cpp) is compiled with the product's source, under the
address and undefined-behaviour sanitizers where the compiler has them, and its output is
compared with the oracle's independent constructions.  The library computes the box's
geometric factors from the analytic trilinear Jacobian and the general-mesh factors by
differentiating GLL coordinates; the oracle differentiates coordinates and inverts numerically.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import workloads as W
from oracle import fd as F
from oracle import theory as TH
from oracle.gll import derivative_matrix, gll_nodes_weights
from oracle.sem import SemLevel

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GID_DIRICHLET, GID_OWNER, GID_MASK = 0x80000000, 0x40000000, 0x3FFFFFFF

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("host_setup")
    exe = str(d / "host_setup_dump")
    src = [os.path.join(ROOT, "tests", "host_setup_dump.cpp"),
           os.path.join(ROOT, "paper_2210_03179_gb300", "csrc", "setup_host.cpp")]
    base = ["g++", "-std=c++17", "-O1", "-g", "-o", exe] + src
    san = ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer"]
    r = subprocess.run(base + san, capture_output=True, text=True)
    if r.returncode != 0:      # no sanitizer runtime: plain build
        r = subprocess.run(base, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1", UBSAN_OPTIONS="halt_on_error=1")

    def run(*args):
        out = subprocess.run([exe] + [str(a) for a in args], capture_output=True, text=True, env=env, timeout=300)
        assert out.returncode == 0, (args, out.stdout[-2000:], out.stderr[-3000:])
        return out.stdout
    return run, d


def _read(path, dtype):
    return np.fromfile(path, dtype=dtype)


@pytest.mark.parametrize("mesh,N", [((3, 2, 4), 1), ((3, 2, 4), 3), ((2, 3, 2), 5), ((2, 2, 3), 7)])
def test_sem_level_matches_the_oracle(driver, tmp_path, mesh, N):
    run, _ = driver
    nex, ney, nez = mesh
    v = W.sem_box_vertices(nex, ney, nez)
    vpath = tmp_path / "verts.bin"
    np.ascontiguousarray(v, dtype=np.float64).tofile(vpath)
    E, n = (int(t) for t in run("sem", nex, ney, nez, N, vpath, tmp_path).split())
    O = SemLevel(v, N)
    NQ = N + 1
    assert (E, n) == (O.E, O.n)
    # GLL data
    x, w = gll_nodes_weights(N)
    np.testing.assert_allclose(_read(tmp_path / "x.bin", np.float64), x, rtol=0, atol=1e-15)
    np.testing.assert_allclose(_read(tmp_path / "w.bin", np.float64), w, rtol=1e-14)
    D = derivative_matrix(x)
    np.testing.assert_allclose(_read(tmp_path / "D.bin", np.float64).reshape(NQ, NQ), D, rtol=0,
                               atol=1e-13 * np.abs(D).max())
    # ids: lattice numbering, Dirichlet bit, exactly one owner copy per global node
    gid = _read(tmp_path / "gid.bin", np.uint32).astype(np.int64)
    ids = gid & GID_MASK
    np.testing.assert_array_equal(ids, O.gid.reshape(-1))
    np.testing.assert_array_equal((gid & GID_DIRICHLET) != 0, O.dirichlet[ids])
    owners = np.bincount(ids[(gid & GID_OWNER) != 0], minlength=n)
    assert np.all(owners == 1)
    np.testing.assert_array_equal(_read(tmp_path / "dirichlet.bin", np.uint8) != 0, O.dirichlet)
    # geometric factors [E][6][NP] and the assembled diagonal, box and general-mesh routes
    Gref = O.G.reshape(E, 6, -1)
    dref = O.diagonal()
    for gname, dname in (("G.bin", "diag.bin"), ("G_mesh.bin", "diag_mesh.bin")):
        G = _read(tmp_path / gname, np.float64).reshape(E, 6, -1)
        assert np.abs(G - Gref).max() <= 1e-12 * np.abs(Gref).max(), gname
        d = _read(tmp_path / dname, np.float64)
        assert np.abs(d - dref).max() <= 1e-12 * np.abs(dref).max(), dname
        assert np.all(d[O.dirichlet] == 0.0)


@pytest.mark.parametrize("mesh,N,Nt", [((3, 2, 4), 7, 3), ((3, 2, 4), 3, 1), ((2, 3, 2), 7, 5), ((2, 2, 3), 5, 1)])
def test_general_mesh_coarse_level_is_the_box_level_relabelled(driver, tmp_path, mesh, N, Nt):
    # the order-Nt level of a general mesh (coordinates interpolated from order N, nodes numbered
    # from the mesh topology) must be the box's order-Nt level under a relabelling of its nodes:
    # one bijection between the two numberings maps every element copy, the Dirichlet flags, the
    # assembled diagonal, and the geometric factors agree point by point
    run, _ = driver
    v = W.sem_box_vertices(*mesh)
    vpath = tmp_path / "verts.bin"
    np.ascontiguousarray(v, dtype=np.float64).tofile(vpath)
    nb, nm = (int(t) for t in run("coarse", *mesh, N, Nt, vpath, tmp_path).split())
    assert nb == nm
    bg = _read(tmp_path / "box_gid.bin", np.uint32).astype(np.int64)
    mg = _read(tmp_path / "mesh_gid.bin", np.uint32).astype(np.int64)
    bi, mi = bg & GID_MASK, mg & GID_MASK
    perm = np.full(nb, -1)
    perm[bi] = mi
    assert np.all(perm >= 0) and len(np.unique(perm)) == nb       # a bijection of the nodes
    np.testing.assert_array_equal(perm[bi], mi)                   # consistent on every copy
    np.testing.assert_array_equal((bg & GID_DIRICHLET) != 0, (mg & GID_DIRICHLET) != 0)
    np.testing.assert_array_equal(_read(tmp_path / "mesh_dirichlet.bin", np.uint8)[mi] != 0,
                                  (bg & GID_DIRICHLET) != 0)
    owners = np.bincount(mi[(mg & GID_OWNER) != 0], minlength=nm)
    assert np.all(owners == 1)
    Gb = _read(tmp_path / "box_G.bin", np.float64)
    Gm = _read(tmp_path / "mesh_G.bin", np.float64)
    assert np.abs(Gb - Gm).max() <= 1e-12 * np.abs(Gb).max()
    db = _read(tmp_path / "box_diag.bin", np.float64)
    dm = _read(tmp_path / "mesh_diag.bin", np.float64)
    assert np.abs(dm[perm] - db).max() <= 1e-12 * np.abs(db).max()
    # and the box level itself is the oracle's order-Nt level
    O = SemLevel(v, Nt)
    np.testing.assert_array_equal(bi, O.gid.reshape(-1))
    assert np.abs(Gb.reshape(O.G.shape[0], 6, -1) - O.G.reshape(O.G.shape[0], 6, -1)).max() <= 1e-12 * np.abs(O.G).max()


def _rotations():
    """The 24 orientation-preserving relabellings of an element's (k, j, i) axes: an axis
    permutation with an even total count of (odd permutation, flipped axes)."""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        odd = sum(1 for a in range(3) for b in range(a + 1, 3) if perm[a] > perm[b]) % 2
        for flips in itertools.product((0, 1), repeat=3):
            if (odd + sum(flips)) % 2 == 0:
                out.append((perm, flips))
    return out


def _rotate(A, rot):
    perm, flips = rot
    B = np.transpose(A, perm + tuple(range(3, A.ndim)))
    for ax in range(3):
        if flips[ax]:
            B = np.flip(B, axis=ax)
    return np.ascontiguousarray(B)


@pytest.mark.parametrize("mesh,N,Nt", [((3, 2, 4), 7, 3), ((2, 3, 2), 5, 1), ((2, 2, 3), 3, 3)])
def test_shuffled_rotated_mesh_gives_the_box_levels(driver, tmp_path, mesh, N, Nt):
    # the box handed over as a general mesh with its global ids permuted at random and every
    # element's local axes turned by one of the 24 rotations: its order-Nt level must be the
    # oracle's order-Nt box level under one node relabelling (ids consistent on every element
    # copy, Dirichlet set, assembled diagonal); at Nt = N the caller's ids are kept as given
    run, _ = driver
    v = W.sem_box_vertices(*mesh)
    O = SemLevel(v, N)
    rng = np.random.default_rng(17)
    pi = rng.permutation(O.n)
    rots = _rotations()
    pick = rng.integers(0, len(rots), O.E)
    coords = np.stack([_rotate(O.coords[e], rots[pick[e]]) for e in range(O.E)])
    gid = np.stack([_rotate(pi[O.gid[e]], rots[pick[e]]) for e in range(O.E)])
    dirichlet = np.zeros(O.n, dtype=np.uint8)
    dirichlet[pi] = O.dirichlet
    d_in = tmp_path / "in"
    d_in.mkdir()
    coords.astype(np.float64).tofile(d_in / "coords.bin")
    gid.astype(np.int64).tofile(d_in / "gid.bin")
    dirichlet.tofile(d_in / "dirichlet.bin")
    nt = int(run("meshfile", O.E, N, O.n, Nt, d_in, tmp_path).split()[0])
    T = SemLevel(v, Nt)
    assert nt == T.n
    mg = _read(tmp_path / "gid_t.bin", np.uint32).astype(np.int64).reshape(T.gid.shape)
    mi = mg & GID_MASK
    bi = np.stack([_rotate(T.gid[e], rots[pick[e]]) for e in range(T.E)])
    perm = np.full(T.n, -1)
    perm[bi] = mi
    assert np.all(perm >= 0) and len(np.unique(perm)) == T.n
    np.testing.assert_array_equal(perm[bi], mi)
    if Nt == N:
        np.testing.assert_array_equal(mi, gid)
    dm = _read(tmp_path / "dirichlet_t.bin", np.uint8) != 0
    np.testing.assert_array_equal(dm[perm], T.dirichlet)
    np.testing.assert_array_equal((mg & GID_DIRICHLET) != 0, T.dirichlet[bi])
    owners = np.bincount(mi[(mg & GID_OWNER) != 0], minlength=T.n)
    assert np.all(owners == 1)
    diag = _read(tmp_path / "diag_t.bin", np.float64)
    dref = T.diagonal()
    assert np.abs(diag[perm] - dref).max() <= 1e-12 * np.abs(dref).max()


@pytest.mark.parametrize("mesh,N", [((3, 2, 4), 1), ((2, 2, 2), 2)])
def test_assembled_ell_matches_the_dense_oracle(driver, tmp_path, mesh, N):
    # the coarse CG's matrix: rows and columns of Dirichlet nodes removed (empty rows padded
    # with their own column and zero), every other entry the oracle's assembled A
    run, _ = driver
    v = W.sem_box_vertices(*mesh)
    vpath = tmp_path / "verts.bin"
    np.ascontiguousarray(v, dtype=np.float64).tofile(vpath)
    nslot, n = (int(t) for t in run("ell", *mesh, N, vpath, tmp_path).split())
    O = SemLevel(v, N)
    assert n == O.n
    col = _read(tmp_path / "col.bin", np.int32).reshape(nslot, n)
    val = _read(tmp_path / "val.bin", np.float64).reshape(nslot, n)
    A = np.zeros((n, n))
    for s_ in range(nslot):
        np.add.at(A, (np.arange(n), col[s_]), val[s_])
    live = ~O.dirichlet
    Aref = O.dense()
    Aref[~live, :] = 0.0
    Aref[:, ~live] = 0.0
    assert np.abs(A - Aref).max() <= 1e-12 * np.abs(Aref).max()
    assert np.all(col[:, ~live] == np.arange(n)[~live]) and np.all(val[:, ~live] == 0.0)
    # the rows hold exactly the oracle's nonzeros, one slot per column; the width is at most the
    # (2N+1)^3 nodes of the elements around a vertex (27 lattice neighbours at N = 1)
    nnz = (val != 0).sum(axis=0)
    np.testing.assert_array_equal(nnz, (Aref != 0).sum(axis=1))
    for g in np.flatnonzero(live)[:50]:
        used = col[:, g][val[:, g] != 0]
        assert len(set(used.tolist())) == len(used)
    assert nnz.max() <= nslot <= (2 * N + 1) ** 3 and np.all((col >= 0) & (col < n))


def _interior_stencil(A, mx, i, j):
    A = A.tocsr()
    row = j * mx + i
    st = np.zeros(9)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            st[(a + 1) * 3 + (b + 1)] = A[row, (j + a) * mx + (i + b)]
    return st


@pytest.mark.parametrize("Lx,c", [(1.0, 2), (8.0, 2), (1.0, 8)])
def test_fd_stencils_match_the_oracle(driver, tmp_path, Lx, c):
    run, _ = driver
    m = 63 if c == 2 else 127
    levels, _ = F.fd_levels(m, Lx=Lx, Ly=1.0, c=c, coarsest=7 if c == 2 else 15)
    hx, hy = Lx / (m + 1), 1.0 / (m + 1)
    run("fd", repr(hx), repr(hy), c, tmp_path)
    both = _read(tmp_path / "stencils.bin", np.float64)
    fine, coarse = both[:9], both[9:]
    L0, L1 = levels[0], levels[1]
    ref0 = _interior_stencil(L0.A, L0.mx, L0.mx // 2, L0.my // 2)
    ref1 = _interior_stencil(L1.A, L1.mx, L1.mx // 2, L1.my // 2)
    np.testing.assert_allclose(fine, ref0, rtol=1e-14, atol=1e-14 * np.abs(ref0).max())
    np.testing.assert_allclose(coarse, ref1, rtol=1e-12, atol=1e-12 * np.abs(ref1).max())


@pytest.mark.parametrize("m,Lx,c,coarsest", [(63, 1.0, 2, 7), (63, 8.0, 2, 7), (127, 1.0, 8, 15)])
def test_fd_coarse_dense_inverse(driver, tmp_path, m, Lx, c, coarsest):
    # the coarsest FD solve: the inverse of the repeated-Galerkin operator (Cholesky on the host)
    run, _ = driver
    mc = int(run("fdinv", m, repr(Lx), c, coarsest, tmp_path))
    levels, _ = F.fd_levels(m, Lx=Lx, Ly=1.0, c=c, coarsest=coarsest)
    Ac = levels[-1].A.toarray()
    assert Ac.shape == (mc * mc, mc * mc)
    inv = _read(tmp_path / "inv.bin", np.float64).reshape(mc * mc, mc * mc)
    np.testing.assert_allclose(inv, np.linalg.inv(Ac), rtol=1e-10, atol=1e-12 * np.abs(inv).max())
    assert np.abs(inv @ Ac - np.eye(mc * mc)).max() < 1e-11


@pytest.mark.parametrize("Nf,Nc", [(7, 3), (3, 1), (7, 5), (5, 3), (9, 5)])
def test_pmg_interpolation_matches_the_oracle(driver, tmp_path, Nf, Nc):
    from oracle.gll import interpolation_matrix
    run, _ = driver
    run("interp", Nc, Nf, tmp_path)
    J = _read(tmp_path / "J.bin", np.float64).reshape(Nf + 1, Nc + 1)
    xc, _ = gll_nodes_weights(Nc)
    xf, _ = gll_nodes_weights(Nf)
    np.testing.assert_allclose(J, interpolation_matrix(xc, xf), rtol=0, atol=1e-14)


@pytest.mark.parametrize("k", [1, 2, 3, 6, 10])
def test_optimal_lambda_min_matches_the_oracle_maximiser(driver, k):
    run, _ = driver
    ratio = float(run("lmin", k))
    res = minimize_scalar(lambda lm: -TH.gamma_inv("1st", k, lmin_ratio=lm), bounds=(1e-3, 0.6),
                          method="bounded", options={"xatol": 1e-7})
    assert abs(ratio - res.x) <= 1e-5 * res.x
