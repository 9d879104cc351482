"""The seeded input recipe: sizes, determinism, the perturbed box's geometry and the boundary.

The benchmark mesh is the unit box split into 32^3 trilinear elements at N = 7 (n = 225^3 =
11,390,625 global nodes, 223^3 of them interior); interior vertices are shifted by at most
0.1 h per coordinate and then moved by 0.05 sin(pi x) sin(pi y) sin(pi z) along (1,1,1);
boundary vertices stay on the cube's faces.
"""
import numpy as np
import pytest

import workloads as W


def test_benchmark_sizes():
    NX, NY, NZ = W.sem_lattice_shape(32, 32, 32, 7)
    assert (NX, NY, NZ) == (225, 225, 225) and NX * NY * NZ == 11_390_625
    mask = W.sem_boundary_mask(32, 32, 32, 7)
    assert mask.size == 11_390_625 and int((~mask).sum()) == 223 ** 3 == 11_089_567
    assert W.sem_lattice_shape(16, 16, 16, 7) == (113, 113, 113) and 113 ** 3 == 1_442_897
    assert W.sem_lattice_shape(32, 32, 32, 1) == (33, 33, 33) and 33 ** 3 == 35_937
    assert W.sem_lattice_shape(8, 8, 8, 7) == (57, 57, 57) and 57 ** 3 == 185_193


def test_generators_are_deterministic_and_seeded():
    np.testing.assert_array_equal(W.sem_box_vertices(4, 3, 5), W.sem_box_vertices(4, 3, 5))
    assert not np.array_equal(W.sem_box_vertices(4, 3, 5), W.sem_box_vertices(4, 3, 5, seed=8))
    np.testing.assert_array_equal(W.sem_rhs(3, 3, 3, 5), W.sem_rhs(3, 3, 3, 5))
    assert not np.array_equal(W.sem_rhs(3, 3, 3, 5, seed=1), W.sem_rhs(3, 3, 3, 5, seed=2))
    np.testing.assert_array_equal(W.fd_rhs(63), W.fd_rhs(63, seed=0))
    assert W.fd_rhs(63).shape == (3969,) and W.fd_rhs(7, my=5).shape == (35,)
    R = W.random_vectors(100, 3, seed=4)
    assert R.shape == (3, 100) and np.all(np.abs(R) <= 1.0)


@pytest.mark.parametrize("mesh", [(4, 3, 5), (8, 8, 8)])
def test_box_geometry(mesh):
    nex, ney, nez = mesh
    v = W.sem_box_vertices(nex, ney, nez)
    assert v.shape == (nez + 1, ney + 1, nex + 1, 3)
    h = np.array([1.0 / nex, 1.0 / ney, 1.0 / nez])
    Z, Y, X = np.meshgrid(np.arange(nez + 1), np.arange(ney + 1), np.arange(nex + 1), indexing="ij")
    grid = np.stack([X, Y, Z], axis=-1) * h
    interior = np.zeros(v.shape[:3], dtype=bool)
    interior[1:-1, 1:-1, 1:-1] = True
    # boundary vertices are the unperturbed grid, so every face is a plane of the cube
    np.testing.assert_allclose(v[~interior], grid[~interior], atol=1e-15)
    for axis, sl in ((2, np.s_[0]), (2, np.s_[-1]), (1, np.s_[:, 0]), (1, np.s_[:, -1]),
                     (0, np.s_[:, :, 0]), (0, np.s_[:, :, -1])):
        assert np.all(np.isin(v[sl][..., axis], (0.0, 1.0)))
    # interior: a shift of at most 0.1 h per coordinate, then the same bump on all three
    d = v[interior] - grid[interior]
    bump = d - d.mean(axis=1, keepdims=True)     # differences between coordinates come from the shift
    assert np.all(np.abs(bump) <= 0.2 * h.max() + 1e-15)
    assert np.all(np.abs(d) <= 0.1 * h + 0.05 + 1e-15)
    assert np.all((v > 0.0) & (v < 1.0) | ~interior[..., None])
    # every element is well shaped: the corner Jacobians of the trilinear map are positive
    for ez in range(nez):
        for ey in range(ney):
            for ex in range(nex):
                c = v[ez:ez + 2, ey:ey + 2, ex:ex + 2]
                for k in range(2):
                    for j in range(2):
                        for i in range(2):
                            a = c[k, j, 1 - i] - c[k, j, i]
                            b = c[k, 1 - j, i] - c[k, j, i]
                            e = c[1 - k, j, i] - c[k, j, i]
                            sgn = (1 - 2 * i) * (1 - 2 * j) * (1 - 2 * k)
                            assert sgn * np.dot(a, np.cross(b, e)) > 0.0


def test_rhs_is_uniform_and_zero_on_the_boundary():
    b = W.sem_rhs(6, 5, 4, 7)
    mask = W.sem_boundary_mask(6, 5, 4, 7)
    assert b.shape == mask.shape
    assert np.all(b[mask] == 0.0)
    inner = b[~mask]
    assert np.all(np.abs(inner) <= 1.0) and np.all(inner != 0.0)
    # uniform[-1,1]: mean 0, variance 1/3 (n ~ 28,000 interior values)
    assert abs(inner.mean()) < 0.02 and abs(inner.var() - 1.0 / 3.0) < 0.01
