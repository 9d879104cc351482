"""Pins of the oracle's SEM operator, Jacobi diagonal and p-multigrid transfers.

Each check is fixed by the mathematics of the discretisation (Sec. 1, Eq. 1.3),
not by re-running the oracle's own formulas.
"""
import numpy as np
import pytest

import workloads as W
from oracle.gll import gll_nodes_weights, derivative_matrix
from oracle.sem import SemLevel, SemTransfer


def unmasked_apply(L, u):
    return np.bincount(L.gid.ravel(), L.ax_local(u[L.gid]).ravel(), minlength=L.n)


def nodal(L, f):
    v = np.zeros(L.n)
    v[L.gid] = f(L.coords[..., 0], L.coords[..., 1], L.coords[..., 2])
    return v


@pytest.fixture(scope="module")
def deformed():
    return SemLevel(W.sem_box_vertices(3, 2, 2), 5)


@pytest.fixture(scope="module")
def undeformed():
    return SemLevel(W.sem_box_vertices(2, 3, 2, perturb=0.0, amplitude=0.0), 4)


def test_constant_in_kernel(deformed):
    y = unmasked_apply(deformed, np.ones(deformed.n))
    assert np.abs(y).max() < 1e-13


@pytest.mark.parametrize("a,b,c", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 2, -1), (0.5, -3, 2)])
def test_energy_of_linear_fields_is_volume_times_gradient(deformed, a, b, c):
    # u = a x + b y + c z lies in the isoparametric space; int |grad u|^2 = (a^2+b^2+c^2) |Omega|,
    # integrated exactly by GLL because the trilinear Jacobian has degree <= 2 per direction.
    u = nodal(deformed, lambda x, y, z: a * x + b * y + c * z)
    energy = u @ unmasked_apply(deformed, u)
    assert abs(energy - (a * a + b * b + c * c)) < 1e-12 * (a * a + b * b + c * c)


def test_mixed_energy_vanishes(deformed):
    ux = nodal(deformed, lambda x, y, z: x)
    uy = nodal(deformed, lambda x, y, z: y)
    assert abs(ux @ unmasked_apply(deformed, uy)) < 1e-13


def test_symmetric_positive_definite_and_diagonal(deformed):
    A = deformed.dense()
    live = ~deformed.dirichlet
    assert np.abs(A - A.T).max() < 1e-14 * np.abs(A).max()
    ev = np.linalg.eigvalsh(A[np.ix_(live, live)])
    assert ev.min() > 0
    np.testing.assert_allclose(deformed.diagonal(), np.diag(A), rtol=1e-13, atol=1e-15)
    assert np.all(A[deformed.dirichlet] == 0) and np.all(A[:, deformed.dirichlet] == 0)


def test_x_squared_gives_minus_two_lumped_mass(undeformed):
    # On affine elements GLL integrates grad(phi_i).grad(x^2) exactly, so A x^2 = -2 B at interior nodes.
    L = undeformed
    u = nodal(L, lambda x, y, z: x * x + 2 * y * y - z * z)
    w3 = L.w[:, None, None] * L.w[None, :, None] * L.w[None, None, :]
    B = np.bincount(L.gid.ravel(), (w3[None] * L.jac).ravel(), minlength=L.n)
    y = unmasked_apply(L, u)
    live = ~L.dirichlet
    np.testing.assert_allclose(y[live], -2.0 * (1 + 2 - 1) * B[live], rtol=1e-12)


def test_affine_box_is_kronecker_sum(undeformed):
    # Textbook tensor form: A = Bz x By x Kx + Bz x Ky x Bx + Kz x By x Bx from 1-D GLL stiffness/mass.
    L = undeformed
    x, w = gll_nodes_weights(L.N)
    D = derivative_matrix(x)

    def assemble_1d(ne):
        h = 1.0 / ne
        m = ne * L.N + 1
        K = np.zeros((m, m))
        Bm = np.zeros((m, m))
        for e in range(ne):
            s = slice(e * L.N, e * L.N + L.N + 1)
            K[s, s] += (2.0 / h) * D.T @ np.diag(w) @ D
            Bm[s, s] += (h / 2.0) * np.diag(w)
        return K, Bm

    Kx, Bx = assemble_1d(L.nex)
    Ky, By = assemble_1d(L.ney)
    Kz, Bz = assemble_1d(L.nez)
    A_ref = (np.kron(Bz, np.kron(By, Kx)) + np.kron(Bz, np.kron(Ky, Bx)) + np.kron(Kz, np.kron(By, Bx)))
    live = ~L.dirichlet
    A = L.dense()
    np.testing.assert_allclose(A[np.ix_(live, live)], A_ref[np.ix_(live, live)], atol=1e-12)


def test_transfers_are_transposes_and_interpolate_exactly():
    v = W.sem_box_vertices(3, 3, 3)
    Lf, Lc = SemLevel(v, 4), SemLevel(v, 2)
    T = SemTransfer(Lf, Lc)
    P = np.stack([T.prolong(np.eye(Lc.n)[g]) for g in range(Lc.n)], axis=1)
    R = np.stack([T.restrict(np.eye(Lf.n)[g]) for g in range(Lf.n)], axis=1)
    np.testing.assert_allclose(R, P.T, atol=1e-15)
    # x, y, z are trilinear in the reference coordinates, so they lie in the order-2 space:
    # interpolation must reproduce them wherever the Dirichlet mask does not interfere,
    # i.e. on elements that touch no boundary (the centre element of a 3x3x3 box).
    f = lambda x, y, z: 3 * x - y + 0.5 * z
    uc, uf = nodal(Lc, f), nodal(Lf, f)
    got = T.prolong(uc)
    centre = (Lf.ex == 1) & (Lf.ey == 1) & (Lf.ez == 1)
    g = Lf.gid[centre].ravel()
    np.testing.assert_allclose(got[g], uf[g], atol=1e-13)
    assert np.all(got[Lf.dirichlet] == 0.0)


def test_element_subset_matches_full_operator_at_interior_samples():
    v = W.sem_box_vertices(3, 3, 3)
    full = SemLevel(v, 3)
    u = np.random.default_rng(3).uniform(-1, 1, full.n)
    yfull = full.apply_A(u)
    # node at the centre vertex between elements: touching elements only
    g = (1 * 3 * full.NY + 1 * 3) * full.NX + 1 * 3
    touching = [e for e in range(full.E) if g in full.gid[e]]
    assert len(touching) == 8
    sub = SemLevel(v, 3, elements=touching)
    assert abs(sub.apply_A(u)[g] - yfull[g]) < 1e-13 * max(1, abs(yfull[g]))
