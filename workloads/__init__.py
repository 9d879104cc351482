"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module holds none of the method's arithmetic: it only draws random numbers
and lays out index sets (lattice numbering, boundary flags).  Both the oracle
(`oracle/`) and the GPU library consume exactly these arrays, so parity tests
compare the two implementations on bitwise-identical inputs.

Workloads (Phillips & Fischer, arXiv 2210.03179):

* 2-D finite differences (Sec. 3): an ``m x m`` interior grid on
  ``[0,Lx] x [0,Ly]`` with homogeneous Dirichlet boundaries; the right-hand side
  is iid uniform[-1,1] drawn from ``numpy.random.default_rng(seed)``.
* 3-D spectral elements (Sec. 4-5): a box ``[0,1]^3`` split into
  ``nex x ney x nez`` hexahedra.  The paper's Kershaw and pebble-bed meshes are
  not available, so a perturbed box stands in for them: every interior vertex
  is shifted by iid uniform[-0.1 h, 0.1 h] per coordinate (h the element
  width in that direction), then all vertices are mapped by
  ``x -> x + a sin(pi x) sin(pi y) sin(pi z) (1,1,1)`` with ``a = 0.05``.
  Boundary vertices stay on the cube faces, so the domain is exactly the unit
  cube.  Elements are trilinear in their eight vertices.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "fd_rhs",
    "sem_box_vertices",
    "sem_lattice_shape",
    "sem_boundary_mask",
    "sem_rhs",
    "random_vectors",
]

# Default seeds: RHS seeds follow the workload definitions (FD seed 0, SEM seed 1);
# the mesh perturbation uses its own stream.
FD_RHS_SEED = 0
SEM_RHS_SEED = 1
SEM_MESH_SEED = 7
PERTURB_FRACTION = 0.1
SINE_AMPLITUDE = 0.05


def fd_rhs(m: int, seed: int = FD_RHS_SEED, my: int | None = None) -> np.ndarray:
    """Uniform[-1,1] right-hand side on an ``m x my`` interior FD grid (x fastest)."""
    my = m if my is None else my
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=m * my)


def sem_box_vertices(nex: int, ney: int, nez: int, seed: int = SEM_MESH_SEED,
                     perturb: float = PERTURB_FRACTION,
                     amplitude: float = SINE_AMPLITUDE) -> np.ndarray:
    """Vertex lattice of the perturbed unit box, shape ``(nez+1, ney+1, nex+1, 3)``.

    Index order is ``[vz, vy, vx, coordinate]``; element ``(ex, ey, ez)`` has
    corners ``verts[ez:ez+2, ey:ey+2, ex:ex+2]``.
    """
    hx, hy, hz = 1.0 / nex, 1.0 / ney, 1.0 / nez
    vx = np.arange(nex + 1) * hx
    vy = np.arange(ney + 1) * hy
    vz = np.arange(nez + 1) * hz
    vx[-1] = vy[-1] = vz[-1] = 1.0
    Z, Y, X = np.meshgrid(vz, vy, vx, indexing="ij")
    verts = np.stack([X, Y, Z], axis=-1)
    rng = np.random.default_rng(seed)
    shift = rng.uniform(-1.0, 1.0, size=verts.shape) * (perturb * np.array([hx, hy, hz]))
    interior = np.zeros(verts.shape[:3], dtype=bool)
    interior[1:-1, 1:-1, 1:-1] = True
    verts = verts + shift * interior[..., None]
    bump = amplitude * (np.sin(np.pi * verts[..., 0]) * np.sin(np.pi * verts[..., 1])
                        * np.sin(np.pi * verts[..., 2]))
    bump = bump * interior
    verts = verts + bump[..., None]
    return np.ascontiguousarray(verts)


def sem_lattice_shape(nex: int, ney: int, nez: int, N: int) -> tuple[int, int, int]:
    """Global GLL lattice size ``(NX, NY, NZ)``; global id = ``(gz*NY + gy)*NX + gx``."""
    return nex * N + 1, ney * N + 1, nez * N + 1


def sem_boundary_mask(nex: int, ney: int, nez: int, N: int) -> np.ndarray:
    """Boolean Dirichlet flags of the global lattice nodes (true on the cube boundary)."""
    NX, NY, NZ = sem_lattice_shape(nex, ney, nez, N)
    m = np.zeros((NZ, NY, NX), dtype=bool)
    m[0, :, :] = m[-1, :, :] = True
    m[:, 0, :] = m[:, -1, :] = True
    m[:, :, 0] = m[:, :, -1] = True
    return m.reshape(-1)


def sem_rhs(nex: int, ney: int, nez: int, N: int, seed: int = SEM_RHS_SEED) -> np.ndarray:
    """Uniform[-1,1] RHS over the global lattice in global-id order, zero on the boundary."""
    NX, NY, NZ = sem_lattice_shape(nex, ney, nez, N)
    rng = np.random.default_rng(seed)
    b = rng.uniform(-1.0, 1.0, size=NX * NY * NZ)
    b[sem_boundary_mask(nex, ney, nez, N)] = 0.0
    return b


def random_vectors(n: int, count: int, seed: int) -> np.ndarray:
    """``count`` iid uniform[-1,1] vectors of length ``n`` (rows), one generator."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(count, n))
