"""Structured hexahedral mesh of the oracle (Sections 3.1 and 7.1).

Displacement mesh: nx*ny*nz cubes of edge 1, element id e = ex + nx*(ey +
ny*ez).  Lagrange degree k puts nodes on a (k nx+1, k ny+1, k nz+1) lattice
(node id i + Lx*(j + Ly*l)); DOF = 3*node + component.  Each displacement
element holds n^3 density cells (Section 3.1), density cell id
cx + Dx*(cy + Dy*cz) with Dx = n*nx, and subcell index a + n*(b + n*c) inside
its element, where (cx, cy, cz) = (n ex + a, n ey + b, n ez + c).
"""
from __future__ import annotations

import numpy as np


def element_dofs(nx: int, ny: int, nz: int, k: int) -> np.ndarray:
    """(E, 3 (k+1)^3) global DOF indices of each element, in element DOF
    order 3*a + c with local node a = ix + (k+1)*(iy + (k+1)*iz)."""
    Lx, Ly = k * nx + 1, k * ny + 1
    nn = (k + 1) ** 3
    E = nx * ny * nz
    out = np.zeros((E, 3 * nn), dtype=np.int64)
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ex, ey, ez = ex.reshape(-1), ey.reshape(-1), ez.reshape(-1)
    for iz in range(k + 1):
        for iy in range(k + 1):
            for ix in range(k + 1):
                a = ix + (k + 1) * (iy + (k + 1) * iz)
                node = (k * ex + ix) + Lx * ((k * ey + iy) + Ly * (k * ez + iz))
                for c in range(3):
                    out[:, 3 * a + c] = 3 * node + c
    return out


def subcell_density_index(nx: int, ny: int, nz: int, n: int) -> np.ndarray:
    """(E, n^3): density-cell id of subcell i of element e."""
    Dx, Dy = n * nx, n * ny
    E = nx * ny * nz
    out = np.zeros((E, n ** 3), dtype=np.int64)
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ex, ey, ez = ex.reshape(-1), ey.reshape(-1), ez.reshape(-1)
    for c in range(n):
        for b in range(n):
            for a in range(n):
                i = a + n * (b + n * c)
                out[:, i] = (n * ex + a) + Dx * ((n * ey + b) + Dy * (n * ez + c))
    return out


def node_coords(nx: int, ny: int, nz: int, k: int) -> np.ndarray:
    """(nnodes, 3) coordinates of the lattice nodes (element edge 1)."""
    Lx, Ly, Lz = k * nx + 1, k * ny + 1, k * nz + 1
    l, j, i = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return np.stack([i.reshape(-1) / k, j.reshape(-1) / k, l.reshape(-1) / k], axis=1)
