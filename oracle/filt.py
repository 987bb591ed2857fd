"""Density filter / design-variable projection of the oracle.

Section 2.2, Eq. filter_weights: for density cell i and design cell j whose
centres are dist(i, j) apart,
    w_ij = exp(-dist^2 / (2 (r/3)^2)) / (2 pi r/3)   if dist <= r, else 0,
and rho_i = sum_j (w_ij / w_i) x_j with w_i = sum_j w_ij.
Section 3.2, Eq. projdsgn: the same weights project design variables onto
density cells; with the design grid equal to the density grid
(d_mr = n_mr) the projection is the filter itself.

Readings taken here:
  * distances are measured in displacement-element units (element edge 1),
    so with n density cells per element edge a cell offset (di, dj, dk) is at
    distance sqrt(di^2 + dj^2 + dk^2) / n;
  * the neighbourhood is inclusive: offsets with di^2+dj^2+dk^2 <=
    (r n)^2 (1 + 1e-12) are neighbours -- ties occur (r = 1.5, n = 2) and the
    test is taken on the integer sum of squares;
  * near the boundary the neighbourhood is truncated to cells inside the
    domain and w_i sums only those;
  * the constant 1 / (2 pi r/3) cancels in w_ij / w_i and is dropped;
  * r = 0 means no filter: rho = x (only with d_mr = n_mr).
With a coarser design grid (d_mr < n_mr design cells per element edge)
the projection uses the same weights between the centres of density cells
((c + 1/2) / n_mr in element units) and design cells ((j + 1/2) / d_mr),
neighbours being those at dist <= r (1 + 1e-12 on the squared distance).
"""
from __future__ import annotations

import math
import numpy as np
import scipy.sparse as sp


def filter_offsets(n: int, rmin: float):
    """Integer offsets inside the ball and their unnormalised weights."""
    rc2 = (rmin * n) ** 2
    R = int(math.floor(rmin * n + 1e-9))
    offs, wts = [], []
    sigma = rmin / 3.0
    for dk in range(-R, R + 1):
        for dj in range(-R, R + 1):
            for di in range(-R, R + 1):
                q = di * di + dj * dj + dk * dk
                if q <= rc2 * (1.0 + 1e-12):
                    dist2 = q / float(n * n)
                    offs.append((di, dj, dk))
                    wts.append(math.exp(-dist2 / (2.0 * sigma * sigma)))
    return np.array(offs, dtype=np.int64).reshape(-1, 3), np.array(wts)


def filter_matrix(shape, n: int, rmin: float) -> sp.csr_matrix:
    """Explicit sparse H (n_cells x n_cells), rho = H x, for a density grid
    of shape (Dz, Dy, Dx) flattened x fastest."""
    Dz, Dy, Dx = shape
    N = Dx * Dy * Dz
    if rmin <= 0.0:
        return sp.identity(N, format="csr")
    offs, wts = filter_offsets(n, rmin)
    cz, cy, cx = np.meshgrid(np.arange(Dz), np.arange(Dy), np.arange(Dx), indexing="ij")
    cx, cy, cz = cx.reshape(-1), cy.reshape(-1), cz.reshape(-1)
    rows, cols, vals = [], [], []
    for (di, dj, dk), w in zip(offs, wts):
        jx, jy, jz = cx + di, cy + dj, cz + dk
        ok = (jx >= 0) & (jx < Dx) & (jy >= 0) & (jy < Dy) & (jz >= 0) & (jz < Dz)
        i = np.nonzero(ok)[0]
        rows.append(i)
        cols.append(jx[ok] + Dx * (jy[ok] + Dy * jz[ok]))
        vals.append(np.full(i.size, w))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    W = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
    wsum = np.asarray(W.sum(axis=1)).reshape(-1)
    return sp.diags(1.0 / wsum) @ W


def projection_matrix(nx: int, ny: int, nz: int, n: int, d: int, rmin: float) -> sp.csr_matrix:
    """Explicit sparse P (n_density x n_design), rho = P x, Eq. projdsgn,
    for a mesh of nx x ny x nz elements with n density and d design cells
    per element edge (both grids flattened x fastest)."""
    if d == n:
        return filter_matrix((n * nz, n * ny, n * nx), n, rmin)
    if not rmin > 0.0:
        raise ValueError("a coarser design grid needs a projection radius > 0")
    D = (n * nx, n * ny, n * nz)
    G = (d * nx, d * ny, d * nz)
    sig = rmin / 3.0
    r2 = rmin * rmin * (1.0 + 1e-12)
    R = int(math.ceil(rmin * d)) + 1
    cz, cy, cx = np.meshgrid(np.arange(D[2]), np.arange(D[1]), np.arange(D[0]), indexing="ij")
    cx, cy, cz = cx.reshape(-1), cy.reshape(-1), cz.reshape(-1)
    pos = [(cx + 0.5) / n, (cy + 0.5) / n, (cz + 0.5) / n]
    base = [np.floor(p * d - 0.5).astype(np.int64) for p in pos]
    rows, cols, vals = [], [], []
    for dk in range(-R, R + 2):
        for dj in range(-R, R + 2):
            for di in range(-R, R + 2):
                jx, jy, jz = base[0] + di, base[1] + dj, base[2] + dk
                ok = (jx >= 0) & (jx < G[0]) & (jy >= 0) & (jy < G[1]) & (jz >= 0) & (jz < G[2])
                dist2 = (((jx + 0.5) / d - pos[0]) ** 2 + ((jy + 0.5) / d - pos[1]) ** 2
                         + ((jz + 0.5) / d - pos[2]) ** 2)
                ok &= dist2 <= r2
                i = np.nonzero(ok)[0]
                rows.append(i)
                cols.append(jx[ok] + G[0] * (jy[ok] + G[1] * jz[ok]))
                vals.append(np.exp(-dist2[ok] / (2.0 * sig * sig)))
    rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    W = sp.csr_matrix((vals, (rows, cols)), shape=(cx.size, G[0] * G[1] * G[2]))
    wsum = np.asarray(W.sum(axis=1)).reshape(-1)
    return (sp.diags(1.0 / wsum) @ W).tocsr()
