"""Mixed trilinear / triquadratic meshes on one degree-2 lattice (oracle).

Section 7.4 raises the element degree to reduce the artefacts of the
multiresolution scheme; a mesh in which only some elements are quadratic
needs a conforming coupling, which the paper does not spell out.  Reading
taken here: every element carries the triquadratic element matrix of
Eq. matrixK_mr; a lattice node that is not an element vertex is a free
unknown only if every element containing it is quadratic, otherwise its
value is slaved to the linear interpolation of the vertices of the edge,
face or cell it lies on.  With u = T u_r (T: identity on free nodes,
interpolation rows on slaved nodes) the system is T^T K T u_r = T^T f on the
unknowns that are neither supported nor slaved.  A trilinear element then
carries exactly the trilinear element energy (its displacement is trilinear
and the quadratic integration rule is exact for it), and the coupling is
conforming.  Compliance f^T u and the subcell energies use the expanded u.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fe import Model


def slaved_nodes(prob) -> np.ndarray:
    """(nnodes,) bool: non-vertex lattice nodes touching a trilinear element."""
    Lx, Ly, Lz = prob.lattice
    slv = np.zeros((Lz, Ly, Lx), dtype=bool)
    q1 = prob.elem_q1.reshape(prob.nz, prob.ny, prob.nx).astype(bool)
    for ez, ey, ex in zip(*np.nonzero(q1)):
        slv[2 * ez: 2 * ez + 3, 2 * ey: 2 * ey + 3, 2 * ex: 2 * ex + 3] = True
    l, j, i = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    vertex = (i % 2 == 0) & (j % 2 == 0) & (l % 2 == 0)
    return (slv & ~vertex).reshape(-1)


def interpolation(prob) -> sp.csr_matrix:
    """T (ndof x ndof): u = T u_r.  Row of a slaved node: weight 2^-q on each
    of the 2^q vertices around it (q = number of odd lattice coordinates);
    every other row is the identity; slaved columns are empty."""
    Lx, Ly, Lz = prob.lattice
    slv = slaved_nodes(prob)
    rows, cols, vals = [], [], []
    for node in range(Lx * Ly * Lz):
        i, j, l = node % Lx, (node // Lx) % Ly, node // (Lx * Ly)
        if not slv[node]:
            rows.append(node); cols.append(node); vals.append(1.0)
            continue
        opts = [[c] if c % 2 == 0 else [c - 1, c + 1] for c in (i, j, l)]
        par = [(a, b, c) for c in opts[2] for b in opts[1] for a in opts[0]]
        for a, b, c in par:
            rows.append(node); cols.append(a + Lx * (b + Ly * c)); vals.append(1.0 / len(par))
    Tn = sp.csr_matrix((vals, (rows, cols)), shape=(Lx * Ly * Lz,) * 2)
    return sp.kron(Tn, sp.identity(3), format="csr")


class MixedModel(Model):
    """Model of a mixed-degree problem: same interface as Model."""

    def __init__(self, prob):
        super().__init__(prob)
        self.T = interpolation(prob)
        slv = np.repeat(slaved_nodes(prob), 3)
        self.slaved = slv
        self.free = np.nonzero((prob.mask == 0) & ~slv)[0]

    def solve(self, w_e, f, method="auto", tol=1e-13, K=None):
        if K is None:
            K = self.assemble(w_e)
        Kr = (self.T.T @ K @ self.T).tocsr()
        ur = super().solve(w_e, self.T.T @ f, method=method, tol=tol, K=Kr)
        return self.T @ ur

    def run(self, x=None, method="auto", rtol=1e-13, levels=None):
        if method == "mg":
            raise ValueError("the mixed oracle solves directly")
        return super().run(x, method=method, rtol=rtol, levels=levels)
