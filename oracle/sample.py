"""Sampled outputs of the path for meshes too large to assemble (oracle).

Every quantity here is one row (or one cell) of what oracle/fe.py computes
for the whole mesh, evaluated from its definition on the few elements that
row touches:
  * rho at a cell: Eq. projdsgn / the filter (one row of H) -- needs x only;
  * (K u) at a node: Eq. matrixK_mr over the elements containing the node,
    K^(e) = sum_i w_{e,i} K^(e_i), supports as identity rows and zero
    columns (mixed meshes: T_e^T K^(e) T_e with the element-local coupling
    of oracle/mixed.py, slaved rows identity);
  * dc/drho at a cell: -p rho^(p-1) (E0 - Emin) u_e^T K^(e_i) u_e (Sec. 3.4);
  * dc/dx at a design cell: one row of H^T applied to dc/drho (Sec. 3.4).
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from . import fem, filt
from .fe import rigid_projector, simp_weights


class Sampler:
    def __init__(self, prob):
        self.p = prob
        self.k, self.n = prob.degree, prob.n_mr
        self.K = fem.subcell_stiffness(self.k, self.n, prob.nu, family=getattr(prob, "family", "lagrange"))
        self.Dx, self.Dy, self.Dz = self.n * prob.nx, self.n * prob.ny, self.n * prob.nz
        self.offs, self.wts = filt.filter_offsets(self.n, prob.rmin) if prob.rmin > 0 else ([(0, 0, 0)], [1.0])
        self.slv = None
        if getattr(prob, "elem_q1", None) is not None:
            from .mixed import slaved_nodes
            self.slv = slaved_nodes(prob)

    # ---- density side --------------------------------------------------
    def _in(self, cx, cy, cz):
        return 0 <= cx < self.Dx and 0 <= cy < self.Dy and 0 <= cz < self.Dz

    def _cell(self, cx, cy, cz):
        return cx + self.Dx * (cy + self.Dy * cz)

    def rho(self, x, cell):
        """rho_i = sum_j w_ij x_j / sum_j w_ij over the cells j of the ball."""
        cx, cy, cz = cell % self.Dx, (cell // self.Dx) % self.Dy, cell // (self.Dx * self.Dy)
        num = den = 0.0
        for (di, dj, dk), w in zip(self.offs, self.wts):
            if self._in(cx + di, cy + dj, cz + dk):
                num += w * x[self._cell(cx + di, cy + dj, cz + dk)]
                den += w
        return num / den

    # ---- elements --------------------------------------------------------
    def _elem_nodes(self, ex, ey, ez):
        k = self.k
        Lx, Ly, _ = self.p.lattice
        return [(k * ex + ix) + Lx * ((k * ey + iy) + Ly * (k * ez + iz))
                for iz in range(k + 1) for iy in range(k + 1) for ix in range(k + 1)]

    def _elem_cells(self, ex, ey, ez):
        n = self.n
        return [self._cell(n * ex + a, n * ey + b, n * ez + c)
                for c in range(n) for b in range(n) for a in range(n)]

    def _T_e(self, nodes):
        """Element-local u_e = T_e u_e: slaved local nodes interpolated from
        the element's own vertices (identity without a mixed mesh)."""
        d = 3 * len(nodes)
        T = np.identity(d)
        if self.slv is None:
            return T
        for a, nd in enumerate(nodes):
            if not self.slv[nd]:
                continue
            ax, ay, az = a % 3, (a // 3) % 3, a // 9
            opts = [[c] if c != 1 else [0, 2] for c in (ax, ay, az)]
            par = [x + 3 * (y + 3 * z) for z in opts[2] for y in opts[1] for x in opts[0]]
            for c in range(3):
                T[3 * a + c, 3 * a + c] = 0.0
                for q in par:
                    T[3 * a + c, 3 * q + c] = 1.0 / len(par)
        return T

    def elem_matrix(self, x, ex, ey, ez, rho_cache):
        cells = self._elem_cells(ex, ey, ez)
        rho = np.array([rho_cache.setdefault(c, self.rho(x, c)) for c in cells])
        w = simp_weights(rho, self.p.E0, self.p.Emin, self.p.penal)
        return np.tensordot(w, self.K, axes=1), rho

    def elements_of(self, node):
        k = self.k
        Lx, Ly, _ = self.p.lattice
        i, j, l = node % Lx, (node // Lx) % Ly, node // (Lx * Ly)
        ext = (self.p.nx, self.p.ny, self.p.nz)
        rng = []
        for c, e in zip((i, j, l), ext):
            lo, hi = (c - 1) // k if c % k == 0 else c // k, c // k
            rng.append([q for q in range(max(lo, 0), min(hi, e - 1) + 1)])
        return [(ex, ey, ez) for ez in rng[2] for ey in rng[1] for ex in rng[0]]

    def apply_rows(self, x, u, nodes):
        """(len(nodes), 3): rows of the solver's operator at the given nodes."""
        held = self.p.mask.astype(bool).copy()
        if self.slv is not None:
            held |= np.repeat(self.slv, 3)
        uf = np.where(held, 0.0, u)
        cache = {}
        out = np.zeros((len(nodes), 3))
        for q, nd in enumerate(nodes):
            for (ex, ey, ez) in self.elements_of(nd):
                Ke, _ = self.elem_matrix(x, ex, ey, ez, cache)
                en = self._elem_nodes(ex, ey, ez)
                T = self._T_e(en)
                Kr = T.T @ Ke @ T
                dofs = np.array([3 * m + c for m in en for c in range(3)])
                a = en.index(nd)
                out[q] += Kr[3 * a: 3 * a + 3] @ uf[dofs]
            for c in range(3):
                if held[3 * nd + c]:
                    out[q, c] = u[3 * nd + c]
        return out

    def apply_rows_scale(self, x, u, nodes):
        """(len(nodes), 3): sum_j |K_ij u_j| of the same rows, the scale of
        their rounding (K u is much smaller than its terms where u is a
        converged displacement: the rows nearly cancel to the load)."""
        held = self.p.mask.astype(bool).copy()
        if self.slv is not None:
            held |= np.repeat(self.slv, 3)
        uf = np.abs(np.where(held, 0.0, u))
        cache = {}
        out = np.zeros((len(nodes), 3))
        for q, nd in enumerate(nodes):
            for (ex, ey, ez) in self.elements_of(nd):
                Ke, _ = self.elem_matrix(x, ex, ey, ez, cache)
                en = self._elem_nodes(ex, ey, ez)
                T = self._T_e(en)
                Kr = np.abs(T.T @ Ke @ T)
                dofs = np.array([3 * m + c for m in en for c in range(3)])
                a = en.index(nd)
                out[q] += Kr[3 * a: 3 * a + 3] @ uf[dofs]
            for c in range(3):
                if held[3 * nd + c]:
                    out[q, c] = abs(u[3 * nd + c])
        return out

    def apply_rows_subcell_scale(self, x, u, nodes, deflate=False, elem_max=False):
        """(len(nodes), 3): sum over the elements e at the node and their
        subcells i of w_{e,i} sum_j |K^(e_i)_rj| |u_j| -- the rounding scale
        of the stacked form of Eq. matrixK_mr (one rounded product per
        subcell); supports |u|.  Mixed meshes: a triquadratic element rounds
        its expanded vector T_e u_e and its result is folded by T_e^T (>= 0
        entrywise), so it adds T_e^T |K^(e_i)| |T_e u_e|; a trilinear element
        rounds its vertex vector against the trilinear subcell matrices
        (T^T K^(e_i) T restricted to the vertices); slaved rows are identity
        rows.  deflate: each rounded vector minus its least-squares rigid
        motion (rigid_projector); elem_max: its entries replaced by their
        largest magnitude."""
        if self.slv is not None:
            return self._mixed_subcell_scale(x, u, nodes, deflate, elem_max)
        held = self.p.mask.astype(bool)
        uf = np.where(held, 0.0, u)
        P = rigid_projector(self.k) if deflate else None
        cache = {}
        out = np.zeros((len(nodes), 3))
        for q, nd in enumerate(nodes):
            for (ex, ey, ez) in self.elements_of(nd):
                cells = self._elem_cells(ex, ey, ez)
                rho = np.array([cache.setdefault(c, self.rho(x, c)) for c in cells])
                w = simp_weights(rho, self.p.E0, self.p.Emin, self.p.penal)
                en = self._elem_nodes(ex, ey, ez)
                dofs = np.array([3 * m + c for m in en for c in range(3)])
                ue = np.abs(uf[dofs] if P is None else P @ uf[dofs])
                if elem_max:
                    ue = np.full_like(ue, ue.max())
                a = en.index(nd)
                for i in range(len(cells)):
                    out[q] += w[i] * (np.abs(self.K[i][3 * a: 3 * a + 3]) @ ue)
            for c in range(3):
                if held[3 * nd + c]:
                    out[q, c] = abs(u[3 * nd + c])
        return out

    def _mixed_subcell_scale(self, x, u, nodes, deflate, elem_max):
        held = self.p.mask.astype(bool) | np.repeat(self.slv, 3)
        uf = np.where(held, 0.0, u)
        P2 = rigid_projector(2) if deflate else None
        P1 = rigid_projector(1) if deflate else None
        if not hasattr(self, "K1"):
            self.K1 = fem.subcell_stiffness(1, self.n, self.p.nu)
        vloc = [2 * (v & 1) + 3 * (2 * ((v >> 1) & 1)) + 9 * (2 * (v >> 2)) for v in range(8)]
        cache = {}
        out = np.zeros((len(nodes), 3))
        for q, nd in enumerate(nodes):
            for (ex, ey, ez) in self.elements_of(nd):
                cells = self._elem_cells(ex, ey, ez)
                rho = np.array([cache.setdefault(c, self.rho(x, c)) for c in cells])
                w = simp_weights(rho, self.p.E0, self.p.Emin, self.p.penal)
                en = self._elem_nodes(ex, ey, ez)
                a = en.index(nd)
                dofs = np.array([3 * m + c for m in en for c in range(3)])
                e = ex + self.p.nx * (ey + self.p.ny * ez)
                if self.p.elem_q1[e]:
                    if a not in vloc:
                        continue  # a slaved node of this element: identity row
                    vd = np.array([3 * vloc[v] + c for v in range(8) for c in range(3)])
                    ue = uf[dofs][vd]
                    ue = np.abs(ue if P1 is None else P1 @ ue)
                    if elem_max:
                        ue = np.full_like(ue, ue.max())
                    v = vloc.index(a)
                    for i in range(len(cells)):
                        out[q] += w[i] * (np.abs(self.K1[i][3 * v: 3 * v + 3]) @ ue)
                else:
                    T = self._T_e(en)
                    ue = T @ uf[dofs]
                    ue = np.abs(ue if P2 is None else P2 @ ue)
                    if elem_max:
                        ue = np.full_like(ue, ue.max())
                    z = np.zeros(3 * len(en))
                    for i in range(len(cells)):
                        z += w[i] * (np.abs(self.K[i]) @ ue)
                    out[q] += (T.T @ z)[3 * a: 3 * a + 3]
            for c in range(3):
                if held[3 * nd + c]:
                    out[q, c] = abs(u[3 * nd + c])
        return out

    # ---- gradient ---------------------------------------------------------
    def drho(self, x, u, cell):
        """dc/drho at one density cell for the (expanded) displacement u."""
        n = self.n
        cx, cy, cz = cell % self.Dx, (cell // self.Dx) % self.Dy, cell // (self.Dx * self.Dy)
        ex, ey, ez = cx // n, cy // n, cz // n
        i = (cx % n) + n * ((cy % n) + n * (cz % n))
        en = self._elem_nodes(ex, ey, ez)
        ue = u[np.array([3 * m + c for m in en for c in range(3)])]
        s = ue @ self.K[i] @ ue
        r = self.rho(x, cell)
        return -self.p.penal * r ** (self.p.penal - 1.0) * (self.p.E0 - self.p.Emin) * s

    def drho_scale(self, x, u, cell):
        """|dc/drho| scale of the rounding of the quadratic form at a cell:
        p rho^(p-1) (E0 - Emin) sum_ab |K_ab u_a u_b|.  Two FP64 evaluations
        of u_e^T K^(e_i) u_e in different orders differ by a small multiple
        of eps times this (much more than eps |dc/drho| where u_e is close
        to a rigid motion and the terms cancel)."""
        n = self.n
        cx, cy, cz = cell % self.Dx, (cell // self.Dx) % self.Dy, cell // (self.Dx * self.Dy)
        ex, ey, ez = cx // n, cy // n, cz // n
        i = (cx % n) + n * ((cy % n) + n * (cz % n))
        en = self._elem_nodes(ex, ey, ez)
        ue = np.abs(u[np.array([3 * m + c for m in en for c in range(3)])])
        r = self.rho(x, cell)
        return self.p.penal * r ** (self.p.penal - 1.0) * (self.p.E0 - self.p.Emin) * (ue @ np.abs(self.K[i]) @ ue)

    def dx_scale(self, x, u, cell):
        """Rounding scale of dx: the filter weights times the drho_scale of
        every density cell in the ball."""
        cx, cy, cz = cell % self.Dx, (cell // self.Dx) % self.Dy, cell // (self.Dx * self.Dy)
        total = 0.0
        for (di, dj, dk), w in zip(self.offs, self.wts):
            jx, jy, jz = cx + di, cy + dj, cz + dk
            if not self._in(jx, jy, jz):
                continue
            den = 0.0
            for (ei, ej, ek), w2 in zip(self.offs, self.wts):
                if self._in(jx + ei, jy + ej, jz + ek):
                    den += w2
            total += w / den * self.drho_scale(x, u, self._cell(jx, jy, jz))
        return total

    def dx(self, x, u, cell):
        """dc/dx at one design cell: sum over the ball of w_ji / omega_j * dc/drho_j."""
        cx, cy, cz = cell % self.Dx, (cell // self.Dx) % self.Dy, cell // (self.Dx * self.Dy)
        total = 0.0
        for (di, dj, dk), w in zip(self.offs, self.wts):
            jx, jy, jz = cx + di, cy + dj, cz + dk
            if not self._in(jx, jy, jz):
                continue
            den = 0.0
            for (ei, ej, ek), w2 in zip(self.offs, self.wts):
                if self._in(jx + ei, jy + ej, jz + ek):
                    den += w2
            total += w / den * self.drho(x, u, self._cell(jx, jy, jz))
        return total
