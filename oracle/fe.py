"""Assembled-sparse FP64 elasticity solve, compliance and gradient (oracle).

Section 2, Eq. matrixK and Section 3.3, Eq. matrixK_mr:
    K^(e)(rho) = sum_i (Emin + rho_{e_i}^p (E0 - Emin)) K^(e_i),
K = superposition of the K^(e); K u = f with the supports removed
(Section 2: after imposing the boundary conditions K is positive definite).
Compliance f^T u (Problem topopt).  Section 3.4: with
s_{e,i} = u_e^T K^(e_i) u_e,
    d f / d rho_i = -p rho_i^(p-1) (E0 - Emin) s_{e,i},
    d f / d x_k   = sum_i (w_ik / w_i) d f / d rho_i   (= H^T g).
Multiple load cases are independent solves with the same K; the compliance
is reported per case and the gradient is summed over cases.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, filt, mesh


def simp_weights(rho: np.ndarray, E0: float, Emin: float, p: float) -> np.ndarray:
    """w = Emin + rho^p (E0 - Emin)  (Eq. matrixK)."""
    return Emin + rho ** p * (E0 - Emin)


def rigid_projector(k: int) -> np.ndarray:
    """(d, d) orthogonal projector onto the complement of the six rigid
    motions (translations, infinitesimal rotations omega x x) of one element
    of degree k, in the Euclidean inner product of its d = 3 (k+1)^3 nodal
    values, nodes at reference positions -1 + 2 a / k (lattice order, x
    fastest).  Rigid motions carry no strain, so K^(e_i) P = K^(e_i)."""
    na = k + 1
    pos = np.array([[-1.0 + 2.0 * ax / k, -1.0 + 2.0 * ay / k, -1.0 + 2.0 * az / k]
                    for az in range(na) for ay in range(na) for ax in range(na)])
    nn = pos.shape[0]
    R = np.zeros((3 * nn, 6))
    for a, (x, y, z) in enumerate(pos):
        R[3 * a: 3 * a + 3, 0:3] = np.identity(3)
        R[3 * a: 3 * a + 3, 3:6] = [[0.0, z, -y], [-z, 0.0, x], [y, -x, 0.0]]  # omega x pos
    Q, _ = np.linalg.qr(R)
    return np.identity(3 * nn) - Q @ Q.T


class Model:
    """Everything the oracle needs for one problem (see workloads.Problem)."""

    def __init__(self, prob):
        self.p = prob
        k, n = prob.degree, prob.n_mr
        self.k, self.n = k, n
        self.Ktab = fem.subcell_stiffness(k, n, prob.nu, family=getattr(prob, "family", "lagrange"))  # (m, d, d)
        self.edofs = mesh.element_dofs(prob.nx, prob.ny, prob.nz, k)
        self.sub2cell = mesh.subcell_density_index(prob.nx, prob.ny, prob.nz, n)
        d = getattr(prob, "d_mr", None) or n
        self.H = filt.projection_matrix(prob.nx, prob.ny, prob.nz, n, d, prob.rmin)
        self.ndof = prob.ndof
        self.free = np.nonzero(prob.mask == 0)[0]

    # -- density side --------------------------------------------------
    def densities(self, x: np.ndarray) -> np.ndarray:
        """rho = H x (Eq. projdsgn / the filter)."""
        return self.H @ x

    def weights(self, rho: np.ndarray) -> np.ndarray:
        """(E, m) SIMP weights of every subcell."""
        pr = self.p
        return simp_weights(rho, pr.E0, pr.Emin, pr.penal)[self.sub2cell]

    # -- operator ------------------------------------------------------
    def element_matrices(self, w_e: np.ndarray) -> np.ndarray:
        """(E, d, d): K^(e) = sum_i w_{e,i} K^(e_i)  (Eq. matrixK_mr)."""
        m, d, _ = self.Ktab.shape
        return (w_e @ self.Ktab.reshape(m, d * d)).reshape(-1, d, d)

    def assemble(self, w_e: np.ndarray) -> sp.csr_matrix:
        """Global K(rho) by superposition of element matrices (no BCs)."""
        Ke = self.element_matrices(w_e)
        E, d, _ = Ke.shape
        rows = np.repeat(self.edofs, d, axis=1).reshape(-1)
        cols = np.tile(self.edofs, (1, d)).reshape(-1)
        K = sp.coo_matrix((Ke.reshape(-1), (rows, cols)), shape=(self.ndof, self.ndof))
        return K.tocsr()

    def apply(self, w_e: np.ndarray, u: np.ndarray) -> np.ndarray:
        """y = K u with the supports' rows and columns replaced by identity
        (the operator the solver sees; u, y are full-length)."""
        mask = self.p.mask.astype(bool)
        uf = np.where(mask, 0.0, u)
        y = self.assemble(w_e) @ uf
        y[mask] = u[mask]
        return y

    def subcell_scale(self, w_e: np.ndarray, u: np.ndarray, deflate: bool = False,
                      elem_max: bool = False) -> np.ndarray:
        """Per DOF, sum over the elements e and subcells i of
        w_{e,i} (|K^(e_i)| |u_e|): the scale of the rounding error of the
        stacked form of Eq. matrixK_mr, which forms each subcell's product
        K^(e_i) u_e on its own before the weighted sum (supports: |u|, as
        identity rows; their columns are zero as in apply).  deflate: u_e
        minus its least-squares rigid motion (rigid_projector), which every
        K^(e_i) annihilates, in place of u_e.  elem_max: every |u_e| entry
        replaced by max |u_e| (the scale of errors relative to an element's
        largest value, as a power-of-two scaled 16-bit split makes)."""
        mask = self.p.mask.astype(bool)
        ue = np.where(mask, 0.0, u)[self.edofs]  # (E, d)
        if deflate:
            ue = ue @ rigid_projector(self.k).T
        ua = np.abs(ue)
        if elem_max:
            ua = np.repeat(ua.max(axis=1, keepdims=True), ua.shape[1], axis=1)
        z = np.einsum("eid,idf,ef->ed", np.broadcast_to(w_e[:, :, None], w_e.shape + (self.Ktab.shape[1],)),
                      np.abs(self.Ktab), ua, optimize=True)
        out = np.zeros(self.ndof)
        np.add.at(out, self.edofs, z)
        out[mask] = np.abs(u[mask])
        return out

    # -- solve -----------------------------------------------------------
    def solve(self, w_e: np.ndarray, f: np.ndarray, method: str = "auto",
              tol: float = 1e-13, K: sp.csr_matrix | None = None) -> np.ndarray:
        """u with K_ff u_f = f_f and u = 0 on the supports.

        method: 'dense' (Cholesky, numpy/scipy), 'splu' (SuperLU), 'cg'
        (Jacobi-preconditioned CG to ||r||/||f|| <= tol) or 'auto'."""
        if K is None:
            K = self.assemble(w_e)
        fr = self.free
        Kff = K[fr][:, fr]
        ff = f[fr]
        nf = fr.size
        if method == "auto":
            method = "dense" if nf <= 3000 else ("splu" if nf <= 400000 else "cg")
        if method == "dense":
            c = sla.cho_factor(Kff.toarray(), lower=True)
            uf = sla.cho_solve(c, ff)
        elif method == "splu":
            lu = spla.splu(Kff.tocsc(), permc_spec="MMD_AT_PLUS_A")
            uf = lu.solve(ff)
        elif method == "cg":
            dinv = 1.0 / Kff.diagonal()
            M = spla.LinearOperator(Kff.shape, matvec=lambda v: dinv * v)
            uf, info = spla.cg(Kff, ff, rtol=tol, atol=0.0, maxiter=200000, M=M)
            if info != 0:
                raise RuntimeError(f"oracle CG did not converge (info={info})")
        else:
            raise ValueError(method)
        u = np.zeros(self.ndof)
        u[fr] = uf
        return u

    # -- objective and gradient -------------------------------------------
    @staticmethod
    def compliance(f: np.ndarray, u: np.ndarray, mask: np.ndarray) -> float:
        """c = f^T u over the free DOFs (f at supports is ignored)."""
        free = mask == 0
        return float(np.dot(f[free], u[free]))

    def subcell_energies(self, u: np.ndarray) -> np.ndarray:
        """(E, m): s_{e,i} = u_e^T K^(e_i) u_e (Section 3.4)."""
        ue = u[self.edofs]  # (E, d)
        return np.einsum("ed,idf,ef->ei", ue, self.Ktab, ue, optimize=True)

    def density_gradient(self, rho: np.ndarray, s: np.ndarray) -> np.ndarray:
        """d f / d rho on the density grid: -p rho^(p-1) (E0 - Emin) s."""
        pr = self.p
        g = np.zeros(rho.size)
        g[self.sub2cell.reshape(-1)] = s.reshape(-1)
        return -pr.penal * rho ** (pr.penal - 1.0) * (pr.E0 - pr.Emin) * g

    def design_gradient(self, g_rho: np.ndarray) -> np.ndarray:
        """d f / d x = H^T g  (chain rule through Eq. projdsgn)."""
        return self.H.T @ g_rho

    def run(self, x: np.ndarray | None = None, method: str = "auto", rtol: float = 1e-13,
            levels: int | None = None):
        """The whole path for all load cases: rho, w, u, c, dc/drho, dc/dx.

        method 'mg' solves with the oracle's own MG-PCG (oracle/mg.py, pinned
        against the direct solve) to ||r||/||f|| <= rtol; it is the large-size
        path (a sparse direct solve of 10^5 3D elasticity DOFs takes minutes)."""
        pr = self.p
        x = pr.x if x is None else x
        rho = self.densities(x)
        w_e = self.weights(rho)
        K = self.assemble(w_e)
        hier = None
        if method == "mg":
            from . import mg
            hier = mg.Hierarchy(pr, rho, levels or pr.mg_levels or 1)
        us, cs = [], []
        g_rho = np.zeros(rho.size)
        for r in range(pr.nrhs):
            f = pr.f[r].copy()
            f[pr.mask.astype(bool)] = 0.0
            if hier is not None:
                from . import mg
                u, _, _ = mg.pcg(hier, f, rtol=rtol, maxit=5000)
            else:
                u = self.solve(w_e, f, method=method, K=K)
            us.append(u)
            cs.append(self.compliance(f, u, pr.mask))
            g_rho += self.density_gradient(rho, self.subcell_energies(u))
        return dict(rho=rho, w=w_e, u=np.array(us), c=np.array(cs), g_rho=g_rho,
                    g_x=self.design_gradient(g_rho))
