"""Geometric multigrid cycle and MG-preconditioned CG (oracle).

Section 2.3, Algorithm 1 (two-grid cycle), applied recursively for more
levels: smooth eta1 times, residual, restrict with R = P^T, solve (or recurse
gamma times: gamma = 1 is a V-cycle, 2 a W-cycle) on the coarse grid, prolong
and correct, smooth eta2 times.  Section 2.3: a coarse element holds 2x2x2
fine elements and P is linear interpolation between the node lattices.
Section 7 (intro): damped Jacobi, omega = 0.5, eta1 = eta2 = 1.
Section 7.2: the coarsest system is solved by a Cholesky factorization; PCG
stops when ||r|| / ||f|| < 1e-8 (the denominator reading: ||f||).

Readings taken here (the paper does not say):
  * coarse operators are re-discretised from the density field itself: a
    level-l element (edge 2^l) covers (n 2^l)^3 density cells and its matrix
    is Eq. matrixK_mr with that many subcells.  For Lagrange Q1 this equals
    the Galerkin product P^T A P exactly (tested), since trilinear
    interpolation reproduces the coarse shape functions;
  * supports: a coarse DOF is fixed iff the coincident fine DOF is fixed;
    fixed rows/columns of every level operator are replaced by identity and
    P is masked on both sides, P = M_f P_lin M_c;
  * the prolongation is trilinear interpolation on the node lattices (the
    paper's choice for Lagrange elements) for degree 1, where it is also the
    shape-function interpolation, and on request for degree 2; by default a
    degree-2 level is interpolated with the coarse shape functions, the
    construction the paper proposes for serendipity elements: the quadratic
    spaces are nested, so the re-discretised coarse operator is then the
    Galerkin product P^T A P (tested);
  * serendipity levels hold their face and element-centre nodes at 0 like
    supports, and use omega = 0.3 (damped Jacobi with 0.5 diverges on these
    elements: lambda_max(D^-1 A) is about 5.3 for degree 2, 5.0 for degree
    3); Lagrange hierarchies of degree 2 and 3 use 0.4 (lambda_max about 4.7
    for degree 2 with n = 2 subcells per edge, 4.9 with n = 3, 4.0 for
    degree 3: 0.5 would exceed 2 / lambda_max, the damped iteration's
    stability bound, while Sec. 7's 0.5 stays for trilinear elements);
  * Chebyshev smoothing (the alternative to damped Jacobi that the method
    statement names; the paper itself smooths degree >= 2 with SSOR,
    Sec. 7.5): the Chebyshev iteration of Saad, Iterative Methods for Sparse
    Linear Systems, Sec. 12.3, on D^-1 A over [0.3 b, b] with b = 1.1 x the
    largest eigenvalue of D^-1 A as estimated by `lanczos_steps` Lanczos
    steps from a fixed start vector (the Weyl sequence frac(d phi) - 1/2 over
    the DOF index d, zero at fixed DOFs), `cheb_degree` steps before and
    after the coarse correction.  The same polynomial pre and post keeps the
    cycle symmetric.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fem, mesh
from .fe import simp_weights


def _interp_1d(nf: int) -> sp.csr_matrix:
    """Linear interpolation from a lattice of (nf-1)/2+1 nodes to nf nodes."""
    nc = (nf - 1) // 2 + 1
    rows, cols, vals = [], [], []
    for i in range(nf):
        if i % 2 == 0:
            rows.append(i); cols.append(i // 2); vals.append(1.0)
        else:
            rows += [i, i]; cols += [(i - 1) // 2, (i + 1) // 2]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def prolongation(lat_fine) -> sp.csr_matrix:
    """Unmasked trilinear P_lin between node lattices, DOF-interleaved."""
    Lx, Ly, Lz = lat_fine
    Pn = sp.kron(sp.kron(_interp_1d(Lz), _interp_1d(Ly)), _interp_1d(Lx))
    return sp.kron(Pn, sp.identity(3), format="csr")


def _quad_1d(nf: int) -> sp.csr_matrix:
    """Interpolation by the coarse quadratic Lagrange basis from a degree-2
    lattice of (nf-1)/2+1 nodes to the degree-2 lattice of twice as many
    elements (nf nodes): fine node i lies in coarse element min(i // 4, E - 1)
    at xi = -1 + (i - 4 e) / 2."""
    E = (nf - 1) // 4
    nc = 2 * E + 1
    rows, cols, vals = [], [], []
    for i in range(nf):
        e = min(i // 4, E - 1)
        xi = -1.0 + 0.5 * (i - 4 * e)
        N = (0.5 * xi * (xi - 1.0), 1.0 - xi * xi, 0.5 * xi * (xi + 1.0))
        for j in range(3):
            if N[j] != 0.0:
                rows.append(i); cols.append(2 * e + j); vals.append(N[j])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def prolongation_shape(lat_fine, family: str = "lagrange") -> sp.csr_matrix:
    """Interpolation by the coarse degree-2 shape functions (Lagrange: the
    tensor product of _quad_1d; serendipity: the 20-node shape functions of
    oracle/fem.py in the coarse element owning each fine node)."""
    Lx, Ly, Lz = lat_fine
    if family == "lagrange":
        Pn = sp.kron(sp.kron(_quad_1d(Lz), _quad_1d(Ly)), _quad_1d(Lx))
        return sp.kron(Pn, sp.identity(3), format="csr")
    Ex, Ey, Ez = (Lx - 1) // 4, (Ly - 1) // 4, (Lz - 1) // 4
    Lxc, Lyc = 2 * Ex + 1, 2 * Ey + 1
    nc = Lxc * Lyc * (2 * Ez + 1)
    rows, cols, vals = [], [], []
    for node in range(Lx * Ly * Lz):
        i, j, l = node % Lx, (node // Lx) % Ly, node // (Lx * Ly)
        ex, ey, ez = min(i // 4, Ex - 1), min(j // 4, Ey - 1), min(l // 4, Ez - 1)
        N, _ = fem.serendipity2_shape(-1.0 + 0.5 * (i - 4 * ex), -1.0 + 0.5 * (j - 4 * ey),
                                      -1.0 + 0.5 * (l - 4 * ez))
        for a in range(27):
            if N[a] != 0.0:
                cn = (2 * ex + a % 3) + Lxc * ((2 * ey + (a // 3) % 3) + Lyc * (2 * ez + a // 9))
                rows.append(node); cols.append(cn); vals.append(N[a])
    Pn = sp.csr_matrix((vals, (rows, cols)), shape=(Lx * Ly * Lz, nc))
    return sp.kron(Pn, sp.identity(3), format="csr")


def serendipity_absent(lat, k: int = 2) -> np.ndarray:
    """(3 nnodes,) bool: DOFs of degree-k lattice nodes with two or three
    coordinates inside an element edge (no serendipity node there)."""
    Lx, Ly, Lz = lat
    n = np.arange(Lx * Ly * Lz)
    i, j, l = n % Lx, (n // Lx) % Ly, n // (Lx * Ly)
    return np.repeat((i % k != 0).astype(int) + (j % k != 0) + (l % k != 0) >= 2, 3)


def prolongation_p(mesh_shape, family: str = "lagrange") -> sp.csr_matrix:
    """Degree 2 -> degree 3 on the same mesh: the value at every node of the
    degree-3 lattice of the degree-2 shape functions of the element owning
    it (element min(i // 3, E - 1) along each axis, local xi = -1 + 2 f / 3).
    The quadratic spaces are contained in the cubic ones of the same family,
    so the degree-2 operator re-discretised on the same mesh is the Galerkin
    product."""
    nx, ny, nz = mesh_shape
    L3 = (3 * nx + 1, 3 * ny + 1, 3 * nz + 1)
    L2x, L2y = 2 * nx + 1, 2 * ny + 1
    nc = L2x * L2y * (2 * nz + 1)
    rows, cols, vals = [], [], []
    lag = lambda j, x: (0.5 * x * (x - 1.0), 1.0 - x * x, 0.5 * x * (x + 1.0))[j]
    for node in range(L3[0] * L3[1] * L3[2]):
        i, j, l = node % L3[0], (node // L3[0]) % L3[1], node // (L3[0] * L3[1])
        ex, ey, ez = min(i // 3, nx - 1), min(j // 3, ny - 1), min(l // 3, nz - 1)
        x = (-1.0 + 2.0 * (i - 3 * ex) / 3.0, -1.0 + 2.0 * (j - 3 * ey) / 3.0, -1.0 + 2.0 * (l - 3 * ez) / 3.0)
        if family == "lagrange":
            N = np.array([lag(a % 3, x[0]) * lag((a // 3) % 3, x[1]) * lag(a // 9, x[2]) for a in range(27)])
        else:
            N, _ = fem.serendipity2_shape(*x)
        for a in range(27):
            if N[a] != 0.0:
                cn = (2 * ex + a % 3) + L2x * ((2 * ey + (a // 3) % 3) + L2y * (2 * ez + a // 9))
                rows.append(node); cols.append(cn); vals.append(N[a])
    Pn = sp.csr_matrix((vals, (rows, cols)), shape=(L3[0] * L3[1] * L3[2], nc))
    return sp.kron(Pn, sp.identity(3), format="csr")


def p_coarse_mask(mask3: np.ndarray, mesh_shape) -> np.ndarray:
    """Degree-2 mask from a degree-3 mask on the same mesh: a degree-2 DOF is
    fixed iff every degree-3 DOF of the same component at its place is
    fixed -- per axis, a vertex coordinate 2I meets the node 3I, a midpoint
    2I + 1 the two nodes 3I + 1 and 3I + 2 inside the same edge."""
    nx, ny, nz = mesh_shape
    L3 = (3 * nx + 1, 3 * ny + 1, 3 * nz + 1)
    m3 = mask3.reshape(L3[2], L3[1], L3[0], 3).astype(bool)
    def idx(I):
        return [3 * I // 2] if I % 2 == 0 else [3 * (I - 1) // 2 + 1, 3 * (I - 1) // 2 + 2]
    out = np.zeros((2 * nz + 1, 2 * ny + 1, 2 * nx + 1, 3), dtype=np.uint8)
    for K in range(2 * nz + 1):
        for J in range(2 * ny + 1):
            for I in range(2 * nx + 1):
                sub = m3[np.ix_(idx(K), idx(J), idx(I))]
                out[K, J, I] = sub.reshape(-1, 3).all(axis=0)
    return out.reshape(-1)


GOLDEN = 0.6180339887498949  # (sqrt 5 - 1) / 2


def weyl_start(ndof: int, mask: np.ndarray) -> np.ndarray:
    """The Lanczos start vector: frac(d * phi) - 1/2 for DOF index d
    (a Weyl sequence), 0 at the fixed DOFs."""
    x = np.arange(ndof, dtype=np.float64) * GOLDEN
    x = x - np.floor(x) - 0.5
    x[np.asarray(mask) != 0] = 0.0
    return x


def lanczos_lmax(A, Dinv: np.ndarray, mask: np.ndarray, steps: int) -> float:
    """Estimate of the largest eigenvalue of D^-1 A: the largest Ritz value
    after `steps` Lanczos steps on the symmetric D^-1/2 A D^-1/2 from
    D^1/2 weyl_start, written in the unscaled vectors p = D^-1/2 q:
        alpha_j = p_j^T A p_j,
        s = D^-1 A p_j - alpha_j p_j - beta_j p_{j-1},
        beta_{j+1} = (s^T D s)^1/2,  p_{j+1} = s / beta_{j+1},
    with p_1^T D p_1 = 1; the Ritz values are the eigenvalues of the
    tridiagonal matrix (alpha; beta_2 ..), each at most lambda_max."""
    from scipy.linalg import eigvalsh_tridiagonal

    p = weyl_start(A.shape[0], mask)
    p = p / np.sqrt(p @ (p / Dinv))
    p_prev = np.zeros_like(p)
    alphas, betas = [], []
    beta = 0.0
    for j in range(steps):
        y = A @ p
        alpha = p @ y
        alphas.append(alpha)
        if j == steps - 1:
            break
        sv = Dinv * y - alpha * p - beta * p_prev
        beta = np.sqrt(sv @ (sv / Dinv))
        betas.append(beta)
        p_prev, p = p, sv / beta
    return float(eigvalsh_tridiagonal(np.array(alphas), np.array(betas))[-1])


def chebyshev_coefficients(lmax_est: float, degree: int):
    """Interval [0.3 b, b], b = 1.1 lmax_est: centre theta, half-width delta.
    Returns 1/theta (the first step, x1 = x0 + D^-1 r0 / theta) and, for each
    further step i, (rho_i rho_{i-1}, 2 rho_i / delta) with rho_0 =
    delta / theta and rho_i = 1 / (2 theta / delta - rho_{i-1}) (Saad,
    Algorithm 12.1 on D^-1 A)."""
    hi = 1.1 * lmax_est
    lo = 0.3 * hi
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    coefs = []
    for _ in range(1, degree):
        rho_n = 1.0 / (2.0 * sigma - rho)
        coefs.append((rho_n * rho, 2.0 * rho_n / delta))
        rho = rho_n
    return 1.0 / theta, coefs, theta, delta


def chebyshev_smooth(L, b: np.ndarray, x: np.ndarray) -> np.ndarray:
    """cheb_degree Chebyshev steps on A x = b from x: x1 = x0 + D^-1 (b - A
    x0) / theta, then x_i = x_{i-1} + c1_i (x_{i-1} - x_{i-2}) + c2_i D^-1 (b
    - A x_{i-1})."""
    inv_theta, coefs = L.cheb[0], L.cheb[1]
    x_prev = x
    x = x + inv_theta * L.Dinv * (b - L.A @ x)
    for c1, c2 in coefs:
        x_new = x + c1 * (x - x_prev) + c2 * L.Dinv * (b - L.A @ x)
        x_prev, x = x, x_new
    return x


def coarse_mask(mask_f: np.ndarray, lat_fine) -> np.ndarray:
    """Coarse DOF fixed iff the coincident fine DOF is fixed."""
    Lx, Ly, Lz = lat_fine
    m = mask_f.reshape(Lz, Ly, Lx, 3)
    return np.ascontiguousarray(m[::2, ::2, ::2, :]).reshape(-1)


class Level:
    pass


class Hierarchy:
    """Level operators A_l (supports -> identity), Jacobi diagonals, P_l and
    the dense Cholesky factor of the coarsest operator."""

    def __init__(self, prob, rho: np.ndarray, levels: int, transfer: str | None = None,
                 smoother: str = "jacobi", cheb_degree: int = 2, lanczos_steps: int = 8):
        if smoother not in ("jacobi", "chebyshev"):
            raise ValueError("smoother is 'jacobi' or 'chebyshev'")
        self.smoother = smoother
        if prob.degree == 3:
            self._init_cubic(prob, rho, levels, smoother, cheb_degree, lanczos_steps)
            self._init_chebyshev(cheb_degree, lanczos_steps)
            return
        k, n = prob.degree, prob.n_mr
        family = getattr(prob, "family", "lagrange")
        if transfer is None:
            transfer = "shape" if k == 2 else "linear"
        if family == "serendipity" and transfer != "shape":
            raise ValueError("serendipity levels take shape-function transfers")
        self.omega = 0.3 if family == "serendipity" else (0.4 if k >= 2 else 0.5)
        nx, ny, nz = prob.nx, prob.ny, prob.nz
        w_cells = simp_weights(rho, prob.E0, prob.Emin, prob.penal)
        self.levels = []
        mask = prob.mask.astype(np.uint8)
        for l in range(levels):
            s = 2 ** l
            if nx % s or ny % s or nz % s:
                raise ValueError("mesh not divisible for this many levels")
            L = Level()
            L.nx, L.ny, L.nz = nx // s, ny // s, nz // s
            L.nsub = n * s
            L.lat = (k * L.nx + 1, k * L.ny + 1, k * L.nz + 1)
            L.ndof = 3 * L.lat[0] * L.lat[1] * L.lat[2]
            L.mask = mask
            Ktab = fem.subcell_stiffness(k, L.nsub, prob.nu, h=float(s), family=family)
            m, d, _ = Ktab.shape
            w_e = w_cells[mesh.subcell_density_index(L.nx, L.ny, L.nz, L.nsub)]
            Ke = (w_e @ Ktab.reshape(m, d * d)).reshape(-1, d, d)
            ed = mesh.element_dofs(L.nx, L.ny, L.nz, k)
            rows = np.repeat(ed, d, axis=1).reshape(-1)
            cols = np.tile(ed, (1, d)).reshape(-1)
            K = sp.coo_matrix((Ke.reshape(-1), (rows, cols)), shape=(L.ndof, L.ndof)).tocsr()
            free = (mask == 0).astype(np.float64)
            Mf = sp.diags(free)
            L.A = (Mf @ K @ Mf + sp.diags(1.0 - free)).tocsr()
            L.Dinv = 1.0 / L.A.diagonal()
            self.levels.append(L)
            if l + 1 < levels:
                mask = coarse_mask(mask, L.lat)
                if family == "serendipity":
                    lat_c = (k * (nx // (2 * s)) + 1, k * (ny // (2 * s)) + 1, k * (nz // (2 * s)) + 1)
                    mask = (mask.astype(bool) | serendipity_absent(lat_c)).astype(np.uint8)
        for l in range(levels - 1):
            F, C = self.levels[l], self.levels[l + 1]
            P = prolongation_shape(F.lat, family) if transfer == "shape" else prolongation(F.lat)
            Mf = sp.diags((F.mask == 0).astype(np.float64))
            Mc = sp.diags((C.mask == 0).astype(np.float64))
            F.P = (Mf @ P @ Mc).tocsr()
        last = self.levels[-1]
        last.chol = sla.cho_factor(last.A.toarray(), lower=True)
        self._init_chebyshev(cheb_degree, lanczos_steps)

    def _init_chebyshev(self, degree: int, steps: int):
        """Chebyshev data of every level but the coarsest (Jacobi: none)."""
        for L in self.levels[:-1]:
            L.lmax = lanczos_lmax(L.A, L.Dinv, L.mask, steps) if self.smoother == "chebyshev" else None
            L.cheb = chebyshev_coefficients(L.lmax, degree) if L.lmax is not None else None


def _cubic_levels(self, prob, rho, levels, smoother="jacobi", cheb_degree=2, lanczos_steps=8):
    """Degree 3 (Lagrange or serendipity): level 0 is the degree-3 mesh,
    level 1 the degree-2 mesh of the same family on the same elements (the
    degree is coarsened first, Sec. 2.3's shape-function interpolation as
    P), and the further levels the degree-2 hierarchy below it."""
    family = getattr(prob, "family", "lagrange")
    if levels < 2:
        raise ValueError("degree 3 takes at least two levels")
    # levels 1.. : the degree-2 hierarchy of the same mesh and densities
    import copy

    q = copy.copy(prob)
    q.degree = 2
    lat2 = (2 * prob.nx + 1, 2 * prob.ny + 1, 2 * prob.nz + 1)
    m2 = p_coarse_mask(prob.mask, (prob.nx, prob.ny, prob.nz))
    if family == "serendipity":
        m2 = (m2.astype(bool) | serendipity_absent(lat2, 2)).astype(np.uint8)
    q.mask = m2
    sub = Hierarchy(q, rho, levels - 1, smoother=smoother, cheb_degree=cheb_degree, lanczos_steps=lanczos_steps)
    self.omega = 0.3 if family == "serendipity" else 0.4
    w_cells = simp_weights(rho, prob.E0, prob.Emin, prob.penal)
    F = Level()
    F.nx, F.ny, F.nz = prob.nx, prob.ny, prob.nz
    F.nsub = prob.n_mr
    F.lat = (3 * F.nx + 1, 3 * F.ny + 1, 3 * F.nz + 1)
    F.ndof = 3 * F.lat[0] * F.lat[1] * F.lat[2]
    F.mask = prob.mask.astype(np.uint8)
    Ktab = fem.subcell_stiffness(3, F.nsub, prob.nu, family=family)
    m, d, _ = Ktab.shape
    w_e = w_cells[mesh.subcell_density_index(F.nx, F.ny, F.nz, F.nsub)]
    Ke = (w_e @ Ktab.reshape(m, d * d)).reshape(-1, d, d)
    ed = mesh.element_dofs(F.nx, F.ny, F.nz, 3)
    K = sp.coo_matrix((Ke.reshape(-1), (np.repeat(ed, d, axis=1).reshape(-1), np.tile(ed, (1, d)).reshape(-1))),
                      shape=(F.ndof, F.ndof)).tocsr()
    free = (F.mask == 0).astype(np.float64)
    Mf = sp.diags(free)
    F.A = (Mf @ K @ Mf + sp.diags(1.0 - free)).tocsr()
    F.Dinv = 1.0 / F.A.diagonal()
    C = sub.levels[0]
    Mc = sp.diags((C.mask == 0).astype(np.float64))
    F.P = (Mf @ prolongation_p((F.nx, F.ny, F.nz), family) @ Mc).tocsr()
    self.levels = [F] + sub.levels


Hierarchy._init_cubic = _cubic_levels


def vcycle(h: Hierarchy, b: np.ndarray, l: int = 0, omega: float | None = None, eta1: int = 1,
           eta2: int = 1, gamma: int = 1) -> np.ndarray:
    """Approximate A_l^{-1} b by one multigrid cycle from a zero initial guess
    (Algorithm 1 applied recursively).  omega: the hierarchy's default."""
    omega = h.omega if omega is None else omega
    L = h.levels[l]
    if l == len(h.levels) - 1:
        return sla.cho_solve(L.chol, b)
    cheb = getattr(h, "smoother", "jacobi") == "chebyshev"
    v = np.zeros_like(b)
    for _ in range(eta1):  # step 1: pre-smoothing, damped Jacobi or Chebyshev
        v = chebyshev_smooth(L, b, v) if cheb else v + omega * L.Dinv * (b - L.A @ v)
    r = b - L.A @ v  # step 2: residual
    rH = L.P.T @ r  # step 3: restriction R = P^T
    eH = np.zeros_like(rH)
    for _ in range(gamma):  # step 4: coarse solve by recursion
        eH = eH + vcycle(h, rH - h.levels[l + 1].A @ eH, l + 1, omega, eta1, eta2, gamma)
    v = v + L.P @ eH  # steps 5-6: prolong and correct
    for _ in range(eta2):  # step 7: post-smoothing
        v = chebyshev_smooth(L, b, v) if cheb else v + omega * L.Dinv * (b - L.A @ v)
    return v


def pcg(h: Hierarchy, f: np.ndarray, u0: np.ndarray | None = None, rtol: float = 1e-8,
        maxit: int = 1000, **cyc):
    """Preconditioned CG on A_0 u = f (supports are identity rows; f must be
    zero there).  Stops when ||f - A u|| / ||f|| <= rtol.  Returns
    (u, iterations, relative residual history)."""
    A = h.levels[0].A
    u = np.zeros_like(f) if u0 is None else u0.copy()
    r = f - A @ u
    nf = np.linalg.norm(f)
    hist = [np.linalg.norm(r) / nf]
    if hist[-1] <= rtol:
        return u, 0, hist
    z = vcycle(h, r, **cyc)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = A @ p
        alpha = rz / (p @ q)
        u += alpha * p
        r -= alpha * q
        hist.append(np.linalg.norm(r) / nf)
        if hist[-1] <= rtol:
            return u, it, hist
        z = vcycle(h, r, **cyc)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return u, maxit, hist
