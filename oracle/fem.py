"""Element library of the oracle: Lagrange hexahedra of degree k = 1..3 and
the 20-node serendipity hexahedron.

Section 2.1 (finite element types): rectangular prismatic elements, three
displacement DOFs per node, Lagrange elements with (k+1)^3 nodes, and the
serendipity family, whose quadratic member has nodes at the 8 vertices and
the 12 edge midpoints only.  The serendipity element is written on the
27-node lattice of the quadratic Lagrange element (same local numbering),
with identically zero shape functions at the 6 face centres and the centre:
its matrices are 81 x 81 with zero rows and columns there.
Section 3.3 (assembly, Eq. matrixK_mr): a displacement element split into
n^3 density elements ("subcells"); the subcell matrices
    K^(e_i) = int_{Omega_{e_i}} B^T D B dOmega
are computed once for a regular mesh and K^(e) = sum_i w_i K^(e_i).

Conventions (shared with the C ABI by documentation only, not by code):
  * reference element [-1,1]^3, physical cube of edge h, so x = h/2 * xi;
  * local nodes on the equispaced (k+1)^3 lattice, index ix + (k+1)*(iy +
    (k+1)*iz), xi_ix = -1 + 2*ix/k;
  * element DOF 3*a + c for local node a and component c;
  * subcell (a, b, c) in 0..n-1 per axis has index a + n*(b + n*c) and covers
    xi in [-1 + 2a/n, -1 + 2(a+1)/n] (same for eta, zeta);
  * Voigt strain order (xx, yy, zz, xy, yz, zx) with engineering shears.
"""
from __future__ import annotations

import functools

import numpy as np
from numpy.polynomial import polynomial as npoly
from numpy.polynomial import legendre as nleg


def lagrange_1d(k: int):
    """Coefficients of the equispaced 1D Lagrange basis on [-1, 1].

    Returns (nodes, C, dC) with N_j(xi) = sum_p C[j, p] xi^p and
    N_j'(xi) = sum_p dC[j, p] xi^p.
    """
    nodes = np.linspace(-1.0, 1.0, k + 1)
    C = np.zeros((k + 1, k + 1))
    dC = np.zeros((k + 1, k + 1))
    for j in range(k + 1):
        others = np.delete(nodes, j)
        c = npoly.polyfromroots(others)  # prod (xi - xi_m)
        c = c / npoly.polyval(nodes[j], c)
        C[j, : len(c)] = c
        d = npoly.polyder(c)
        dC[j, : len(d)] = d
    return nodes, C, dC


def shape_1d(k: int, xi: float):
    """Values and derivatives of the k+1 1D basis functions at xi."""
    _, C, dC = lagrange_1d(k)
    return npoly.polyval(xi, C.T), npoly.polyval(xi, dC.T)


def shape_3d(k: int, xi: float, eta: float, zeta: float, h: float = 1.0):
    """Tensor-product shape functions at (xi, eta, zeta).

    Returns N (nn,) and dNdx (nn, 3), the physical gradient for a cube of
    edge h (d/dx = (2/h) d/dxi)."""
    Nx, dNx = shape_1d(k, xi)
    Ny, dNy = shape_1d(k, eta)
    Nz, dNz = shape_1d(k, zeta)
    nn = (k + 1) ** 3
    N = np.zeros(nn)
    dN = np.zeros((nn, 3))
    for iz in range(k + 1):
        for iy in range(k + 1):
            for ix in range(k + 1):
                a = ix + (k + 1) * (iy + (k + 1) * iz)
                N[a] = Nx[ix] * Ny[iy] * Nz[iz]
                dN[a, 0] = dNx[ix] * Ny[iy] * Nz[iz]
                dN[a, 1] = Nx[ix] * dNy[iy] * Nz[iz]
                dN[a, 2] = Nx[ix] * Ny[iy] * dNz[iz]
    return N, dN * (2.0 / h)


def serendipity2_shape(xi: float, eta: float, zeta: float, h: float = 1.0):
    """The 20-node serendipity shape functions on the 27-node lattice order.

    A vertex (xi_a, eta_a, zeta_a in {-1, 1}) has
        N = (1 + xi xi_a)(1 + eta eta_a)(1 + zeta zeta_a)(xi xi_a + eta eta_a + zeta zeta_a - 2) / 8,
    an edge midpoint with xi_a = 0 has N = (1 - xi^2)(1 + eta eta_a)(1 + zeta zeta_a) / 4
    (and the same with the roles of the coordinates exchanged); face centres
    and the centre have N = 0.  Returns N (27,) and the physical gradient
    dN (27, 3) for a cube of edge h."""
    x = (xi, eta, zeta)
    N = np.zeros(27)
    dN = np.zeros((27, 3))
    for iz in range(3):
        for iy in range(3):
            for ix in range(3):
                a = ix + 3 * (iy + 3 * iz)
                c = (ix - 1, iy - 1, iz - 1)
                mids = [q for q in range(3) if c[q] == 0]
                if len(mids) == 0:
                    f = [1.0 + x[q] * c[q] for q in range(3)]
                    s = x[0] * c[0] + x[1] * c[1] + x[2] * c[2] - 2.0
                    N[a] = f[0] * f[1] * f[2] * s / 8.0
                    for q in range(3):
                        o = [f[r] for r in range(3) if r != q]
                        dN[a, q] = (c[q] * o[0] * o[1] * s + f[0] * f[1] * f[2] * c[q]) / 8.0
                elif len(mids) == 1:
                    m = mids[0]
                    f = [(1.0 - x[q] * x[q]) if q == m else (1.0 + x[q] * c[q]) for q in range(3)]
                    df = [(-2.0 * x[q]) if q == m else c[q] for q in range(3)]
                    N[a] = f[0] * f[1] * f[2] / 4.0
                    dN[a, 0] = df[0] * f[1] * f[2] / 4.0
                    dN[a, 1] = f[0] * df[1] * f[2] / 4.0
                    dN[a, 2] = f[0] * f[1] * df[2] / 4.0
    return N, dN * (2.0 / h)


def serendipity2_present() -> np.ndarray:
    """(27,) bool: the 20 lattice positions that carry a serendipity node."""
    out = np.zeros(27, dtype=bool)
    for iz in range(3):
        for iy in range(3):
            for ix in range(3):
                out[ix + 3 * (iy + 3 * iz)] = (ix % 2) + (iy % 2) + (iz % 2) <= 1
    return out


def serendipity3_shape(xi: float, eta: float, zeta: float, h: float = 1.0):
    """The 32-node cubic serendipity shape functions on the 64-node lattice
    order of the cubic Lagrange element (lattice positions -1, -1/3, 1/3, 1
    per axis; index ix + 4 (iy + 4 iz)).

    A vertex (all coordinates +-1) has
        N = (1 + xi xi_a)(1 + eta eta_a)(1 + zeta zeta_a)(9 (xi^2 + eta^2 + zeta^2) - 19) / 64,
    an edge node with xi_a = +-1/3 (the others +-1)
        N = 9 (1 - xi^2)(1 + 9 xi xi_a)(1 + eta eta_a)(1 + zeta zeta_a) / 64
    (and the same with the coordinates exchanged); positions with two or
    three interior coordinates carry no node (N = 0).  Returns N (64,) and the
    physical gradient (64, 3) for a cube of edge h."""
    x = np.array([xi, eta, zeta], dtype=np.float64)
    pos = (-1.0, -1.0 / 3.0, 1.0 / 3.0, 1.0)
    N = np.zeros(64)
    dN = np.zeros((64, 3))
    for iz in range(4):
        for iy in range(4):
            for ix in range(4):
                a = ix + 4 * (iy + 4 * iz)
                c = np.array([pos[ix], pos[iy], pos[iz]])
                inner = [q for q in range(3) if abs(c[q]) < 1.0]
                if len(inner) == 0:
                    f = 1.0 + x * c
                    s = 9.0 * float(x @ x) - 19.0
                    N[a] = f[0] * f[1] * f[2] * s / 64.0
                    for q in range(3):
                        o = np.prod([f[r] for r in range(3) if r != q])
                        dN[a, q] = (c[q] * o * s + f[0] * f[1] * f[2] * 18.0 * x[q]) / 64.0
                elif len(inner) == 1:
                    m = inner[0]
                    f = np.array([(1.0 - x[q] * x[q]) * (1.0 + 9.0 * x[q] * c[q]) if q == m else 1.0 + x[q] * c[q]
                                  for q in range(3)])
                    df = np.array([(-2.0 * x[q]) * (1.0 + 9.0 * x[q] * c[q]) + (1.0 - x[q] * x[q]) * 9.0 * c[q]
                                   if q == m else c[q] for q in range(3)])
                    N[a] = 9.0 * f[0] * f[1] * f[2] / 64.0
                    dN[a, 0] = 9.0 * df[0] * f[1] * f[2] / 64.0
                    dN[a, 1] = 9.0 * f[0] * df[1] * f[2] / 64.0
                    dN[a, 2] = 9.0 * f[0] * f[1] * df[2] / 64.0
    return N, dN * (2.0 / h)


def serendipity_present(k: int) -> np.ndarray:
    """((k+1)^3,) bool: the lattice positions of the degree-k serendipity
    element (at most one interior coordinate): 20 for k = 2, 32 for k = 3."""
    na = k + 1
    out = np.zeros(na ** 3, dtype=bool)
    for iz in range(na):
        for iy in range(na):
            for ix in range(na):
                inner = sum(1 for c in (ix, iy, iz) if 0 < c < k)
                out[ix + na * (iy + na * iz)] = inner <= 1
    return out


def elasticity_D(nu: float, E: float = 1.0) -> np.ndarray:
    """Isotropic linear-elastic constitutive matrix (Voigt, engineering
    shear strains), the D of Eq. matrixK."""
    c = E / ((1.0 + nu) * (1.0 - 2.0 * nu))
    D = np.zeros((6, 6))
    D[:3, :3] = c * nu
    for i in range(3):
        D[i, i] = c * (1.0 - nu)
    for i in range(3, 6):
        D[i, i] = c * (1.0 - 2.0 * nu) / 2.0
    return D


def strain_displacement(dNdx: np.ndarray) -> np.ndarray:
    """B (6 x 3nn): strain = B u_e for element DOFs ordered 3*a + c."""
    nn = dNdx.shape[0]
    B = np.zeros((6, 3 * nn))
    for a in range(nn):
        gx, gy, gz = dNdx[a]
        B[0, 3 * a + 0] = gx
        B[1, 3 * a + 1] = gy
        B[2, 3 * a + 2] = gz
        B[3, 3 * a + 0] = gy
        B[3, 3 * a + 1] = gx
        B[4, 3 * a + 1] = gz
        B[4, 3 * a + 2] = gy
        B[5, 3 * a + 0] = gz
        B[5, 3 * a + 2] = gx
    return B


def subcell_stiffness(k: int, n: int, nu: float, h: float = 1.0, family: str = "lagrange") -> np.ndarray:
    """The stacked subcell stiffness table of Eq. matrixK_mr (a fresh copy of
    the memoised table: Section 3.3 computes it once for a regular mesh).
    family 'serendipity' (k = 2): the 20-node element on the 27-node lattice."""
    if family == "serendipity":
        if k == 2:
            return _subcell_stiffness_s2(int(n), float(nu), float(h)).copy()
        if k == 3:
            return _subcell_stiffness_s3(int(n), float(nu), float(h)).copy()
        raise ValueError("the serendipity element is built for degree 2 and 3")
    return _subcell_stiffness(int(k), int(n), float(nu), float(h)).copy()


@functools.lru_cache(maxsize=8)
def _subcell_stiffness_s2(n: int, nu: float, h: float) -> np.ndarray:
    """As _subcell_stiffness for the 20-node serendipity element: its
    integrand is also of degree at most 4 in each coordinate, so 3 Gauss
    points per axis and subcell are exact."""
    D = elasticity_D(nu)
    gp, gw = nleg.leggauss(3)
    jac = (h / 2.0) ** 3
    half = 1.0 / n
    out = np.zeros((n ** 3, 81, 81))
    for c in range(n):
        for b in range(n):
            for a in range(n):
                cx = -1.0 + (2 * a + 1) / n
                cy = -1.0 + (2 * b + 1) / n
                cz = -1.0 + (2 * c + 1) / n
                Ki = np.zeros((81, 81))
                for qz in range(3):
                    for qy in range(3):
                        for qx in range(3):
                            wq = gw[qx] * gw[qy] * gw[qz] * half ** 3
                            _, dN = serendipity2_shape(cx + half * gp[qx], cy + half * gp[qy],
                                                       cz + half * gp[qz], h)
                            B = strain_displacement(dN)
                            Ki += wq * jac * (B.T @ D @ B)
                out[a + n * (b + n * c)] = Ki
    return out


@functools.lru_cache(maxsize=8)
def _subcell_stiffness_s3(n: int, nu: float, h: float) -> np.ndarray:
    """The 32-node cubic serendipity element: its shape functions have degree
    at most 3 in each coordinate, so 4 Gauss points per axis and subcell are
    exact for the integrand (degree <= 6 per axis)."""
    D = elasticity_D(nu)
    gp, gw = nleg.leggauss(4)
    jac = (h / 2.0) ** 3
    half = 1.0 / n
    out = np.zeros((n ** 3, 192, 192))
    for c in range(n):
        for b in range(n):
            for a in range(n):
                cx, cy, cz = -1.0 + (2 * a + 1) / n, -1.0 + (2 * b + 1) / n, -1.0 + (2 * c + 1) / n
                Ki = np.zeros((192, 192))
                for qz in range(4):
                    for qy in range(4):
                        for qx in range(4):
                            wq = gw[qx] * gw[qy] * gw[qz] * half ** 3
                            _, dN = serendipity3_shape(cx + half * gp[qx], cy + half * gp[qy],
                                                       cz + half * gp[qz], h)
                            B = strain_displacement(dN)
                            Ki += wq * jac * (B.T @ D @ B)
                out[a + n * (b + n * c)] = Ki
    return out


@functools.lru_cache(maxsize=32)
def _subcell_stiffness(k: int, n: int, nu: float, h: float) -> np.ndarray:
    """The stacked subcell stiffness table of Eq. matrixK_mr.

    K[i] = int over subcell i of B^T D B dx (E = 1), for the n^3 subcells of a
    degree-k Lagrange cube of edge h.  Each subcell is integrated with its own
    tensor Gauss-Legendre rule of k+1 points per axis, which is exact: the
    integrand is a polynomial of degree at most 2k in each coordinate.
    Returns an array (n^3, d, d), d = 3 (k+1)^3.
    """
    D = elasticity_D(nu)
    d = 3 * (k + 1) ** 3
    gp, gw = nleg.leggauss(k + 1)
    jac = (h / 2.0) ** 3  # dx dy dz = (h/2)^3 dxi deta dzeta
    half = 1.0 / n  # half-width of a subinterval in xi
    out = np.zeros((n ** 3, d, d))
    for c in range(n):
        for b in range(n):
            for a in range(n):
                i = a + n * (b + n * c)
                cx = -1.0 + (2 * a + 1) / n
                cy = -1.0 + (2 * b + 1) / n
                cz = -1.0 + (2 * c + 1) / n
                Ki = np.zeros((d, d))
                for qz in range(k + 1):
                    for qy in range(k + 1):
                        for qx in range(k + 1):
                            xi = cx + half * gp[qx]
                            eta = cy + half * gp[qy]
                            zeta = cz + half * gp[qz]
                            wq = gw[qx] * gw[qy] * gw[qz] * half ** 3
                            _, dN = shape_3d(k, xi, eta, zeta, h)
                            B = strain_displacement(dN)
                            Ki += wq * jac * (B.T @ D @ B)
                out[i] = Ki
    return out


def element_stiffness(k: int, nu: float, h: float = 1.0) -> np.ndarray:
    """Whole-element matrix int_{Omega_e} B^T D B (Eq. matrixK with E = 1)."""
    return subcell_stiffness(k, 1, nu, h)[0]


def rigid_body_modes(k: int, h: float = 1.0) -> np.ndarray:
    """The six rigid-body displacement fields of one element, (6, d):
    three translations and three infinitesimal rotations about the centre."""
    nodes = np.linspace(-1.0, 1.0, k + 1) * (h / 2.0)
    nn = (k + 1) ** 3
    R = np.zeros((6, 3 * nn))
    for iz in range(k + 1):
        for iy in range(k + 1):
            for ix in range(k + 1):
                a = ix + (k + 1) * (iy + (k + 1) * iz)
                x, y, z = nodes[ix], nodes[iy], nodes[iz]
                R[0, 3 * a + 0] = 1.0
                R[1, 3 * a + 1] = 1.0
                R[2, 3 * a + 2] = 1.0
                # rotation about z: (-y, x, 0); about x: (0, -z, y); about y: (z, 0, -x)
                R[3, 3 * a: 3 * a + 3] = (-y, x, 0.0)
                R[4, 3 * a: 3 * a + 3] = (0.0, -z, y)
                R[5, 3 * a: 3 * a + 3] = (z, 0.0, -x)
    return R
