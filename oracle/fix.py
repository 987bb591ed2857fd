"""Fixing design variables and suppressing displacement DOFs (oracle).

Section 6.1.  With the thresholds rho_fix^l, rho_fix^u and eps_grad:
  * a displacement element is void when every density cell inside it has
    rho <= rho_fix^l and every design variable inside it has a gradient
    component >= -eps_grad; it is solid when every density is >= rho_fix^u
    and every such gradient component is <= eps_grad;
  * only elements surrounded by elements of their own kind are fixed;
  * the design variables of fixed elements stay where they are (the LP gets
    zero bounds for them) and the gradient components of fixed void
    elements are set to 0;
  * the displacements of the nodes of fixed void elements are suppressed:
    their rows and columns leave K, their loads leave f, and u = 0 there,
    like a support; the multigrid setup is redone afterwards.

Readings (the section does not fix them):
  * "surrounded" = every element that shares at least one node with it, the
    26 neighbours, counting only those inside the domain;
  * a node is suppressed when every element that contains it is a fixed void
    element (this covers the nodes interior to one element, and keeps the
    nodes on the border of the fixed void region, whose stiffness entries
    are of order Emin);
  * without a gradient (grad = None) only the density conditions apply.

Test infrastructure only: nothing on the product path imports this module.
"""
from __future__ import annotations

import numpy as np

VOID, SOLID = 1, 2


def _cells_of_elements(nx: int, ny: int, nz: int, n: int) -> np.ndarray:
    """(E, n^3): indices (x fastest) of the n^3 cells inside each element."""
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ex, ey, ez = ex.reshape(-1, 1), ey.reshape(-1, 1), ez.reshape(-1, 1)
    c, b, a = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    a, b, c = a.reshape(1, -1), b.reshape(1, -1), c.reshape(1, -1)
    Dx, Dy = n * nx, n * ny
    return (n * ex + a) + Dx * ((n * ey + b) + Dy * (n * ez + c))


def element_class(prob, rho: np.ndarray, grad: np.ndarray | None, rho_lo: float, rho_hi: float,
                  eps_grad: float) -> np.ndarray:
    """Per element (x fastest): VOID, SOLID or 0 (Sec. 6.1, the two sets of
    conditions).  rho lives on the density grid (n_mr per element edge),
    grad on the design grid (d_mr per element edge)."""
    n = prob.n_mr
    d = getattr(prob, "d_mr", None) or n
    r = rho[_cells_of_elements(prob.nx, prob.ny, prob.nz, n)]
    void = (r <= rho_lo).all(axis=1)
    solid = (r >= rho_hi).all(axis=1)
    if grad is not None:
        g = grad[_cells_of_elements(prob.nx, prob.ny, prob.nz, d)]
        void &= (g >= -eps_grad).all(axis=1)
        solid &= (g <= eps_grad).all(axis=1)
    out = np.zeros(prob.nx * prob.ny * prob.nz, dtype=np.int8)
    out[void] = VOID
    out[solid & ~void] = SOLID
    return out


def fixed_elements(prob, cls: np.ndarray) -> np.ndarray:
    """Per element: its class if every neighbour sharing a node with it
    (inside the domain) has the same class, else 0."""
    nx, ny, nz = prob.nx, prob.ny, prob.nz
    c = cls.reshape(nz, ny, nx)
    out = np.zeros_like(c)
    for ez in range(nz):
        for ey in range(ny):
            for ex in range(nx):
                k = c[ez, ey, ex]
                if k == 0:
                    continue
                nb = c[max(ez - 1, 0):ez + 2, max(ey - 1, 0):ey + 2, max(ex - 1, 0):ex + 2]
                if (nb == k).all():
                    out[ez, ey, ex] = k
    return out.reshape(-1)


def fixed_design_variables(prob, fixed: np.ndarray) -> np.ndarray:
    """Per design variable: the class of the fixed element containing it."""
    d = getattr(prob, "d_mr", None) or prob.n_mr
    cells = _cells_of_elements(prob.nx, prob.ny, prob.nz, d)
    out = np.zeros(cells.size, dtype=np.int8)
    out[cells] = fixed[:, None]
    return out


def suppressed_nodes(prob, fixed: np.ndarray) -> np.ndarray:
    """Per lattice node: True when every element containing it is a fixed
    void element."""
    k = prob.degree
    Lx, Ly, Lz = prob.lattice
    f = fixed.reshape(prob.nz, prob.ny, prob.nx) == VOID
    out = np.zeros(Lx * Ly * Lz, dtype=bool)
    for l in range(Lz):
        for j in range(Ly):
            for i in range(Lx):
                rng = []
                for c, e in ((i, prob.nx), (j, prob.ny), (l, prob.nz)):
                    lo = (c - 1) // k if c % k == 0 else c // k
                    hi = c // k
                    rng.append(range(max(lo, 0), min(hi, e - 1) + 1))
                out[i + Lx * (j + Ly * l)] = all(f[ez, ey, ex] for ez in rng[2] for ey in rng[1]
                                                 for ex in rng[0])
    return out


def suppressed_problem(prob, sup_nodes: np.ndarray):
    """A copy of prob whose supports also hold the suppressed nodes' DOFs
    (Sec. 6.1: u = 0 there, rows and columns removed, loads ignored)."""
    q = prob.__class__(**{k: getattr(prob, k) for k in prob.__dataclass_fields__})
    q.mask = (np.asarray(prob.mask) != 0) | np.repeat(sup_nodes, 3)
    q.mask = q.mask.astype(np.uint8)
    return q


def zero_fixed_void_gradient(grad: np.ndarray, fixed_x: np.ndarray) -> np.ndarray:
    """The gradient with the components of fixed void design variables set
    to 0 (Sec. 6.1)."""
    g = np.array(grad, dtype=np.float64)
    g[fixed_x == VOID] = 0.0
    return g
