"""Seeded synthetic problems for the elasticity solve.

This module is shared by the CPU oracle tests, the CUDA parity tests and the
benchmark.  It holds none of the method's arithmetic: it only builds, from a
seed, the inputs a caller hands to the solver -- the Dirichlet mask per DOF,
the nodal load vectors and the design-variable field.

Conventions (the same ones the C ABI documents):
  * displacement mesh of nx*ny*nz cubic elements of edge 1 (the paper's
    problems use unit elements, Section 7.1);
  * Lagrange degree k gives a node lattice of (k*nx+1, k*ny+1, k*nz+1) nodes,
    node id = i + Lx*(j + Ly*l) (x fastest), DOF = 3*node + component;
  * the design / density grid has n_mr cells per element edge, flattened
    x fastest: cell id = cx + Dx*(cy + Dy*cz) with Dx = n_mr*nx, ...;
  * mask[dof] = 1 marks a fixed (Dirichlet) DOF.

The load patterns stand in for the paper's test structures (Section 7.1):
the cantilever (left face clamped, downward load on the bottom edge of the
right face) and the bridge (corner supports, distributed top load).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

__all__ = [
    "Problem",
    "lattice_shape",
    "cantilever",
    "bridge",
    "batched_instances",
    "uniform_field",
    "smooth_field",
]

# Newton-Cotes weights: the integral of each equispaced 1D Lagrange basis
# function of degree k over one unit element edge.  A uniform line (or face)
# load of unit intensity becomes these nodal forces per element.
_NEWTON_COTES = {
    1: np.array([1.0, 1.0]) / 2.0,
    2: np.array([1.0, 4.0, 1.0]) / 6.0,
    3: np.array([1.0, 3.0, 3.0, 1.0]) / 8.0,
}


def lattice_shape(nx: int, ny: int, nz: int, k: int) -> tuple[int, int, int]:
    """Node lattice extents (Lx, Ly, Lz) for Lagrange degree k."""
    return (k * nx + 1, k * ny + 1, k * nz + 1)


@dataclass
class Problem:
    """One solve request: mesh, material, boundary conditions, loads, design."""

    name: str
    nx: int
    ny: int
    nz: int
    degree: int
    n_mr: int
    rmin: float
    E0: float
    Emin: float
    nu: float
    penal: float
    mask: np.ndarray  # uint8 (3*nnodes,), 1 = Dirichlet
    f: np.ndarray  # float64 (nrhs, 3*nnodes)
    x: np.ndarray  # float64 (n_mr^3 * nx*ny*nz,), design variables
    mg_levels: int
    meta: dict = field(default_factory=dict)
    # mixed degree (degree-2 lattice): uint8 per element, 1 = trilinear
    elem_q1: np.ndarray | None = None
    # design cells per element edge (None: the density grid, d_mr = n_mr)
    d_mr: int | None = None
    # element family: "lagrange", or "serendipity" (degree 2: the 20-node
    # element on the degree-2 lattice, no nodes at face and cell centres)
    family: str = "lagrange"

    @property
    def lattice(self) -> tuple[int, int, int]:
        return lattice_shape(self.nx, self.ny, self.nz, self.degree)

    @property
    def nnodes(self) -> int:
        Lx, Ly, Lz = self.lattice
        return Lx * Ly * Lz

    @property
    def ndof(self) -> int:
        return 3 * self.nnodes

    @property
    def nfree(self) -> int:
        return int(self.ndof - int(self.mask.sum()))

    @property
    def nrhs(self) -> int:
        return int(self.f.shape[0])

    @property
    def density_shape(self) -> tuple[int, int, int]:
        """(Dz, Dy, Dx) of the density / design grid."""
        n = self.n_mr
        return (n * self.nz, n * self.ny, n * self.nx)


def uniform_field(shape, lo: float, hi: float, rng: np.random.Generator) -> np.ndarray:
    """iid U[lo, hi] values on a (Dz, Dy, Dx) grid, flattened x fastest."""
    return rng.uniform(lo, hi, size=shape).astype(np.float64).reshape(-1)


def _upsample_axis(a: np.ndarray, axis: int, n_out: int) -> np.ndarray:
    """Linear resampling along one axis, cell-centred (half-pixel) convention,
    clamped at the edges -- the usual 'align_corners=False' image resize."""
    n_in = a.shape[axis]
    dst = np.arange(n_out, dtype=np.float64)
    src = (dst + 0.5) * (n_in / n_out) - 0.5
    src = np.clip(src, 0.0, n_in - 1)
    i0 = np.floor(src).astype(np.int64)
    i1 = np.minimum(i0 + 1, n_in - 1)
    t = src - i0
    a0 = np.take(a, i0, axis=axis)
    a1 = np.take(a, i1, axis=axis)
    shp = [1] * a.ndim
    shp[axis] = n_out
    t = t.reshape(shp)
    return a0 * (1.0 - t) + a1 * t


def smooth_field(shape, rng: np.random.Generator, coarse=(6, 6, 12), lo: float = 0.001,
                 hi: float = 1.0) -> np.ndarray:
    """Smooth random design field: iid U[0,1] values at the centres of a
    coarse (cz, cy, cx) grid, trilinearly resampled to the (Dz, Dy, Dx) cell
    centres, clipped to [lo, hi].  Flattened x fastest."""
    c = rng.uniform(0.0, 1.0, size=coarse)
    for axis, n_out in enumerate(shape):
        c = _upsample_axis(c, axis, n_out)
    return np.clip(c, lo, hi).reshape(-1).astype(np.float64)


def _node(i, j, l, lat):
    Lx, Ly, _ = lat
    return i + Lx * (j + Ly * l)


def _line_weights(n_elems: int, k: int) -> np.ndarray:
    """Consistent nodal weights of a unit-intensity uniform load on a line of
    n_elems unit elements of degree k (k*n_elems+1 nodes)."""
    w = np.zeros(k * n_elems + 1)
    nc = _NEWTON_COTES[k]
    for e in range(n_elems):
        w[k * e: k * e + k + 1] += nc
    return w


def ibeam_field(shape) -> np.ndarray:
    """(Dz, Dy, Dx) cells, flattened x fastest: 1 in the bottom and top
    flanges (Dz/8 cells thick each, rounded up) and in the web (Dy/8 cells
    wide, centred), 0 elsewhere."""
    Dz, Dy, Dx = shape
    t = max(1, -(-Dz // 8))
    wy = max(1, -(-Dy // 8))
    y0 = (Dy - wy) // 2
    z = np.arange(Dz)[:, None, None]
    y = np.arange(Dy)[None, :, None]
    solid = (z < t) | (z >= Dz - t) | ((y >= y0) & (y < y0 + wy))
    return np.broadcast_to(solid, (Dz, Dy, Dx)).astype(np.float64).reshape(-1)


def cantilever(nx: int, ny: int, nz: int, *, degree: int = 1, n_mr: int = 1,
               rmin: float = 0.0, density: str = "uniform", seed: int = 0,
               E0: float = 1.0, Emin: float = 1e-9, nu: float = 0.3,
               penal: float = 3.0, mg_levels: int = 0, lo: float = 0.01,
               hi: float = 1.0) -> Problem:
    """3D cantilever: face x=0 clamped (all DOFs of its nodes); a unit total
    downward (-z) load spread uniformly along the edge x=nx, z=0 with
    consistent nodal weights.

    density='uniform': design variables iid U[lo, hi];
    density='smooth' : smooth_field (coarse 12x6x6 iid U[0,1], trilinear
                       resampling, clipped to [0.001, 1]);
    density='ibeam'  : a 0/1 design with large void regions, the kind an
                       optimisation ends with (Sec. 6.1 fixes variables in
                       such regions): an I-beam along x, flanges of an
                       eighth of the height at the bottom and top, a web of
                       an eighth of the width in the middle, x = 0 elsewhere.
    """
    lat = lattice_shape(nx, ny, nz, degree)
    Lx, Ly, Lz = lat
    nn = Lx * Ly * Lz
    mask = np.zeros(3 * nn, dtype=np.uint8)
    for l in range(Lz):
        for j in range(Ly):
            nd = _node(0, j, l, lat)
            mask[3 * nd: 3 * nd + 3] = 1
    f = np.zeros((1, 3 * nn))
    wl = _line_weights(ny, degree) / ny  # total load 1
    for j in range(Ly):
        nd = _node(Lx - 1, j, 0, lat)
        f[0, 3 * nd + 2] -= wl[j]
    rng = np.random.default_rng(seed)
    shape = (n_mr * nz, n_mr * ny, n_mr * nx)
    if density == "uniform":
        x = uniform_field(shape, lo, hi, rng)
    elif density == "smooth":
        x = smooth_field(shape, rng)
    elif density == "solid":
        x = np.ones(int(np.prod(shape)))
    elif density == "ibeam":
        x = ibeam_field(shape)
    else:
        raise ValueError(density)
    return Problem(f"cantilever{nx}x{ny}x{nz}_k{degree}_n{n_mr}", nx, ny, nz, degree,
                   n_mr, float(rmin), E0, Emin, nu, penal, mask, f, x, mg_levels,
                   meta={"seed": seed, "density": density})


def bridge(nx: int, ny: int, nz: int, *, degree: int = 1, n_mr: int = 1,
           rmin: float = 0.0, seed: int = 0, E0: float = 1.0, Emin: float = 1e-9,
           nu: float = 0.3, penal: float = 3.0, mg_levels: int = 0,
           lo: float = 0.01, hi: float = 1.0) -> Problem:
    """Bridge stand-in: the four bottom-corner nodes pinned (all DOFs), a
    uniform downward pressure of 1 per unit area on the top face z=nz with
    consistent (tensor Newton-Cotes) nodal weights; design variables iid
    U[lo, hi]."""
    lat = lattice_shape(nx, ny, nz, degree)
    Lx, Ly, Lz = lat
    nn = Lx * Ly * Lz
    mask = np.zeros(3 * nn, dtype=np.uint8)
    for i in (0, Lx - 1):
        for j in (0, Ly - 1):
            nd = _node(i, j, 0, lat)
            mask[3 * nd: 3 * nd + 3] = 1
    f = np.zeros((1, 3 * nn))
    wx = _line_weights(nx, degree)
    wy = _line_weights(ny, degree)
    for j in range(Ly):
        for i in range(Lx):
            nd = _node(i, j, Lz - 1, lat)
            f[0, 3 * nd + 2] -= wx[i] * wy[j]
    rng = np.random.default_rng(seed)
    shape = (n_mr * nz, n_mr * ny, n_mr * nx)
    x = uniform_field(shape, lo, hi, rng)
    return Problem(f"bridge{nx}x{ny}x{nz}_k{degree}_n{n_mr}", nx, ny, nz, degree, n_mr,
                   float(rmin), E0, Emin, nu, penal, mask, f, x, mg_levels,
                   meta={"seed": seed})


def batched_instances(count: int, seed: int, *, min_nx: int = 32, max_nx: int = 128,
                      mult: int = 8, max_rhs: int = 3, Emin: float = 1e-9,
                      nu: float = 0.3, penal: float = 3.0, mg_levels: int = 0) -> list[Problem]:
    """Uneven batch of Q1 cantilever-type instances: nx log-uniform in
    [min_nx, max_nx] rounded to a multiple of `mult`, ny = nz = nx/2; face
    x=0 clamped; 1..max_rhs load cases, each a unit total load spread
    uniformly along a random edge of the face x=nx in a random unit
    direction; design variables iid U[0.01, 1]."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        nx = float(np.exp(rng.uniform(np.log(min_nx), np.log(max_nx))))
        nx = int(max(mult, round(nx / mult) * mult))
        ny = nz = nx // 2
        p = cantilever(nx, ny, nz, degree=1, n_mr=1, density="uniform",
                       seed=int(rng.integers(1 << 31)), Emin=Emin, nu=nu,
                       penal=penal, mg_levels=mg_levels)
        lat = p.lattice
        Lx, Ly, Lz = lat
        nrhs = int(rng.integers(1, max_rhs + 1))
        f = np.zeros((nrhs, p.ndof))
        for r in range(nrhs):
            edge = int(rng.integers(4))
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            if edge in (0, 1):  # along y at z = 0 or z = nz
                l = 0 if edge == 0 else Lz - 1
                wl = _line_weights(ny, 1) / ny
                nodes = [_node(Lx - 1, j, l, lat) for j in range(Ly)]
            else:  # along z at y = 0 or y = ny
                j = 0 if edge == 2 else Ly - 1
                wl = _line_weights(nz, 1) / nz
                nodes = [_node(Lx - 1, j, l, lat) for l in range(Lz)]
            for wgt, nd in zip(wl, nodes):
                f[r, 3 * nd: 3 * nd + 3] += wgt * d
        p.f = f
        p.name = f"batch{b}_{nx}x{ny}x{nz}_rhs{nrhs}"
        out.append(p)
    return out


def serendipity_absent_nodes(p: Problem) -> np.ndarray:
    """(nnodes,) bool: the nodes of the degree-k lattice (k = 2, 3) that no
    serendipity element has: those with two or three coordinates inside an
    element edge (not a multiple of k) -- face and element interiors."""
    k = p.degree
    Lx, Ly, Lz = p.lattice
    n = np.arange(Lx * Ly * Lz)
    i, j, l = n % Lx, (n // Lx) % Ly, n // (Lx * Ly)
    return (i % k != 0).astype(int) + (j % k != 0) + (l % k != 0) >= 2


def with_serendipity(p: Problem) -> Problem:
    """The same problem with serendipity elements (20 nodes for degree 2, 32
    for degree 3) on its lattice: the lattice nodes the element does not
    have are held at 0 with the supports (they carry no unknown).  Loads
    there must be zero."""
    if p.degree not in (2, 3):
        raise ValueError("the serendipity element is built for degree 2 and 3")
    q = Problem(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    absent = serendipity_absent_nodes(p)
    if np.any(np.asarray(p.f)[:, np.repeat(absent, 3)] != 0.0):
        raise ValueError("loads on nodes the serendipity element does not have")
    q.mask = (np.asarray(p.mask) != 0) | np.repeat(absent, 3)
    q.mask = q.mask.astype(np.uint8)
    q.family = "serendipity"
    q.name = p.name.replace(f"_k{p.degree}", f"_s{p.degree}")
    return q


def with_mixed_degree(p: Problem, q1_fraction: float, seed: int) -> Problem:
    """The same problem on its degree-2 lattice with a random q1_fraction of
    the elements trilinear (iid per element, seeded)."""
    if p.degree != 2:
        raise ValueError("mixed degree needs the degree-2 lattice")
    rng = np.random.default_rng(seed)
    E = p.nx * p.ny * p.nz
    q = p.__class__(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.elem_q1 = (rng.random(E) < q1_fraction).astype(np.uint8)
    q.name = p.name + f"_mixed{q1_fraction:g}"
    q.meta = dict(p.meta, q1_fraction=q1_fraction, degree_seed=seed)
    return q


def with_design_grid(p: Problem, d_mr: int, seed: int, lo: float = 0.01, hi: float = 1.0) -> Problem:
    """The same problem with a coarser design grid (d_mr design cells per
    element edge) and new design variables iid U[lo, hi] on it."""
    if not 1 <= d_mr <= p.n_mr:
        raise ValueError("need 1 <= d_mr <= n_mr")
    rng = np.random.default_rng(seed)
    q = p.__class__(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.d_mr = d_mr
    q.x = uniform_field((d_mr * p.nz, d_mr * p.ny, d_mr * p.nx), lo, hi, rng)
    q.name = p.name + f"_d{d_mr}"
    return q
