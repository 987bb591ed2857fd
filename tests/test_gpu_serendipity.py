"""The 20-node serendipity element on the GPU (family = 1, Sec. 2.1)
against the oracle (oracle/fem.py, oracle/fe.py).

* The subcell table to FP64 rounding (1e-14 of its largest entry).
* The level-0 FP64 operator, with the face and element-centre nodes held
  at 0, to 1e-13.
* Solve (rtol 1e-11) to displacement 1e-6, compliance 1e-7, gradient 1e-6,
  for every preconditioner precision: the coarse levels are degree-2
  serendipity meshes re-discretised through the element's moment basis,
  with shape-function transfers (nested spaces: the coarse operators are
  the Galerkin products); the converged solution does not depend on it.
* Level 1 against the oracle's serendipity operator on the coarse mesh.
* Descriptor errors.
"""
import numpy as np
import pytest

import workloads
from oracle import fe, fem
from tests.gpu_helpers import Run, desc_for, lib, rel

pytestmark = pytest.mark.gpu

FP64, FP32, FP32X2 = 0, 1, 3


def _s2(shape=(8, 4, 4), n=2, seed=5, levels=2, rmin=0.0):
    p = workloads.cantilever(*shape, degree=2, n_mr=n, rmin=rmin, seed=seed, mg_levels=levels)
    return workloads.with_serendipity(p)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_subcell_table(n):
    import torch

    q = _s2(n=n, levels=1, shape=(2, 2, 2))
    R = Run(q, FP64)
    tab = torch.zeros((n ** 3, 81, 81), dtype=torch.float64, device=R.dev)
    with torch.cuda.stream(R.stream):
        R.T.tosolve_subcell_table(R.h, tab)
    R.stream.synchronize()
    ref = fem.subcell_stiffness(2, n, 0.3, family="serendipity")
    assert np.abs(tab.cpu().numpy() - ref).max() <= 1e-14 * np.abs(ref).max()
    R.close()


def test_operator_and_unknowns():
    q = _s2(rmin=1.0)
    m = fe.Model(q)
    w = m.weights(m.densities(q.x))
    R = Run(q, FP32X2)
    R.set_densities()
    x = np.random.default_rng(1).normal(size=q.ndof)
    assert rel(R.apply(0, FP64, x), m.apply(w, x)) <= 1e-13
    assert R.T.tosolve_free_dofs(R.h) == q.nfree
    absent = np.repeat(workloads.serendipity_absent_nodes(q), 3)
    assert q.nfree == q.ndof - int((np.asarray(q.mask) != 0).sum()) and absent.sum() > 0
    R.close()


def test_coarse_level_is_the_serendipity_mesh_of_the_coarse_elements():
    """Level 1 is re-discretised through the serendipity moment basis: it
    must equal the oracle's serendipity operator on the 2x coarser mesh whose
    elements hold (2n)^3 density cells (the same density field)."""
    q = _s2(shape=(8, 4, 4), n=2, levels=3, rmin=1.0)
    qc = workloads.with_serendipity(workloads.cantilever(4, 2, 2, degree=2, n_mr=4, rmin=0.0, seed=5))
    m = fe.Model(q)
    rho = m.densities(q.x)
    qc.x = rho  # the coarse elements see the filtered densities of the fine grid
    mc = fe.Model(qc)
    R = Run(q, FP64)
    R.set_densities()
    x = np.random.default_rng(2).normal(size=qc.ndof)
    # level 1 has element edge 2: a 3D stiffness scales with the edge (B ~ 1/h, dV ~ h^3)
    ref = 2.0 * mc.apply(mc.weights(qc.x), x)
    held = np.asarray(qc.mask) != 0
    ref[held] = x[held]
    assert rel(R.apply(1, FP64, x), ref) <= 1e-13
    R.close()


def test_one_cycle_matches_algorithm_1():
    """One V-cycle (omega = 0.3, serendipity levels, shape-function
    transfers) against the oracle's Algorithm 1 on the same hierarchy."""
    from oracle import mg

    q = _s2(shape=(8, 4, 4), n=2, levels=3, rmin=1.0)
    m = fe.Model(q)
    h = mg.Hierarchy(q, m.densities(q.x), 3)
    b = np.where(q.mask == 0, np.random.default_rng(4).normal(size=q.ndof), 0.0)
    R = Run(q, FP64)
    R.set_densities()
    assert rel(R.precondition(b), mg.vcycle(h, b)) <= 1e-9
    R.close()


@pytest.mark.parametrize("precision", [FP64, FP32, FP32X2])
def test_solve_matches_oracle(precision):
    q = _s2(shape=(8, 4, 4), n=2, levels=3)
    ref = fe.Model(q).run(method="splu")
    R = Run(q, precision)
    R.set_densities()
    u, info = R.solve(rtol=1e-11)
    assert info.rel_residual <= 1e-11
    un = u.cpu().numpy()[0]
    assert rel(un, ref["u"][0]) <= 1e-6
    absent = np.repeat(workloads.serendipity_absent_nodes(q), 3)
    assert np.all(un[absent] == 0.0)
    c, gx, gr = R.grad(u)
    assert abs(c[0] - ref["c"][0]) <= 1e-7 * abs(ref["c"][0])
    assert rel(gr, ref["g_rho"]) <= 1e-6
    assert rel(gx, ref["g_x"]) <= 1e-6
    R.close()


def test_descriptor_errors():
    T = lib()
    p1 = workloads.cantilever(4, 2, 2, degree=1, seed=0)
    d = desc_for(T, p1, FP64)
    d.family = 1
    with pytest.raises(T.TosolveError):
        T.tosolve_create(d, p1.mask)
    q = _s2(shape=(4, 2, 2), levels=1)
    d = desc_for(T, q, FP64)
    d.family = 2
    with pytest.raises(T.TosolveError):
        T.tosolve_create(d, q.mask)
    d.family = 1
    with pytest.raises(T.TosolveError):
        T.tosolve_create_mixed(d, q.mask, np.zeros(q.nx * q.ny * q.nz, dtype=np.uint8))
