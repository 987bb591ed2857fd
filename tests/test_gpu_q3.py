"""Degree 3 on the GPU (Lagrange, and the 32-node serendipity element)
against the oracle.  The finest level is the cubic mesh; the next level is
the degree-2 mesh of the same family on the same elements, reached by the
quadratic shape functions at the cubic nodes (the oracle pins that its
re-discretised operator is the Galerkin product); the degree-2 hierarchy
follows.

* The subcell table to FP64 rounding (1e-14 of its largest entry).
* The level-0 operator to 1e-13.
* One V-cycle against the oracle's Algorithm 1 on the same hierarchy (to
  1e-7: the cubic-to-quadratic weights are held in FP32).
* Solve (rtol 1e-11) to displacement 1e-6, compliance 1e-7, gradient 1e-6.
* A cubic descriptor with a single level is refused.
"""
import numpy as np
import pytest

import workloads
from oracle import fe, fem, mg
from tests.gpu_helpers import Run, desc_for, lib, rel

pytestmark = pytest.mark.gpu

FP64, FP32, FP32X2 = 0, 1, 3


def _q3(family, shape=(4, 2, 2), n=2, levels=2, rmin=0.0, seed=3):
    p = workloads.cantilever(*shape, degree=3, n_mr=n, rmin=rmin, seed=seed, mg_levels=levels)
    return workloads.with_serendipity(p) if family == "serendipity" else p


@pytest.mark.parametrize("family", ["lagrange", "serendipity"])
def test_subcell_table(family):
    import torch

    p = _q3(family, n=2)
    R = Run(p, FP64)
    tab = torch.zeros((8, 192, 192), dtype=torch.float64, device=R.dev)
    with torch.cuda.stream(R.stream):
        R.T.tosolve_subcell_table(R.h, tab)
    R.stream.synchronize()
    ref = fem.subcell_stiffness(3, 2, 0.3, family=family)
    assert np.abs(tab.cpu().numpy() - ref).max() <= 1e-14 * np.abs(ref).max()
    R.close()


@pytest.mark.parametrize("family", ["lagrange", "serendipity"])
def test_operator_and_one_cycle(family):
    p = _q3(family, shape=(4, 2, 2), n=2, levels=3 if family == "lagrange" else 2, rmin=1.0)
    m = fe.Model(p)
    rho = m.densities(p.x)
    R = Run(p, FP64)
    R.set_densities()
    x = np.random.default_rng(1).normal(size=p.ndof)
    assert rel(R.apply(0, FP64, x), m.apply(m.weights(rho), x)) <= 1e-13
    assert R.T.tosolve_free_dofs(R.h) == p.nfree
    h = mg.Hierarchy(p, rho, R.T.tosolve_level_count(R.h))
    b = np.where(p.mask == 0, np.random.default_rng(2).normal(size=p.ndof), 0.0)
    # the degree-3 -> 2 transfer weights (values of quadratic shape functions
    # at the third points, such as 2/9) are stored in FP32 and are not exact
    # there (the degree-2 weights at the quarter points are dyadic): 1e-7
    assert rel(R.precondition(b), mg.vcycle(h, b)) <= 1e-7
    R.close()


@pytest.mark.parametrize("family", ["lagrange", "serendipity"])
@pytest.mark.parametrize("precision", [FP64, FP32, FP32X2])
def test_solve_matches_oracle(family, precision):
    p = _q3(family, shape=(4, 2, 2), n=2, levels=2, seed=5)
    ref = fe.Model(p).run(method="splu")
    R = Run(p, precision)
    R.set_densities()
    u, info = R.solve(rtol=1e-11)
    assert info.rel_residual <= 1e-11
    assert rel(u.cpu().numpy()[0], ref["u"][0]) <= 1e-6
    c, gx, gr = R.grad(u)
    assert abs(c[0] - ref["c"][0]) <= 1e-7 * abs(ref["c"][0])
    assert rel(gr, ref["g_rho"]) <= 1e-6
    assert rel(gx, ref["g_x"]) <= 1e-6
    R.close()


def test_single_level_is_refused():
    T = lib()
    p = _q3("lagrange", levels=1)
    with pytest.raises(T.TosolveError):
        T.tosolve_create(desc_for(T, p, FP64), p.mask)
