"""Chebyshev smoothing on the GPU (desc.smoother = 1) against the oracle's
Chebyshev cycle (oracle/mg.py): lambda_max(D^-1 A) of every level by eight
Lanczos steps from the Weyl start vector, then Saad's Chebyshev iteration on
D^-1 A over [0.3 b, b], b = 1.1 lambda, two steps before and after the
coarse correction.

* The Lanczos estimate of every smoothed level: FP64 handles to 1e-9
  (the same FP64 recurrences in other summation orders), FP32 handles to
  1e-4 (FP32 vectors and operators, FP64 reductions).
* One V-cycle against Algorithm 1 with Chebyshev smoothing: FP64 to 1e-9
  (1e-7 at degree 3, whose degree-3 -> 2 transfer weights are stored in
  FP32, as for the Jacobi cycle), FP32 to 1e-4 (the estimate's FP32 error
  moves the polynomial).
* Solves reach the direct solution (displacement 1e-6, compliance 1e-7,
  gradient 1e-6) in fewer PCG iterations than with damped Jacobi, for
  Lagrange and serendipity elements of degree 2 and 3, and with the
  tensor-core level 0 (F16X3, with and without inner FP32 iterations).
* Descriptor errors: degree 1 and FP32X2 are rejected.
"""
import numpy as np
import pytest

import workloads
from oracle import fe, mg
from tests.gpu_helpers import Run, desc_for, lib, rel

pytestmark = pytest.mark.gpu

FP64, FP32, FP32X2, F16X3 = 0, 1, 3, 6
CHEB = dict(smoother=1, cheb_degree=2)
CASES = [(2, "lagrange"), (2, "serendipity"), (3, "lagrange"), (3, "serendipity")]


def _prob(deg, family, shape=(8, 4, 4), seed=7):
    levels = 2 if deg == 2 else 3
    p = workloads.cantilever(*shape, degree=deg, n_mr=2, rmin=1.0, seed=seed, mg_levels=levels)
    return workloads.with_serendipity(p) if family == "serendipity" else p


def _hier(p):
    m = fe.Model(p)
    return mg.Hierarchy(p, m.densities(p.x), p.mg_levels, smoother="chebyshev", cheb_degree=2, lanczos_steps=8)


@pytest.mark.parametrize("deg,family", CASES)
@pytest.mark.parametrize("precision,tol", [(FP64, 1e-9), (FP32, 1e-4)])
def test_lanczos_estimates_match_the_oracle(deg, family, precision, tol):
    p = _prob(deg, family)
    h = _hier(p)
    R = Run(p, precision, **CHEB)
    R.set_densities()
    for l in range(len(h.levels) - 1):
        lam = R.T.tosolve_smoother_lmax(R.h, l)
        assert abs(lam - h.levels[l].lmax) <= tol * h.levels[l].lmax, (l, lam, h.levels[l].lmax)
    R.close()


@pytest.mark.parametrize("deg,family", CASES)
@pytest.mark.parametrize("precision,tol", [(FP64, 1e-9), (FP32, 1e-4)])
def test_one_chebyshev_cycle_matches_algorithm_1(deg, family, precision, tol):
    p = _prob(deg, family)
    h = _hier(p)
    b = np.where(np.asarray(p.mask) == 0, np.random.default_rng(4).normal(size=p.ndof), 0.0)
    R = Run(p, precision, **CHEB)
    R.set_densities()
    if deg == 3:  # FP32 storage of the non-dyadic degree-3 -> 2 transfer weights
        tol = max(tol, 1e-7)
    assert rel(R.precondition(b), mg.vcycle(h, b)) <= tol
    R.close()


@pytest.mark.parametrize("deg,family", CASES)
def test_chebyshev_solve_matches_direct_in_fewer_iterations(deg, family):
    p = _prob(deg, family, seed=3)
    ref = fe.Model(p).run(method="splu")
    its = {}
    for name, extra in (("jacobi", {}), ("chebyshev", CHEB)):
        R = Run(p, FP32, **extra)
        R.set_densities()
        u, info = R.solve(rtol=1e-11)
        assert info.rel_residual <= 1e-11
        assert rel(u.cpu().numpy()[0], ref["u"][0]) <= 1e-6
        c, gx, gr = R.grad(u)
        assert abs(c[0] - ref["c"][0]) <= 1e-7 * abs(ref["c"][0])
        assert rel(gx, ref["g_x"]) <= 1e-6
        its[name] = info.iterations
        R.close()
    assert its["chebyshev"] < its["jacobi"], its


@pytest.mark.parametrize("inner", [0, 6])
def test_chebyshev_with_the_tensor_core_level(inner):
    """F16X3 stacked contraction at level 0: its Lanczos estimate uses the
    tensor-core operator, the solve still reaches the direct solution."""
    p = workloads.bridge(8, 4, 4, degree=2, n_mr=3, seed=9, mg_levels=2)
    ref = fe.Model(p).run(method="splu")
    R = Run(p, F16X3, inner_its=inner, **CHEB)
    R.set_densities()
    h = _hier(p)
    lam = R.T.tosolve_smoother_lmax(R.h, 0)
    assert abs(lam - h.levels[0].lmax) <= 1e-3 * h.levels[0].lmax
    u, info = R.solve(rtol=1e-11)
    assert info.rel_residual <= 1e-11
    assert rel(u.cpu().numpy()[0], ref["u"][0]) <= 1e-6
    R.close()


def test_chebyshev_descriptor_errors():
    T = lib()
    p1 = workloads.cantilever(4, 2, 2, degree=1, seed=0)
    with pytest.raises(T.TosolveError) as e:
        T.tosolve_footprint(desc_for(T, p1, FP32, **CHEB))
    assert e.value.status == T.EINVAL
    p2 = _prob(2, "lagrange")
    with pytest.raises(T.TosolveError):
        T.tosolve_footprint(desc_for(T, p2, FP32X2, **CHEB))
    with pytest.raises(T.TosolveError):
        T.tosolve_footprint(desc_for(T, p2, FP32, smoother=1, cheb_degree=5))
    assert T.tosolve_footprint(desc_for(T, p2, FP32, **CHEB)) > T.tosolve_footprint(desc_for(T, p2, FP32))
