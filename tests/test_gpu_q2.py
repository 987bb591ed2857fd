"""Lagrange degree 2 (triquadratic elements) on the GPU vs the CPU oracle.

Tolerances as in the degree-1 parity tests: FP64 operators to FP64 rounding
(1e-13 fine, 1e-12 coarse: the coarse element matrices come from 125
polynomial moments on the GPU and from subcell sums in the oracle); FP32
operators 1e-6; one FP64 cycle 1e-9; solves: displacement 1e-6, compliance
1e-7, gradient 1e-6 at rtol 1e-11.
"""
import numpy as np
import pytest

import workloads
from oracle import fe, fem, mg
from tests.gpu_helpers import Run, rel

pytestmark = pytest.mark.gpu

FP64, FP32, FP32X2 = 0, 1, 3


@pytest.mark.parametrize("n", [1, 2, 3])
def test_q2_subcell_table_matches_oracle(n):
    import torch

    p = workloads.cantilever(2, 2, 2, degree=2, n_mr=n, seed=0, mg_levels=1)
    R = Run(p, FP64)
    t = torch.zeros((n ** 3, 81, 81), dtype=torch.float64, device=R.dev)
    R.T.tosolve_subcell_table(R.h, t)
    R.stream.synchronize()
    ref = fem.subcell_stiffness(2, n, p.nu)
    got = t.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    R.close()


@pytest.mark.parametrize("n,rmin", [(1, 0.0), (2, 1.0), (3, 0.7)])
def test_q2_operators_match_oracle(n, rmin):
    p = workloads.cantilever(8, 4, 4, degree=2, n_mr=n, rmin=rmin, seed=2, mg_levels=3)
    m = fe.Model(p)
    rho = m.densities(p.x)
    h = mg.Hierarchy(p, rho, 3)
    rng = np.random.default_rng(0)
    R = Run(p, FP32)
    R.set_densities()
    for l, L in enumerate(h.levels[:-1]):
        x = rng.normal(size=L.ndof)
        y_ref = L.A @ x
        assert rel(R.apply(l, FP64, x), y_ref) <= (1e-13 if l == 0 else 1e-12), l
        assert rel(R.apply(l, FP32, x), y_ref) <= 1e-6, l
    R.close()
    R = Run(p, FP32X2)
    R.set_densities()
    x = rng.normal(size=p.ndof)
    assert rel(R.apply(0, FP32X2, x), h.levels[0].A @ x) <= 1e-6
    R.close()


@pytest.mark.parametrize("prolongation,transfer", [(0, "shape"), (1, "linear")])
def test_q2_one_cycle_matches_algorithm_1(prolongation, transfer):
    """One V-cycle against the oracle's Algorithm 1, with the coarse shape
    functions as transfers (the default) and with linear interpolation on
    the node lattices (prolongation = 1)."""
    from paper_2311_05595_gb300 import tosolve as T

    p = workloads.cantilever(8, 4, 4, degree=2, n_mr=2, rmin=1.0, seed=4, mg_levels=3, lo=0.3)
    m = fe.Model(p)
    h = mg.Hierarchy(p, m.densities(p.x), 3, transfer=transfer)
    b = np.where(p.mask == 0, np.random.default_rng(2).normal(size=p.ndof), 0.0)
    R = Run(p, FP64)
    if prolongation:
        R.close()
        R.solver = T.Solver(T.make_desc(p.nx, p.ny, p.nz, degree=2, n_mr=p.n_mr, rmin=p.rmin, nu=p.nu,
                                        penal=p.penal, Emin=p.Emin, mg_levels=3, prolongation=1),
                            p.mask, R.stream)
        R.h = R.solver.h
    R.set_densities()
    assert rel(R.precondition(b), mg.vcycle(h, b)) <= 1e-9
    R.close()


@pytest.mark.parametrize("precision", [FP64, FP32, FP32X2])
def test_q2_cantilever_matches_direct_solve(precision):
    p = workloads.cantilever(8, 4, 4, degree=2, n_mr=2, rmin=1.0, seed=5, mg_levels=3)
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


@pytest.mark.parametrize("shape,n,levels", [((8, 4, 4), 3, 2), ((6, 4, 2), 1, 1), ((4, 4, 4), 2, 3)])
def test_q2_bridge_and_ragged_meshes(shape, n, levels):
    p = workloads.bridge(*shape, degree=2, n_mr=n, rmin=0.0, seed=6, mg_levels=levels)
    ref = fe.Model(p).run(method="splu")
    for prec in (FP64, FP32X2):
        R = Run(p, prec)
        R.set_densities()
        u, info = R.solve(rtol=1e-11)
        assert rel(u.cpu().numpy()[0], ref["u"][0]) <= 1e-6
        c, gx, _ = R.grad(u)
        assert abs(c[0] - ref["c"][0]) <= 1e-7 * abs(ref["c"][0])
        assert rel(gx, ref["g_x"]) <= 1e-6
        R.close()
