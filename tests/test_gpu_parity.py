"""CUDA path vs the CPU oracle, step by step and end to end (through the C ABI).

Tolerances (the bar of the task, stated per check):
  * subcell table, densities, weights, FP64 operators: FP64 rounding only,
    relative 1e-13 (different summation orders / formulas on each side);
  * FP32 preconditioner operators: relative 1e-6 (single rounding of FP64
    values plus FP32 accumulation of 27 blocks);
  * FP32X2 operator apply (FP32 coefficients, float-pair arithmetic) against
    the FP64 product with the FP32-rounded oracle operator: relative 1e-9
    (the float-pair sum carries about 48 bits; the GPU's and the oracle's
    FP64 operators agree to 1e-13, so their FP32 roundings differ in at most
    a few entries by one FP32 ulp);
  * one multigrid cycle in FP64: relative 1e-9 (the coarse solve applies an
    explicit inverse formed by blocked Gauss-Jordan sweeps instead of two
    Cholesky triangular solves; its error is about cond(A_c) * 1e-16);
  * solves: true relative residual <= rtol (FP64, recomputed independently
    with the oracle's assembled K), displacement relative L2 error <= 1e-6,
    compliance relative error <= 1e-7, gradient relative L2 error <= 1e-6;
    error checks solve to rtol = 1e-11 so that the discretisation's
    conditioning does not mask a wrong operator.
"""
import numpy as np
import pytest

import workloads
from oracle import fe, fem, mg
from tests.gpu_helpers import Run, rel

pytestmark = pytest.mark.gpu

FP64, FP32, TF32, FP32X2 = 0, 1, 2, 3


_C1_REF = {}


def _c1_reference(m):
    if "ref" not in _C1_REF:
        _C1_REF["ref"] = m.run(method="mg", rtol=1e-13)
    return _C1_REF["ref"]


def oracle_residual(m, w_e, f, u, mask):
    K = m.assemble(w_e)
    free = mask == 0
    r = (f - K @ np.where(free, u, 0.0))[free]
    return np.linalg.norm(r) / np.linalg.norm(f[free])


# ---- step by step -------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3])
def test_subcell_table_matches_oracle(n):
    import torch

    p = workloads.cantilever(4, 2, 2, n_mr=n, seed=0, mg_levels=1)
    R = Run(p, FP64)
    t = torch.zeros((n ** 3, 24, 24), dtype=torch.float64, device=R.dev)
    R.T.tosolve_subcell_table(R.h, t)
    R.stream.synchronize()
    ref = fem.subcell_stiffness(1, n, p.nu)
    got = t.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    R.close()


@pytest.mark.parametrize("n,rmin", [(1, 0.0), (2, 1.5), (3, 0.7), (2, 1.0)])
def test_densities_and_weights_match_oracle(n, rmin):
    import torch

    p = workloads.cantilever(6, 4, 2, n_mr=n, rmin=rmin, seed=5, mg_levels=1)
    R = Run(p, FP64)
    R.set_densities()
    rho = torch.zeros_like(R.x)
    w = torch.zeros_like(R.x)
    R.T.tosolve_densities(R.h, rho, w)
    R.stream.synchronize()
    m = fe.Model(p)
    rho_ref = m.densities(p.x)
    w_ref = fe.simp_weights(rho_ref, p.E0, p.Emin, p.penal)
    assert rel(rho.cpu().numpy(), rho_ref) <= 1e-14
    assert rel(w.cpu().numpy(), w_ref) <= 1e-13
    if rmin == 0.0:
        assert np.array_equal(rho.cpu().numpy(), p.x)
    R.close()


@pytest.mark.parametrize("n,rmin", [(1, 0.0), (2, 1.5), (3, 0.7)])
def test_fine_operator_matches_assembled_K(n, rmin):
    p = workloads.cantilever(8, 4, 4, n_mr=n, rmin=rmin, seed=2, mg_levels=3)
    R = Run(p, FP32)
    R.set_densities()
    m = fe.Model(p)
    w_e = m.weights(m.densities(p.x))
    x = np.random.default_rng(0).normal(size=p.ndof)
    y_ref = m.apply(w_e, x)
    assert rel(R.apply(0, FP64, x), y_ref) <= 1e-13
    assert rel(R.apply(0, FP32, x), y_ref) <= 1e-6
    R.close()


@pytest.mark.parametrize("n,rmin", [(1, 0.0), (2, 1.5)])
def test_tensor_core_stacked_apply_matches_assembled_K(n, rmin):
    """Finest level of the TF32 preconditioner: the stacked subcell
    contraction on tcgen05 (TF32 operands, FP32 accumulation) plus the node
    gather.  TF32 keeps 10 mantissa bits of each operand: relative error of
    the product about 2^-11 per term, 5e-3 in the 2-norm as the bar."""
    p = workloads.cantilever(16, 8, 8, n_mr=n, rmin=rmin, seed=2, mg_levels=3)
    R = Run(p, TF32)
    R.set_densities()
    m = fe.Model(p)
    w_e = m.weights(m.densities(p.x))
    x = np.random.default_rng(0).normal(size=p.ndof)
    y_ref = m.apply(w_e, x)
    y = R.apply(0, TF32, x)
    assert rel(y, y_ref) <= 5e-3
    fixed = p.mask == 1
    np.testing.assert_allclose(y[fixed], x[fixed], rtol=1e-6)  # identity rows
    R.close()


@pytest.mark.parametrize("n", [1, 2])
def test_coarse_operators_match_oracle_hierarchy(n):
    # ragged: 12 x 4 x 8 with 3 levels -> 3 x 1 x 2 elements on the coarsest
    p = workloads.cantilever(12, 4, 8, n_mr=n, rmin=0.9 if n == 2 else 0.0, seed=8, mg_levels=3)
    m = fe.Model(p)
    rho = m.densities(p.x)
    h = mg.Hierarchy(p, rho, 3)
    rng = np.random.default_rng(1)
    R64 = Run(p, FP64)
    R64.set_densities()
    R32 = Run(p, FP32)
    R32.set_densities()
    for l, L in enumerate(h.levels):
        x = rng.normal(size=L.ndof)
        y_ref = L.A @ x
        assert rel(R64.apply(l, FP64, x), y_ref) <= 1e-12, l
        if l < 2:
            assert rel(R32.apply(l, FP32, x), y_ref) <= 1e-5, l
    R64.close()
    R32.close()


def test_one_cycle_matches_algorithm_1():
    p = workloads.cantilever(8, 4, 4, n_mr=2, rmin=1.0, seed=4, mg_levels=3, lo=0.3)
    m = fe.Model(p)
    rho = m.densities(p.x)
    h = mg.Hierarchy(p, rho, 3)
    b = np.where(p.mask == 0, np.random.default_rng(2).normal(size=p.ndof), 0.0)
    z_ref = mg.vcycle(h, b)
    R = Run(p, FP64)
    R.set_densities()
    assert rel(R.precondition(b), z_ref) <= 1e-9
    R.close()
    R = Run(p, FP32)
    R.set_densities()
    assert rel(R.precondition(b), z_ref) <= 1e-5
    R.close()


@pytest.mark.parametrize("n", [1, 2])
def test_fp32x2_operators_and_cycle(n):
    p = workloads.cantilever(12, 4, 8, n_mr=n, rmin=0.9 if n == 2 else 0.0, seed=8, mg_levels=3)
    m = fe.Model(p)
    rho = m.densities(p.x)
    h = mg.Hierarchy(p, rho, 3)
    rng = np.random.default_rng(1)
    R = Run(p, FP32X2)
    R.set_densities()
    for l, L in enumerate(h.levels[:-1]):
        x = rng.normal(size=L.ndof)
        A32 = L.A.astype(np.float32).astype(np.float64)
        y = R.apply(l, FP32X2, x)
        assert rel(y, A32 @ x) <= 1e-9, l
        assert rel(y, L.A @ x) <= 1e-6, l
        assert rel(R.apply(l, FP32, x), A32 @ x) > 1e-9 or l > 0  # FP32 sums are coarser
    b = np.where(p.mask == 0, rng.normal(size=p.ndof), 0.0)
    assert rel(R.precondition(b), mg.vcycle(h, b)) <= 1e-5
    R.close()


def test_fp32x2_keeps_fp64_convergence_on_high_contrast_densities():
    """rho ~ U[0.01, 1] (w from 1e-6 to 1): FP32 vector arithmetic in the
    V-cycle raises the PCG iteration count (about +45% here); float pairs on
    the same FP32 operators stay within 10% of the FP64 count (at this
    conditioning the count moves by a few with any change of rounding)."""
    p = workloads.batched_instances(1, 7, min_nx=64, max_nx=64, mult=8)[0]
    its = {}
    for prec in (FP64, FP32, FP32X2):
        R = Run(p, prec)
        R.set_densities()
        u, info = R.solve(rtol=1e-8)
        assert info.rel_residual <= 1e-8
        its[prec] = info.iterations
        R.close()
    assert its[FP32X2] <= 1.1 * its[FP64], its
    assert its[FP32X2] < its[FP32], its


# ---- whole path ----------------------------------------------------------------

@pytest.mark.parametrize("precision", [FP64, FP32, TF32, FP32X2])
@pytest.mark.parametrize("seed", [0, 1])
def test_cantilever_24x12x12_matches_direct_solve(precision, seed):
    """Config: Q1 24x12x12, n = 1, clamped face, line load, rho ~ U[0.01, 1]."""
    p = workloads.cantilever(24, 12, 12, seed=seed, mg_levels=3)
    m = fe.Model(p)
    ref = m.run(method="splu")
    R = Run(p, precision)
    R.set_densities()
    u, info = R.solve(rtol=1e-8)
    un = u.cpu().numpy()
    assert info.rel_residual <= 1e-8
    assert oracle_residual(m, ref["w"], p.f[0], un[0], p.mask) <= 1.05e-8
    u, info = R.solve(rtol=1e-11)
    un = u.cpu().numpy()
    assert rel(un[0], ref["u"][0]) <= 1e-6
    c, gx, gr = R.grad(u)
    assert abs(c[0] - ref["c"][0]) <= 1e-7 * abs(ref["c"][0])
    assert rel(gr, ref["g_rho"]) <= 1e-6
    assert rel(gx, ref["g_x"]) <= 1e-6
    R.close()


@pytest.mark.parametrize("precision", [FP64, FP32, TF32, FP32X2])
def test_multiresolution_48x24x24_full_size(precision):
    """Config: density 96x48x48, Q1 48x24x24 (n = 2), smooth field, r = 1.5,
    4 levels, FP64 / FP32 / TF32 / FP32X2 preconditioner -- the cantilever
    workload of the benchmark."""
    p = workloads.cantilever(48, 24, 24, n_mr=2, rmin=1.5, density="smooth", seed=0, mg_levels=4)
    m = fe.Model(p)
    ref = _c1_reference(m)
    R = Run(p, precision)
    R.set_densities()
    u, info = R.solve(rtol=1e-8)
    assert info.rel_residual <= 1e-8
    assert oracle_residual(m, ref["w"], p.f[0], u.cpu().numpy()[0], p.mask) <= 1.05e-8
    u, info = R.solve(rtol=1e-11, u0=u)
    assert rel(u.cpu().numpy()[0], ref["u"][0]) <= 1e-6
    c, gx, gr = R.grad(u)
    assert abs(c[0] - ref["c"][0]) <= 1e-7 * abs(ref["c"][0])
    assert rel(gx, ref["g_x"]) <= 1e-6
    R.close()


@pytest.mark.parametrize("shape,n,levels,rmin", [((6, 4, 2), 3, 2, 0.7), ((5, 3, 3), 2, 1, 0.5),
                                                 ((4, 4, 4), 1, 3, 0.0)])
def test_ragged_and_single_level_meshes(shape, n, levels, rmin):
    p = workloads.cantilever(*shape, n_mr=n, rmin=rmin, seed=9, mg_levels=levels)
    m = fe.Model(p)
    ref = m.run(method="dense")
    for prec in (FP64, FP32, TF32, FP32X2):
        if prec == TF32 and n > 2:
            continue
        R = Run(p, prec)
        R.set_densities()
        u, info = R.solve(rtol=1e-11)
        assert rel(u.cpu().numpy()[0], ref["u"][0]) <= 1e-6
        if levels == 1:  # the cycle is the exact coarse solve
            assert info.iterations <= 3
        c, gx, _ = R.grad(u)
        assert abs(c[0] - ref["c"][0]) <= 1e-7 * abs(ref["c"][0])
        assert rel(gx, ref["g_x"]) <= 1e-6
        R.close()


def test_multiple_load_cases_and_warm_start():
    p = workloads.cantilever(16, 8, 8, seed=3, mg_levels=3)
    Lx, Ly, Lz = p.lattice
    f = np.zeros((3, p.ndof))
    f[0] = p.f[0]
    tip = (Lx - 1) + Lx * ((Ly - 1) + Ly * (Lz - 1))
    f[1, 3 * tip + 1] = 1.0                       # sideways point load at a top corner
    f[2, 3 * tip: 3 * tip + 3] = (0.3, -0.2, 0.9)  # oblique point load
    p.f = f
    m = fe.Model(p)
    ref = m.run(method="splu")
    R = Run(p, FP32)
    R.set_densities()
    u, info = R.solve(rtol=1e-11)
    for r in range(p.nrhs):
        assert rel(u.cpu().numpy()[r], ref["u"][r]) <= 1e-6
    c, gx, _ = R.grad(u)
    np.testing.assert_allclose(c, ref["c"], rtol=1e-7)
    assert rel(gx, ref["g_x"]) <= 1e-6
    # warm start from the solution: nothing left to do
    u2, info2 = R.solve(rtol=1e-8, u0=u)
    assert info2.total_iterations == 0
    R.close()


def test_zero_load_maxit_and_order():
    p = workloads.cantilever(8, 4, 4, seed=1, mg_levels=2)
    R = Run(p, FP32)
    T = R.T
    with pytest.raises(T.TosolveError) as e:  # solve before set_densities
        R.solve()
    assert e.value.status == T.EINVAL
    R.set_densities()
    u, info = R.solve(rtol=1e-8, maxit=1, raise_on_error=False)
    assert info.status == T.ENOTCONV and info.iterations == 1 and info.rel_residual > 1e-8
    R.f.zero_()
    u0 = R.torch.ones((1, p.ndof), dtype=R.torch.float64, device=R.dev)
    u, info = R.solve(rtol=1e-8, u0=u0)
    assert info.total_iterations == 0 and float(u.abs().max()) == 0.0
    R.close()


@pytest.mark.parametrize("precision", [FP32, TF32, FP32X2])
def test_bitwise_deterministic(precision):
    p = workloads.cantilever(16, 8, 8, n_mr=2, rmin=1.0, seed=6, mg_levels=3)
    R = Run(p, precision)
    R.set_densities()
    u1, i1 = R.solve(rtol=1e-9)
    R.set_densities()
    u2, i2 = R.solve(rtol=1e-9)
    assert i1.iterations == i2.iterations
    assert R.torch.equal(u1, u2)
    c1, g1, _ = R.grad(u1)
    c2, g2, _ = R.grad(u2)
    assert c1[0] == c2[0] and np.array_equal(g1, g2)
    R.close()


def test_host_buffer_step_matches_device_calls():
    p = workloads.cantilever(16, 8, 8, n_mr=2, rmin=1.0, seed=7, mg_levels=3)
    R = Run(p, FP32)
    R.set_densities()
    u, info = R.solve(rtol=1e-10)
    c, gx, _ = R.grad(u)
    R.close()
    R = Run(p, FP32)
    uh = np.zeros((1, p.ndof))
    gh = np.zeros(p.x.size)
    ch, info2 = R.T.tosolve_step_host(R.h, np.ascontiguousarray(p.x), np.ascontiguousarray(p.f), 1,
                                      1e-10, 2000, 0, uh, gh)
    assert info2.iterations == info.iterations
    np.testing.assert_array_equal(uh, u.cpu().numpy())
    assert ch[0] == c[0] and np.array_equal(gh, gx)
    R.close()


def test_nan_in_load_is_a_breakdown():
    """A NaN in f makes the first residual norm NaN: the solve stops with
    TOSOLVE_EBREAKDOWN at once, fills info (status, iterations 0, NaN
    residual) and leaves the handle usable for the next, finite load."""
    import torch

    p = workloads.cantilever(8, 4, 4, n_mr=2, rmin=1.0, seed=5, mg_levels=2)
    R = Run(p, FP32)
    R.set_densities()
    T = R.T
    good = R.f.clone()
    R.f[0, 17] = float("nan")
    u, info = R.solve(rtol=1e-8, raise_on_error=False)
    assert info.status == T.EBREAKDOWN
    assert info.iterations == 0
    assert not np.isfinite(info.rel_residual)
    assert "breakdown" in T.tosolve_last_error(R.h).lower()
    R.f.copy_(good)
    u, info = R.solve(rtol=1e-8)
    assert info.status == T.OK and info.rel_residual <= 1e-8
    R.close()
