"""Degree-2 finest level of the tensor-core preconditioners vs the oracle.

The precisions TF32, BF16, BF16X3 and F16X3 apply the finest level of the
V-cycle as the stacked subcell contraction of Eq. matrixK_mr on tcgen05.
Each element's vector enters minus its least-squares rigid motion (in
FP32), which every subcell matrix annihilates (oracle fe.rigid_projector).
Rounding bounds, per row, with the subcell rounding scales of the oracle
(fe.Model.subcell_scale, sample.Sampler.apply_rows_subcell_scale):
  * TF32, BF16: each operand rounded once, unit roundoff u = 2^-11 resp.
    2^-8: error <= (2u + u^2) sum_e,i w_{e,i} |K^(e_i)| |P u_e| -- bar 2.2 u
    times that deflated scale;
  * BF16X3: operands split into BF16 pairs (each within 2^-16 of the
    value), three products: error <= 3 * 2^-16 times the scale -- bar 3.3
    * 2^-16 times the deflated element-max scale;
  * F16X3: FP16 pairs after a power-of-two scaling of each element's vector
    (largest entry in [0.5, 1)) and of the table: each pair within 2^-22 of
    its value above FP16's normal range and 2^-25 of the element's largest
    below it -- bar 3.3 * 2^-22 times the deflated element-max scale;
plus, for every mode, the FP32 work (the cast of the vector, the deflation,
the accumulation of up to 288 products, the weighted subcell sum, the node
gather): 64 * 2^-24 times the undeflated scale.  Supports are identity rows.
The solves keep the FP64 outer CG, so displacement, compliance and gradient
meet the parity tolerances of the other solves (1e-6, 1e-7, 1e-6).
"""
import numpy as np
import pytest

import workloads
from oracle import fe, sample
from tests.gpu_helpers import Run, rel

pytestmark = pytest.mark.gpu

FP32, TF32, BF16, BF16X3, F16X3 = 1, 2, 4, 5, 6
MODES = [TF32, BF16, BF16X3, F16X3]
FP32_WORK = 64 * 2.0 ** -24


def _bar(prec, scale_def, scale_max, scale):
    if prec == TF32:
        b = 2.2 * 2.0 ** -11 * scale_def
    elif prec == BF16:
        b = 2.2 * 2.0 ** -8 * scale_def
    elif prec == BF16X3:
        b = 3.3 * 2.0 ** -16 * scale_max
    else:
        b = 3.3 * 2.0 ** -22 * scale_max
    return b + FP32_WORK * scale


def _check_rows(y, y_ref, bar, fixed, x):
    err = np.abs(y - y_ref)
    free = ~fixed
    assert (err[free] <= bar[free]).all(), float((err[free] / np.maximum(bar[free], 1e-300)).max())
    np.testing.assert_allclose(y[fixed], x[fixed], rtol=1e-6)  # identity rows (FP32 round trip)


def _whole_mesh_bar(m, w_e, x, prec):
    return _bar(prec, m.subcell_scale(w_e, x, deflate=True), m.subcell_scale(w_e, x, deflate=True, elem_max=True),
                m.subcell_scale(w_e, x))


@pytest.mark.parametrize("prec", MODES)
@pytest.mark.parametrize("n,rmin", [(1, 0.0), (2, 1.0), (3, 0.0)])
def test_tc2_apply_rows_within_rounding_bound(prec, n, rmin):
    """10x6x4 elements: two 128-element tiles, the second ragged (112)."""
    p = workloads.bridge(10, 6, 4, degree=2, n_mr=n, rmin=rmin, seed=3, mg_levels=2)
    R = Run(p, prec)
    R.set_densities()
    m = fe.Model(p)
    w_e = m.weights(m.densities(p.x))
    x = np.random.default_rng(1).normal(size=p.ndof)
    y = R.apply(0, prec, x)
    _check_rows(y, m.apply(w_e, x), _whole_mesh_bar(m, w_e, x, prec), p.mask == 1, x)
    assert np.array_equal(R.apply(0, prec, x), y)  # fixed order: bitwise repeatable
    R.close()


@pytest.mark.parametrize("prec", MODES)
def test_tc2_near_rigid_input_is_deflated(prec):
    """A large rigid motion plus a small deformation (the shape of a smooth
    multigrid correction): the error follows the deformation.  Without the
    deflation the rounding would act on the rigid part, 10^4 times larger,
    and break the bar."""
    p = workloads.bridge(8, 4, 4, degree=2, n_mr=3, seed=4, mg_levels=2)
    Lx, Ly, Lz = p.lattice
    pos = np.array([[i, j, l] for l in range(Lz) for j in range(Ly) for i in range(Lx)], dtype=float) / 2.0
    rigid = (np.array([3.0, -2.0, 1.0]) + np.cross([0.4, -0.2, 0.3], pos)).reshape(-1)
    x = rigid + 1e-4 * np.random.default_rng(2).normal(size=p.ndof)
    R = Run(p, prec)
    R.set_densities()
    m = fe.Model(p)
    w_e = m.weights(m.densities(p.x))
    y = R.apply(0, prec, x)
    _check_rows(y, m.apply(w_e, x), _whole_mesh_bar(m, w_e, x, prec), p.mask == 1, x)
    R.close()


@pytest.mark.parametrize("prec", MODES)
def test_tc2_cantilever_matches_direct_solve(prec):
    """Filtered multiresolution cantilever, 8x4x4 Q2, n = 2, 3 levels."""
    p = workloads.cantilever(8, 4, 4, degree=2, n_mr=2, rmin=1.0, seed=5, mg_levels=3)
    ref = fe.Model(p).run(method="splu")
    R = Run(p, prec)
    R.set_densities()
    u, info = R.solve(rtol=1e-11)
    assert info.rel_residual <= 1e-11
    assert rel(u.cpu().numpy()[0], ref["u"][0]) <= 1e-6
    c, gx, gr = R.grad(u)
    assert abs(c[0] - ref["c"][0]) <= 1e-7 * abs(ref["c"][0])
    assert rel(gr, ref["g_rho"]) <= 1e-6
    assert rel(gx, ref["g_x"]) <= 1e-6
    R.close()


@pytest.mark.parametrize("prec", MODES)
def test_tc2_bridge_matches_direct_solve(prec):
    """Bridge, 8x4x4 Q2 with n = 3 (27 subcells): the configuration's element."""
    p = workloads.bridge(8, 4, 4, degree=2, n_mr=3, rmin=0.0, seed=6, mg_levels=2)
    ref = fe.Model(p).run(method="splu")
    its = {}
    for q in (FP32, prec):
        R = Run(p, q)
        R.set_densities()
        u, info = R.solve(rtol=1e-11)
        its[q] = info.iterations
        assert rel(u.cpu().numpy()[0], ref["u"][0]) <= 1e-6
        c, gx, _ = R.grad(u)
        assert abs(c[0] - ref["c"][0]) <= 1e-7 * abs(ref["c"][0])
        assert rel(gx, ref["g_x"]) <= 1e-6
        R.close()
    # a rounded finest-level operator may cost iterations, not many
    assert its[prec] <= 1.5 * its[FP32] + 2, its


@pytest.mark.parametrize("prec", [BF16X3, F16X3])
def test_tc2_bridge_full_size(prec):
    """The all-triquadratic bridge of the benchmark, 64x32x32, n = 3 (65,536
    elements: 512 tiles, several per CTA): sampled rows of the tensor-core
    apply within the rounding bound, then the solve to 1e-8 with the
    operator, compliance and gradient checked on samples.  With the FP16
    pairs the iteration count stays within about a third of the FP32
    element matrices' (88 on this input; 106 measured)."""
    from tests.test_gpu_fullsize import _check_sampled

    p = workloads.bridge(64, 32, 32, degree=2, n_mr=3, rmin=0.0, seed=0)
    S = sample.Sampler(p)
    R = Run(p, prec)
    R.set_densities()
    rng = np.random.default_rng(9)
    x = rng.normal(size=p.ndof)
    y = R.apply(0, prec, x).reshape(-1, 3)
    picks = list(rng.choice(p.nnodes, size=120, replace=False)) + [0, p.nnodes - 1]
    yr = S.apply_rows(p.x, x, picks)
    bar = _bar(prec, S.apply_rows_subcell_scale(p.x, x, picks, deflate=True),
               S.apply_rows_subcell_scale(p.x, x, picks, deflate=True, elem_max=True),
               S.apply_rows_subcell_scale(p.x, x, picks))
    fixed = p.mask.reshape(-1, 3)[picks] == 1
    _check_rows(y[picks], yr, bar, fixed, x.reshape(-1, 3)[picks])
    u, info = R.solve(rtol=1e-8)
    assert info.rel_residual <= 1e-8
    if prec == F16X3:
        assert info.iterations <= 120, info.iterations
    _check_sampled(R.T, R, p, u[0], 1e-8, np.random.default_rng(5), nodes=80, cells=20, dcells=4)
    R.close()


@pytest.mark.parametrize("prec,inner", [(F16X3, 6), (BF16, 4), (FP32, 5)])
def test_inner_fp32_iterations_match_direct_solve(prec, inner):
    """Each outer FP64 iteration preconditioned by a few FP32 PCG iterations
    on the preconditioner's level-0 operator (inner_its): the converged
    solution, compliance and gradient are the direct solve's, and the outer
    FP64 iterations drop well below the single-V-cycle count."""
    from paper_2311_05595_gb300 import tosolve as T

    p = workloads.bridge(8, 4, 4, degree=2, n_mr=3, rmin=0.0, seed=6, mg_levels=2)
    ref = fe.Model(p).run(method="splu")
    R = Run(p, prec)
    R.set_densities()
    _, plain = R.solve(rtol=1e-11)
    R.close()
    R = Run(p, prec)
    R.close()
    R.solver = T.Solver(T.make_desc(p.nx, p.ny, p.nz, degree=2, n_mr=p.n_mr, nu=p.nu, penal=p.penal,
                                    Emin=p.Emin, mg_levels=2, precision=prec, inner_its=inner),
                        p.mask, R.stream)
    R.h = R.solver.h
    R.set_densities()
    u, info = R.solve(rtol=1e-11)
    assert info.rel_residual <= 1e-11
    assert info.iterations < plain.iterations, (info.iterations, plain.iterations)
    assert rel(u.cpu().numpy()[0], ref["u"][0]) <= 1e-6
    c, gx, gr = R.grad(u)
    assert abs(c[0] - ref["c"][0]) <= 1e-7 * abs(ref["c"][0])
    assert rel(gr, ref["g_rho"]) <= 1e-6
    R.close()


def test_inner_iterations_on_a_mixed_mesh():
    """FP32 inner iterations on the element matrices of a mixed trilinear /
    triquadratic mesh (slaved midside nodes): the mixed oracle's solution."""
    from oracle import mixed
    from paper_2311_05595_gb300 import tosolve as T

    p = workloads.with_mixed_degree(workloads.bridge(8, 4, 4, degree=2, n_mr=2, seed=3, mg_levels=2), 0.5, 5)
    ref = mixed.MixedModel(p).run(method="splu")
    R = Run(p, FP32)
    R.close()
    R.solver = T.Solver(T.make_desc(p.nx, p.ny, p.nz, degree=2, n_mr=p.n_mr, nu=p.nu, penal=p.penal,
                                    Emin=p.Emin, mg_levels=2, precision=FP32, inner_its=6),
                        p.mask, R.stream, elem_q1=p.elem_q1)
    R.h = R.solver.h
    R.set_densities()
    u, info = R.solve(rtol=1e-11)
    assert info.rel_residual <= 1e-11
    assert rel(u.cpu().numpy()[0], ref["u"][0]) <= 1e-6
    c, gx, _ = R.grad(u)
    assert abs(c[0] - ref["c"][0]) <= 1e-7 * abs(ref["c"][0])
    assert rel(gx, ref["g_x"]) <= 1e-6
    R.close()


def _mixed(shape, n, seed, levels=2):
    return workloads.with_mixed_degree(workloads.bridge(*shape, degree=2, n_mr=n, seed=seed, mg_levels=levels),
                                       0.5, seed + 1)


@pytest.mark.parametrize("prec", MODES)
def test_tc2_mixed_apply_rows_within_rounding_bound(prec):
    """Mixed trilinear / triquadratic mesh: triquadratic elements expand
    their slaved nodes and fold the result back (T_e^T K T_e), trilinear
    ones use the trilinear subcell matrices on their vertices; every row
    within the rounding bound of what each element rounds."""
    p = _mixed((8, 4, 4), 3, 7)
    S = sample.Sampler(p)
    R = Run(p, prec)
    R.set_densities()
    x = np.random.default_rng(3).normal(size=p.ndof)
    y = R.apply(0, prec, x).reshape(-1, 3)
    nodes = list(range(p.nnodes))
    yr = S.apply_rows(p.x, x, nodes)
    bar = _bar(prec, S.apply_rows_subcell_scale(p.x, x, nodes, deflate=True),
               S.apply_rows_subcell_scale(p.x, x, nodes, deflate=True, elem_max=True),
               S.apply_rows_subcell_scale(p.x, x, nodes))
    held = (p.mask.astype(bool) | np.repeat(S.slv, 3)).reshape(-1, 3)
    _check_rows(y, yr, bar, held, x.reshape(-1, 3))
    R.close()


@pytest.mark.parametrize("prec,inner", [(F16X3, 0), (BF16X3, 0), (F16X3, 6), (BF16, 5)])
def test_tc2_mixed_matches_direct_solve(prec, inner):
    from oracle import mixed
    from paper_2311_05595_gb300 import tosolve as T

    p = _mixed((8, 4, 4), 3, 9)
    ref = mixed.MixedModel(p).run(method="splu")
    R = Run(p, FP32)
    R.close()
    R.solver = T.Solver(T.make_desc(p.nx, p.ny, p.nz, degree=2, n_mr=p.n_mr, nu=p.nu, penal=p.penal,
                                    Emin=p.Emin, mg_levels=2, precision=prec, inner_its=inner),
                        p.mask, R.stream, elem_q1=p.elem_q1)
    R.h = R.solver.h
    R.set_densities()
    u, info = R.solve(rtol=1e-11)
    assert info.rel_residual <= 1e-11
    assert rel(u.cpu().numpy()[0], ref["u"][0]) <= 1e-6
    c, gx, gr = R.grad(u)
    assert abs(c[0] - ref["c"][0]) <= 1e-7 * abs(ref["c"][0])
    assert rel(gr, ref["g_rho"]) <= 1e-6
    assert rel(gx, ref["g_x"]) <= 1e-6
    R.close()


@pytest.mark.parametrize("prec,inner", [(F16X3, 16), (BF16, 12), (F16X3, 24)])
def test_tc2_mixed_bridge_full_size(prec, inner):
    """The bridge as specified (64x32x32, n = 3, a seeded half trilinear;
    519,204 unknowns) with the benchmark's tensor-core preconditioners
    (BF16 with 12 inner FP32 iterations per outer one, F16X3 with 16 and
    24): solve to 1e-8, operator rows, compliance and gradient checked on
    samples."""
    from paper_2311_05595_gb300 import tosolve as T
    from tests.test_gpu_fullsize import _check_sampled

    p = workloads.with_mixed_degree(workloads.bridge(64, 32, 32, degree=2, n_mr=3, seed=0), 0.5, 11)
    R = Run(p, FP32)
    R.close()
    R.solver = T.Solver(T.make_desc(p.nx, p.ny, p.nz, degree=2, n_mr=3, nu=p.nu, penal=p.penal, Emin=p.Emin,
                                    mg_levels=0, precision=prec, inner_its=inner),
                        p.mask, R.stream, elem_q1=p.elem_q1)
    R.h = R.solver.h
    R.set_densities()
    u, info = R.solve(rtol=1e-8)
    assert info.rel_residual <= 1e-8
    assert R.T.tosolve_free_dofs(R.h) == 519204
    _check_sampled(R.T, R, p, u[0], 1e-8, np.random.default_rng(3), nodes=100, cells=24, dcells=4)
    R.close()
