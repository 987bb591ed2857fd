"""Parity at the benchmark configurations' full sizes, on sampled outputs.

The meshes here are too large for the oracle to assemble (1.6M DOFs), so the
oracle recomputes sampled rows of K u and sampled cells of the gradient from
their definitions on the few elements involved (oracle/sample.py, pinned
against the whole-mesh oracle).  Checks, each in the launch configuration
the benchmark times:
  * the FP64 operator at sampled nodes, to 1e-12 of each row's rounding
    scale sum_j |K_ij u_j| (at a converged u the rows nearly cancel);
  * the solve: true relative residual <= rtol recomputed with that operator;
  * compliance f^T u (1e-12 relative, a sum over 10^6 terms);
  * dc/drho at sampled cells, to within 1e-12 of the rounding scale of the
    quadratic form u_e^T K^(e_i) u_e (sum of |K_ab u_a u_b|): the same
    formula on the same u in another order, whose terms cancel strongly in
    elements that move almost rigidly; dc/dx equal to it without a filter,
    else one row of H^T at a few design cells, to the same relative bound.
"""
import numpy as np
import pytest

import workloads
from oracle import sample
from tests.gpu_helpers import Run, lib, desc_for, rel

pytestmark = [pytest.mark.gpu]

FP64, FP32X2 = 0, 3


def _check_sampled(T, R, p, u_dev, rtol, rng, nodes=200, cells=40, dcells=8, fixed_void=None):
    import torch

    S = sample.Sampler(p)
    u = u_dev.cpu().numpy().reshape(-1)
    # operator rows
    picks = list(rng.choice(p.nnodes, size=nodes, replace=False)) + [0, p.nnodes - 1]
    y = R.apply(0, FP64, u).reshape(-1, 3)
    ys = S.apply_rows(p.x, u, picks)
    sc = S.apply_rows_scale(p.x, u, picks)
    err = np.abs(y[picks] - ys) / (1e-12 * sc + 1e-300)
    assert err.max() <= 1.0, (err.max(), np.abs(y[picks] - ys).max(), np.abs(y).max())
    # residual with that operator
    f = np.where(p.mask == 0, p.f[0], 0.0)
    if getattr(p, "elem_q1", None) is None:
        r = f - y.reshape(-1)
        r[p.mask != 0] = 0.0
        assert np.linalg.norm(r) <= 1.05 * rtol * np.linalg.norm(f)
    # compliance and gradient
    c, gx, gr = R.grad(u_dev.reshape(1, -1).contiguous(), nrhs=1)
    assert abs(c[0] - float(np.dot(f, u))) <= 1e-12 * abs(c[0])
    cs = rng.choice(p.x.size, size=cells, replace=False)
    ref = np.array([S.drho(p.x, u, ci) for ci in cs])
    scale = np.array([S.drho_scale(p.x, u, ci) for ci in cs])
    err = np.abs(gr[cs] - ref) / np.maximum(1e-12 * scale + 1e-14 * np.abs(ref), 1e-300)
    assert err.max() <= 1.0, (err.max(), np.abs(gr[cs] - ref).max())
    if p.rmin == 0.0:  # the filter is the identity: dc/dx = dc/drho
        np.testing.assert_array_equal(gx[cs], gr[cs])
    else:  # one row of H^T at a few design cells
        ds = cs[:dcells]
        refx = np.array([S.dx(p.x, u, ci) for ci in ds])
        if fixed_void is not None:  # Sec. 6.1: zero for the variables of fixed void elements
            refx[fixed_void[ds] == 1] = 0.0
        scx = np.array([S.dx_scale(p.x, u, ci) for ci in ds])
        errx = np.abs(gx[ds] - refx) / np.maximum(1e-12 * scx + 1e-14 * np.abs(refx), 1e-300)
        assert errx.max() <= 1.0, (errx.max(), np.abs(gx[ds] - refx).max())


def test_largest_batch_instance_full_size():
    """The 128x64x64 Q1 instance (1,622,400 free DOFs) of the 64-instance
    batch, solved with a smaller one in one batched graph launch, FP32X2."""
    import torch

    T = lib()
    probs = workloads.batched_instances(64, 2024, mult=16)
    big = max(probs, key=lambda q: q.nfree)
    small = min(probs, key=lambda q: q.nfree)
    runs = [Run(q, FP32X2) for q in (big, small)]
    for R in runs:
        R.set_densities()
    us = [torch.zeros((q.nrhs, q.ndof), dtype=torch.float64, device=R.dev) for q, R in zip((big, small), runs)]
    b = T.tosolve_batch_create([R.h for R in runs], [q.nrhs for q in (big, small)], [R.f for R in runs], us)
    try:
        infos = T.tosolve_batch_solve(b, 1e-8, 2000, 2)
        assert all(i.status == T.OK for i in infos)
        big1 = big.__class__(**{k: getattr(big, k) for k in big.__dataclass_fields__})
        big1.f = big.f[:1]
        _check_sampled(T, runs[0], big1, us[0][0], 1e-8, np.random.default_rng(7))
    finally:
        T.tosolve_batch_destroy(b)
        for R in runs:
            R.close()


def test_mixed_bridge_full_size():
    """The bridge as specified: 64x32x32, n = 3, half the elements trilinear
    (519,204 unknowns), FP32X2 preconditioner as in the benchmark."""
    import torch

    p = workloads.with_mixed_degree(
        workloads.bridge(64, 32, 32, degree=2, n_mr=3, seed=0), 0.5, 11)
    R = Run(p, FP32X2)
    R.set_densities()
    u, info = R.solve(rtol=1e-8)
    assert info.rel_residual <= 1e-8
    assert R.T.tosolve_free_dofs(R.h) == 519204
    _check_sampled(R.T, R, p, u[0], 1e-8, np.random.default_rng(3), nodes=120, cells=30, dcells=6)
    R.close()


def test_serendipity_cantilever_full_size():
    """The serendipity benchmark configuration: 48x24x24 elements, n = 2,
    the smooth design with r = 1.5, 352,800 unknowns; FP32X2."""
    p = workloads.with_serendipity(workloads.cantilever(48, 24, 24, degree=2, n_mr=2, rmin=1.5,
                                                        density="smooth", seed=0))
    R = Run(p, FP32X2)
    R.set_densities()
    u, info = R.solve(rtol=1e-8, maxit=3000)
    assert info.rel_residual <= 1e-8
    assert R.T.tosolve_free_dofs(R.h) == p.nfree == 352800
    _check_sampled(R.T, R, p, u[0], 1e-8, np.random.default_rng(11), nodes=150, cells=30)
    R.close()


def test_suppression_on_the_ibeam_full_size():
    """The I-beam of the suppression benchmark (96x48x48 Q1, n = 2, r = 1.5):
    the selection bit for bit against the oracle's, then the suppressed
    operator on sampled rows and the solve."""
    import torch

    from oracle import fe, fix

    p = workloads.cantilever(96, 48, 48, n_mr=2, rmin=1.5, density="ibeam", seed=0)
    S = sample.Sampler(p)
    R = Run(p, FP32X2)
    R.set_densities()
    rho_dev = torch.zeros_like(R.x)
    with torch.cuda.stream(R.stream):
        R.T.tosolve_densities(R.h, rho_dev)
    R.stream.synchronize()
    rho = rho_dev.cpu().numpy()
    # the densities themselves are pinned against the sampled oracle
    cells = np.random.default_rng(5).choice(p.x.size, size=200, replace=False)
    np.testing.assert_allclose(rho[cells], [S.rho(p.x, c) for c in cells], rtol=1e-14, atol=1e-300)
    fixed = torch.zeros(p.x.size, dtype=torch.uint8, device=R.dev)
    nsup = R.T.tosolve_fix_variables(R.h, None, 1e-6, 0.9, 1e-6, fixed)
    fx = fix.fixed_elements(p, fix.element_class(p, rho, None, 1e-6, 0.9, 1e-6))
    assert np.array_equal(fixed.cpu().numpy(), fix.fixed_design_variables(p, fx).astype(np.uint8))
    q = fix.suppressed_problem(p, fix.suppressed_nodes(p, fx))
    assert nsup == p.nfree - q.nfree and R.T.tosolve_free_dofs(R.h) == q.nfree
    u, info = R.solve(rtol=1e-8)
    assert info.rel_residual <= 1e-8
    _check_sampled(R.T, R, q, u[0], 1e-8, np.random.default_rng(12), nodes=150, cells=20,
                   fixed_void=fixed.cpu().numpy())
    R.close()


def test_cubic_serendipity_full_size():
    """The 32-node serendipity element at the element-family benchmark's
    size: 96x16x16 elements, n = 4, r = 0.6; FP32X2."""
    p = workloads.with_serendipity(workloads.cantilever(96, 16, 16, degree=3, n_mr=4, rmin=0.6,
                                                        density="smooth", seed=0))
    R = Run(p, FP32X2)
    R.set_densities()
    u, info = R.solve(rtol=1e-8, maxit=3000)
    assert info.rel_residual <= 1e-8
    assert R.T.tosolve_free_dofs(R.h) == p.nfree
    _check_sampled(R.T, R, p, u[0], 1e-8, np.random.default_rng(13), nodes=80, cells=20)
    R.close()
