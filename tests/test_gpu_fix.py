"""Fixing variables and suppressing void-region DOFs on the GPU
(tosolve_fix_variables, Sec. 6.1) against the oracle (oracle/fix.py).

Element classes, fixed design variables and the suppressed set are integer
decisions taken on the same FP64 densities and gradient on both sides: bit
for bit.  The operator after suppression matches the oracle's operator with
the suppressed DOFs among the supports (1e-13); the solve (rtol 1e-11), the
compliance and the gradient (with the fixed void components zeroed) match as
in the other parity tests.  Releasing the selection restores the original
system exactly.
"""
import numpy as np
import pytest

import workloads
from oracle import fe, fix, mesh
from tests.gpu_helpers import Run, rel

pytestmark = pytest.mark.gpu

FP64, FP32, FP32X2 = 0, 1, 3
LO, HI, EPS = 1e-6, 0.9, 1e-6


def _structured(k, n, shape, rmin, seed, levels):
    """A cantilever whose design is solid in the lower half and void above,
    with a few solid islands in the void (so that the fixed void region has
    holes and the border cases of the neighbourhood rule occur)."""
    p = workloads.cantilever(*shape, degree=k, n_mr=n, rmin=rmin, seed=seed, mg_levels=levels)
    Dx, Dy = n * shape[0], n * shape[1]
    c = np.arange(p.x.size)
    cx, cy, cz = c % Dx, (c // Dx) % Dy, c // (Dx * Dy)
    x = np.where(cz < n * shape[2] // 2, 1.0, 0.0)
    rng = np.random.default_rng(seed)
    for _ in range(3):
        ix, iy, iz = rng.integers(0, Dx - n), rng.integers(0, Dy - n), rng.integers(n * shape[2] // 2, n * shape[2] - n)
        x[(cx >= ix) & (cx < ix + n) & (cy >= iy) & (cy < iy + n) & (cz >= iz) & (cz < iz + n)] = 1.0
    p.x = x
    return p


def _structural_dofs(p):
    """DOFs of the solid lower half, the part of the design connected to the
    supports and the load.  Elsewhere the stiffness is of order Emin (and
    the islands float in the void): a residual r moves u there by about
    r / Emin, so u there is compared more loosely."""
    ez = np.arange(p.nx * p.ny * p.nz) // (p.nx * p.ny)
    main = ez < p.nz // 2
    return np.unique(mesh.element_dofs(p.nx, p.ny, p.nz, p.degree)[main].reshape(-1))


def _gradient(p, seed):
    """A synthetic design gradient: mostly tiny, some components beyond the
    safeguards in both directions."""
    rng = np.random.default_rng(seed)
    g = rng.uniform(-0.5e-6, 0.5e-6, size=p.x.size)
    pick = rng.choice(p.x.size, size=max(1, p.x.size // 200), replace=False)
    g[pick] = rng.choice([-1e-3, 1e-3], size=pick.size)
    return g


CASES = [
    (1, 2, (16, 8, 8), 1.0, 3, FP32X2),
    (1, 1, (12, 8, 8), 0.0, 3, FP64),
    (2, 2, (8, 4, 4), 0.0, 2, FP32X2),
]


@pytest.mark.parametrize("k,n,shape,rmin,levels,prec", CASES)
@pytest.mark.parametrize("with_grad", [False, True])
def test_selection_and_solve_match_oracle(k, n, shape, rmin, levels, prec, with_grad):
    import torch

    p = _structured(k, n, shape, rmin, seed=11, levels=levels)
    m = fe.Model(p)
    rho = m.densities(p.x)
    g = _gradient(p, 5) if with_grad else None
    cls = fix.element_class(p, rho, g, LO, HI, EPS)
    fx = fix.fixed_elements(p, cls)
    fxv = fix.fixed_design_variables(p, fx)
    sup = fix.suppressed_nodes(p, fx)
    q = fix.suppressed_problem(p, sup)
    assert sup.any() and (with_grad or (fx == fix.SOLID).any())

    R = Run(p, prec)
    R.set_densities()
    T = R.T
    fixed = torch.zeros(p.x.size, dtype=torch.uint8, device=R.dev)
    gd = None if g is None else torch.tensor(g, device=R.dev)
    nsup = T.tosolve_fix_variables(R.h, gd, LO, HI, EPS, fixed)
    assert np.array_equal(fixed.cpu().numpy(), fxv.astype(np.uint8))
    assert nsup == p.nfree - q.nfree
    assert T.tosolve_free_dofs(R.h) == q.nfree
    # the operator: suppressed DOFs are identity rows with zero columns
    mq = fe.Model(q)
    w = mq.weights(rho)
    xv = np.random.default_rng(0).normal(size=p.ndof)
    assert rel(R.apply(0, FP64, xv), mq.apply(w, xv)) <= 1e-13
    # solve, compliance, gradient with the fixed void components zeroed
    ref = mq.run(method="splu")
    u, info = R.solve(rtol=1e-11)
    assert info.rel_residual <= 1e-11
    sd = _structural_dofs(p)
    un = u.cpu().numpy()[0]
    assert rel(un[sd], ref["u"][0][sd]) <= 1e-6
    assert rel(un, ref["u"][0]) <= 1e-4
    assert (un[np.repeat(sup, 3)] == 0.0).all()
    c, gx, gr = R.grad(u)
    assert abs(c[0] - ref["c"][0]) <= 1e-7 * abs(ref["c"][0])
    assert rel(gr, ref["g_rho"]) <= 1e-6
    gxz = fix.zero_fixed_void_gradient(ref["g_x"], fxv)
    assert rel(gx, gxz) <= 1e-6
    assert (gx[fxv == fix.VOID] == 0.0).all()
    # a new design keeps the selection; release restores the original system
    R.set_densities()
    assert T.tosolve_free_dofs(R.h) == q.nfree
    T.tosolve_release_variables(R.h)
    assert T.tosolve_free_dofs(R.h) == p.nfree
    assert rel(R.apply(0, FP64, xv), m.apply(m.weights(rho), xv)) <= 1e-13
    full = m.run(method="splu")
    u2, info2 = R.solve(rtol=1e-11)
    assert info2.rel_residual <= 1e-11
    assert rel(u2.cpu().numpy()[0][sd], full["u"][0][sd]) <= 1e-6
    # Sec. 6.1: with Emin = 1e-9 E0 the suppression barely changes the compliance
    assert abs(ref["c"][0] - full["c"][0]) <= 1e-6 * full["c"][0]
    R.close()


def test_errors_and_the_trivial_selections():
    import torch

    p = workloads.cantilever(8, 4, 4, seed=1, mg_levels=2)
    R = Run(p, FP32X2)
    T = R.T
    with pytest.raises(T.TosolveError):
        T.tosolve_fix_variables(R.h, None, LO, HI, EPS)  # no densities yet
    R.set_densities()
    for lo, hi, eps in ((0.5, 0.4, 0.0), (-1.0, 0.9, 0.0), (0.0, 1.5, 0.0), (0.0, 0.9, -1.0)):
        with pytest.raises(T.TosolveError):
            T.tosolve_fix_variables(R.h, None, lo, hi, eps)
    # x ~ U[0.01, 1]: nothing is void, nothing suppressed
    assert T.tosolve_fix_variables(R.h, None, LO, HI, EPS) == 0
    assert T.tosolve_free_dofs(R.h) == p.nfree
    # all void: every node is suppressed, the supports included
    R.set_densities(torch.zeros_like(R.x))
    fixed = torch.zeros(p.x.size, dtype=torch.uint8, device=R.dev)
    nsup = T.tosolve_fix_variables(R.h, None, LO, HI, EPS, fixed)
    assert nsup == p.nfree and T.tosolve_free_dofs(R.h) == 0
    assert (fixed.cpu().numpy() == fix.VOID).all()
    R.close()


@pytest.mark.parametrize("prec", [FP64, FP32, FP32X2])
def test_tile_skipping_is_exact(prec):
    """After the suppression the level-0 stencil kernels skip the tiles whose
    DOFs are all fixed.  Level 0 then applies, bit for bit, what a handle
    created with the suppressed DOFs among its supports applies (it reads
    every tile); the coarse levels keep the supports alone and apply what an
    unsuppressed handle applies."""
    import torch

    p = _structured(1, 2, (32, 16, 16), 1.0, seed=4, levels=4)
    m = fe.Model(p)
    rho = m.densities(p.x)
    fx = fix.fixed_elements(p, fix.element_class(p, rho, None, LO, HI, EPS))
    sup = fix.suppressed_nodes(p, fx)
    q = fix.suppressed_problem(p, sup)
    A = Run(p, prec)
    A.set_densities()
    nsup = A.T.tosolve_fix_variables(A.h, None, LO, HI, EPS)
    assert nsup == p.nfree - q.nfree and nsup > p.nfree // 4
    B = Run(q, prec)
    B.set_densities()
    U = Run(p, prec)
    U.set_densities()
    rng = np.random.default_rng(9)
    for level in range(A.T.tosolve_level_count(A.h) - 1):
        ref = B if level == 0 else U
        xv = rng.normal(size=3 * int(np.prod(_dims(A, level))))
        for pr in (FP64, FP32, FP32X2):
            try:
                ya = A.apply(level, pr, xv)
            except A.T.TosolveError:  # no operator of that precision on this level
                with pytest.raises(A.T.TosolveError):
                    ref.apply(level, pr, xv)
                continue
            assert np.array_equal(ya, ref.apply(level, pr, xv)), (level, pr)
    u, info = A.solve(rtol=1e-8)
    assert info.rel_residual <= 1e-8
    for R in (A, B, U):
        R.close()
def _dims(R, level):
    import ctypes as C

    dims = (C.c_int * 3)()
    R.T._lib.tosolve_level_dims(R.h, level, dims)
    return dims[0], dims[1], dims[2]
