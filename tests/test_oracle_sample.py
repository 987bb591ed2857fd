"""The sampled oracle (oracle/sample.py) against the whole-mesh oracle on
meshes small enough for both: every sampled row or cell must equal the
corresponding entry of the assembled computation to FP64 rounding."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import fe, mixed, sample


@pytest.mark.parametrize("k,n,rmin", [(1, 2, 1.0), (2, 3, 0.7), (1, 1, 0.0)])
def test_sampled_rows_and_cells_equal_the_whole_mesh(k, n, rmin):
    p = workloads.cantilever(4, 3, 2, degree=k, n_mr=n, rmin=rmin, seed=3)
    m = fe.Model(p)
    S = sample.Sampler(p)
    rng = np.random.default_rng(0)
    u = rng.normal(size=p.ndof)
    rho = m.densities(p.x)
    y = m.apply(m.weights(rho), u).reshape(-1, 3)
    nodes = list(range(p.nnodes))
    ys = S.apply_rows(p.x, u, nodes)
    assert np.abs(ys - y).max() <= 1e-13 * np.abs(y).max()
    cells = rng.choice(p.x.size, size=12, replace=False)
    np.testing.assert_allclose([S.rho(p.x, c) for c in cells], rho[cells], rtol=1e-14)
    g = m.density_gradient(rho, m.subcell_energies(u))
    gx = m.design_gradient(g)
    np.testing.assert_allclose([S.drho(p.x, u, c) for c in cells], g[cells], rtol=1e-12)
    np.testing.assert_allclose([S.dx(p.x, u, c) for c in cells], gx[cells], rtol=1e-12)


def test_sampled_rows_of_a_mixed_mesh():
    q = workloads.with_mixed_degree(workloads.bridge(4, 2, 2, degree=2, n_mr=2, seed=1), 0.5, 5)
    m = mixed.MixedModel(q)
    S = sample.Sampler(q)
    u = np.random.default_rng(1).normal(size=q.ndof)
    w = m.weights(m.densities(q.x))
    A = (m.T.T @ m.assemble(w) @ m.T).tocsr()
    held = (q.mask != 0) | m.slaved
    keep = sp.diags((~held).astype(float))
    A = keep @ A @ keep + sp.diags(held.astype(float))
    y = (A @ u).reshape(-1, 3)
    ys = S.apply_rows(q.x, u, list(range(q.nnodes)))
    assert np.abs(ys - y).max() <= 1e-13 * np.abs(y).max()


def test_gradient_rounding_scale_bounds_the_error():
    """drho_scale bounds |dc/drho| (triangle inequality) and, for a
    displacement that is a large rigid translation plus a small strain, the
    FP64 error of drho against the exact rational value of the same
    quadratic form stays below 1e-12 of it (while the relative error may not)."""
    from fractions import Fraction

    p = workloads.cantilever(3, 2, 2, degree=1, n_mr=2, seed=5)
    S = sample.Sampler(p)
    rng = np.random.default_rng(2)
    u = np.tile([3e5, -2e5, 1e5], p.nnodes) + 1e-3 * rng.normal(size=p.ndof)
    for c in range(p.x.size):
        d, s = S.drho(p.x, u, c), S.drho_scale(p.x, u, c)
        assert abs(d) <= s * (1 + 1e-12)
        n = S.n
        cx, cy, cz = c % S.Dx, (c // S.Dx) % S.Dy, c // (S.Dx * S.Dy)
        en = S._elem_nodes(cx // n, cy // n, cz // n)
        i = (cx % n) + n * ((cy % n) + n * (cz % n))
        ue = [Fraction(float(u[3 * m + q])) for m in en for q in range(3)]
        K = S.K[i]
        quad = sum(ue[a] * Fraction(float(K[a, b])) * ue[b] for a in range(24) for b in range(24))
        r = S.rho(p.x, c)
        exact = -p.penal * r ** (p.penal - 1.0) * (p.E0 - p.Emin) * float(quad)
        assert abs(d - exact) <= 1e-12 * s


def test_row_rounding_scale_bounds_the_rows():
    p = workloads.cantilever(4, 3, 2, degree=2, n_mr=2, rmin=0.7, seed=3)
    S = sample.Sampler(p)
    u = np.random.default_rng(4).normal(size=p.ndof)
    nodes = list(range(0, p.nnodes, 7))
    y = S.apply_rows(p.x, u, nodes)
    sc = S.apply_rows_scale(p.x, u, nodes)
    assert (sc >= np.abs(y) * (1 - 1e-14)).all() and (sc > 0).all()
    # a displacement with one sign on free DOFs and a diagonal-only check:
    # the scale of a row is at least its diagonal term
    m = fe.Model(p)
    K = m.assemble(m.weights(m.densities(p.x))).tocsr()
    for q, nd in enumerate(nodes):
        for c in range(3):
            d = 3 * nd + c
            if p.mask[d] == 0:
                assert sc[q, c] >= abs(K[d, d] * u[d]) * (1 - 1e-14)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_subcell_rounding_scale(n):
    """The rounding scale of the stacked form: with one subcell per element
    it is the element scale sum_j |K_ij u_j| (|w K| = w |K|); with more it
    bounds that scale from above (triangle inequality over subcells); the
    vectorised whole-mesh version equals the per-node loops of the sampler."""
    p = workloads.bridge(4, 2, 2, degree=2, n_mr=n, seed=5)
    m = fe.Model(p)
    S = sample.Sampler(p)
    u = np.random.default_rng(7).normal(size=p.ndof)
    w_e = m.weights(m.densities(p.x))
    whole = m.subcell_scale(w_e, u).reshape(-1, 3)
    nodes = list(range(p.nnodes))
    loops = S.apply_rows_subcell_scale(p.x, u, nodes)
    np.testing.assert_allclose(loops, whole, rtol=1e-13)
    elem = S.apply_rows_scale(p.x, u, nodes)
    if n == 1:
        np.testing.assert_allclose(whole, elem, rtol=1e-13)
    else:
        assert (whole >= elem * (1 - 1e-13)).all()
        assert (whole > elem * (1 + 1e-6)).any()  # cancellation between subcells exists
    y = m.apply(w_e, u).reshape(-1, 3)
    assert (whole >= np.abs(y) * (1 - 1e-13)).all()


@pytest.mark.parametrize("k,n", [(1, 2), (2, 3), (3, 1)])
def test_rigid_projector_keeps_the_subcell_products(k, n):
    """The deflation behind the tensor-core operand: P is an orthogonal
    projector of rank d - 6 that every subcell matrix sees as the identity
    (K^(e_i) P = K^(e_i): rigid motions carry no strain), and it removes
    translations and rotations exactly."""
    from oracle import fem

    P = fe.rigid_projector(k)
    d = 3 * (k + 1) ** 3
    np.testing.assert_allclose(P @ P, P, atol=1e-13)
    np.testing.assert_allclose(P, P.T, atol=1e-14)
    assert round(np.trace(P)) == d - 6
    K = fem.subcell_stiffness(k, n, 0.3)
    for Ki in K:
        np.testing.assert_allclose(Ki @ P, Ki, atol=1e-12 * np.abs(Ki).max())
    pos = np.array([[-1.0 + 2.0 * ax / k, -1.0 + 2.0 * ay / k, -1.0 + 2.0 * az / k]
                    for az in range(k + 1) for ay in range(k + 1) for ax in range(k + 1)])
    om, t = np.array([0.3, -1.1, 0.7]), np.array([2.0, -0.5, 1.5])
    rigid = (t + np.cross(om, pos)).reshape(-1)
    assert np.abs(P @ rigid).max() <= 1e-13


def test_deflated_scale_equals_between_oracle_forms():
    p = workloads.bridge(4, 2, 2, degree=2, n_mr=2, seed=5)
    m = fe.Model(p)
    S = sample.Sampler(p)
    u = np.random.default_rng(8).normal(size=p.ndof)
    w_e = m.weights(m.densities(p.x))
    whole = m.subcell_scale(w_e, u, deflate=True).reshape(-1, 3)
    loops = S.apply_rows_subcell_scale(p.x, u, list(range(p.nnodes)), deflate=True)
    np.testing.assert_allclose(loops, whole, rtol=1e-12)
    wm = m.subcell_scale(w_e, u, deflate=True, elem_max=True).reshape(-1, 3)
    lm = S.apply_rows_subcell_scale(p.x, u, list(range(p.nnodes)), deflate=True, elem_max=True)
    np.testing.assert_allclose(lm, wm, rtol=1e-12)
    free = (p.mask == 0).reshape(-1, 3)
    assert (wm[free] >= whole[free] * (1 - 1e-13)).all()  # the element max bounds every entry
    # a rigid displacement has a zero deflated scale away from the supports
    pos = np.array([[i, j, l] for l in range(p.lattice[2]) for j in range(p.lattice[1])
                    for i in range(p.lattice[0])], dtype=float)
    rigid = (np.array([1.0, 2.0, 3.0]) + np.cross([0.2, 0.1, -0.3], pos)).reshape(-1)
    free_elems = np.all(p.mask[m.edofs] == 0, axis=1)
    z = m.subcell_scale(w_e, rigid, deflate=True)
    touched = np.unique(m.edofs[free_elems])
    only_free = np.setdiff1d(touched, np.unique(m.edofs[~free_elems]))
    assert np.abs(z[only_free]).max() <= 1e-12 * np.abs(rigid).max()


def test_mixed_subcell_scale_bounds_the_rows():
    """The rounding scale of a mixed mesh's stacked form bounds each row of
    the mixed operator (T^T K T with slaved identity rows) and, with one
    subcell per element, equals the element scale of the unslaved rows of
    triquadratic elements away from trilinear ones."""
    p = workloads.with_mixed_degree(workloads.bridge(4, 2, 2, degree=2, n_mr=2, seed=5), 0.5, 3)
    S = sample.Sampler(p)
    u = np.random.default_rng(6).normal(size=p.ndof)
    nodes = list(range(p.nnodes))
    y = S.apply_rows(p.x, u, nodes)
    sc = S.apply_rows_subcell_scale(p.x, u, nodes)
    assert (sc >= np.abs(y) * (1 - 1e-13)).all()
    scd = S.apply_rows_subcell_scale(p.x, u, nodes, deflate=True)
    scm = S.apply_rows_subcell_scale(p.x, u, nodes, deflate=True, elem_max=True)
    assert (scm >= scd * (1 - 1e-13)).all()
    # a rigid displacement of the free nodes: the deflated scale vanishes
    # in rows whose elements have no support
    Lx, Ly, Lz = p.lattice
    pos = np.array([[i, j, l] for l in range(Lz) for j in range(Ly) for i in range(Lx)], dtype=float)
    rigid = (np.array([1.0, -2.0, 0.5]) + np.cross([0.3, 0.2, -0.1], pos)).reshape(-1)
    free_nodes = [nd for nd in nodes if not p.mask[3 * nd] and not S.slv[nd]
                  and all(not p.mask[3 * m] for e in S.elements_of(nd) for m in S._elem_nodes(*e))]
    if free_nodes:
        zd = S.apply_rows_subcell_scale(p.x, rigid, free_nodes, deflate=True)
        assert np.abs(zd).max() <= 1e-12 * np.abs(rigid).max()
