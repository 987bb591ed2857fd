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
