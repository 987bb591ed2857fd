"""Pins of the oracle's density filter / projection (oracle/filt.py).

  * a worked 3-cell example from Eq. filter_weights (tests/golden), which
    fixes sigma = r/3, the inclusive cut-off and the boundary truncation;
  * the inclusive ball of radius 3 cells holds exactly 123 lattice offsets
    (integer points with i^2+j^2+k^2 <= 9), fixing the distance units;
  * rows of H sum to one (normalisation by w_i), H^T preserves sums, and in
    the interior H is symmetric (equal w_i);
  * r = 0 is the identity (no filter).
"""
import json
import os

import numpy as np
import pytest

from oracle import filt

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_worked_three_cell_example():
    g = json.load(open(os.path.join(GOLDEN, "filter_line3.json")))
    H = filt.filter_matrix(tuple(g["shape_zyx"]), g["n_mr"], g["rmin"])
    np.testing.assert_allclose(H @ np.array(g["x"]), g["rho"], rtol=0, atol=1e-15)


def test_ball_of_radius_three_cells_has_123_offsets():
    offs, w = filt.filter_offsets(2, 1.5)  # r * n = 3 cells, ties at 9 included
    assert len(offs) == 123
    assert (offs ** 2).sum(axis=1).max() == 9
    offs, _ = filt.filter_offsets(4, 0.6)  # (r n)^2 = 5.76: no tie
    assert (offs ** 2).sum(axis=1).max() == 5


def test_rows_sum_to_one_and_transpose_preserves_sums():
    shape = (6, 5, 9)
    H = filt.filter_matrix(shape, 2, 1.5)
    np.testing.assert_allclose(np.asarray(H.sum(axis=1)).ravel(), 1.0, atol=1e-14)
    g = np.random.default_rng(1).normal(size=H.shape[0])
    assert abs((H.T @ g).sum() - g.sum()) < 1e-12
    # interior block: symmetric weights
    Dz, Dy, Dx = shape
    idx = lambda x, y, z: x + Dx * (y + Dy * z)
    a, b = idx(4, 2, 3), idx(5, 2, 3)
    Hd = H.toarray()
    assert Hd[a, b] > 0 and abs(Hd[a, b] - Hd[b, a]) < 1e-15


def test_zero_radius_is_identity():
    H = filt.filter_matrix((2, 3, 4), 1, 0.0)
    assert np.array_equal(H.toarray(), np.identity(24))


def test_projection_equals_filter_on_the_density_grid():
    from oracle import filt

    P = filt.projection_matrix(3, 2, 2, 2, 2, 1.5)
    F = filt.filter_matrix((4, 4, 6), 2, 1.5)
    assert abs(P - F).max() == 0.0


@pytest.mark.parametrize("n,d,r", [(3, 2, 0.6), (2, 1, 0.9), (4, 2, 0.6)])
def test_projection_rows_are_weighted_averages(n, d, r):
    from oracle import filt

    P = filt.projection_matrix(3, 2, 2, n, d, r)
    assert P.shape == (n ** 3 * 12, d ** 3 * 12)
    np.testing.assert_allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, rtol=0, atol=1e-15)
    assert P.min() >= 0.0


def test_projection_with_a_small_radius_takes_the_containing_design_cell():
    """d = 1, n = 2, r = 0.5: a density cell's own element centre is
    sqrt(3)/4 = 0.433 away, every other element centre at least 0.83."""
    from oracle import filt

    nx, ny, nz = 3, 2, 2
    P = filt.projection_matrix(nx, ny, nz, 2, 1, 0.5).toarray()
    for c in range(P.shape[0]):
        cx, cy, cz = c % 6, (c // 6) % 4, c // 24
        e = cx // 2 + nx * (cy // 2 + ny * (cz // 2))
        row = np.zeros(P.shape[1])
        row[e] = 1.0
        np.testing.assert_array_equal(P[c], row)


def test_gradient_through_a_coarser_design_grid_matches_finite_differences():
    import workloads
    from oracle import fe

    p = workloads.with_design_grid(workloads.cantilever(3, 2, 2, n_mr=2, rmin=0.8, seed=1), 1, 4,
                                   lo=0.3, hi=0.9)
    m = fe.Model(p)
    out = m.run(method="dense")
    g = out["g_x"]
    assert g.size == p.x.size == 12
    h = 1e-6
    for j in range(0, 12, 3):
        xp, xm = p.x.copy(), p.x.copy()
        xp[j] += h * p.x[j]
        xm[j] -= h * p.x[j]
        fd = (m.run(x=xp, method="dense")["c"][0] - m.run(x=xm, method="dense")["c"][0]) / (2 * h * p.x[j])
        assert abs(fd - g[j]) <= 1e-6 * abs(g[j])
