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
