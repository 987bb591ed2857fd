"""The seeded input generators against the recipe they implement.

`workloads/` builds the inputs both sides receive (Dirichlet masks, nodal
loads, design fields) and none of the method's arithmetic.  These tests pin
it to the stated recipe: supports where the structure is held, loads whose
totals the load pattern fixes (a unit edge load, a unit pressure over the
top face, consistent Newton-Cotes nodal weights), design fields in their
ranges, the resampling of the smooth field, the trilinear fraction of the
mixed mesh, and the batch's size distribution and load cases.
"""
import numpy as np
import pytest

import workloads as W


def _nodes(p):
    Lx, Ly, Lz = p.lattice
    n = np.arange(Lx * Ly * Lz)
    return n % Lx, (n // Lx) % Ly, n // (Lx * Ly)


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_cantilever_supports_and_unit_edge_load(degree):
    p = W.cantilever(6, 3, 4, degree=degree, n_mr=2, seed=1)
    i, j, l = _nodes(p)
    Lx, Ly, Lz = p.lattice
    fixed = p.mask.reshape(-1, 3)
    assert (fixed[i == 0] == 1).all() and (fixed[i != 0] == 0).all()  # the face x = 0, all components
    f = p.f[0].reshape(-1, 3)
    assert f[:, :2].sum() == 0.0 and f[:, 2].sum() == pytest.approx(-1.0, abs=1e-15)  # unit total, downward
    loaded = f[:, 2] != 0.0
    assert (i[loaded] == Lx - 1).all() and (l[loaded] == 0).all()  # the edge x = nx, z = 0
    assert loaded.sum() == Ly  # every node of that edge, consistent weights all positive
    # consistent weights: the ends carry the first Newton-Cotes weight of one element
    nc = {1: 1 / 2, 2: 1 / 6, 3: 1 / 8}[degree]
    end = f[(i == Lx - 1) & (j == 0) & (l == 0), 2]
    assert end[0] == pytest.approx(-nc / p.ny)
    assert p.x.size == (2 * 6) * (2 * 3) * (2 * 4) and 0.01 <= p.x.min() and p.x.max() <= 1.0


def test_bridge_corners_and_top_pressure():
    p = W.bridge(8, 4, 3, degree=2, n_mr=3, seed=0)
    i, j, l = _nodes(p)
    Lx, Ly, Lz = p.lattice
    fixed = p.mask.reshape(-1, 3).all(axis=1)
    corners = np.isin(i, (0, Lx - 1)) & np.isin(j, (0, Ly - 1)) & (l == 0)
    assert (fixed == corners).all() and corners.sum() == 4 and p.mask.sum() == 12
    f = p.f[0].reshape(-1, 3)
    assert f[:, :2].sum() == 0.0
    assert f[:, 2].sum() == pytest.approx(-8 * 4, rel=1e-14)  # pressure 1 on the 8 x 4 top face
    assert (f[l != Lz - 1] == 0.0).all()
    # tensor Newton-Cotes on the degree-2 top face: corner 1/36, mid-edge 4/36, face centre 16/36
    top = f[:, 2].reshape(Lz, Ly, Lx)[-1]
    assert top[0, 0] == pytest.approx(-1 / 36) and top[0, 1] == pytest.approx(-4 / 36)
    assert top[1, 1] == pytest.approx(-16 / 36) and top[0, 2] == pytest.approx(-2 / 36)


def test_mixed_bridge_as_benchmarked():
    """The benchmark's C2 recipe: 64x32x32 on the degree-2 lattice, n = 3,
    a seeded half trilinear (fraction 0.5, seed 11)."""
    p = W.with_mixed_degree(W.bridge(64, 32, 32, degree=2, n_mr=3, seed=0), 0.5, 11)
    E = 64 * 32 * 32
    assert p.elem_q1.shape == (E,) and int(p.elem_q1.sum()) == 32844  # 32,692 triquadratic
    assert abs(p.elem_q1.mean() - 0.5) < 5 * np.sqrt(0.25 / E)
    assert p.x.size == 192 * 96 * 96 and 0.01 <= p.x.min() and p.x.max() <= 1.0
    assert p.ndof == 3 * 129 * 65 * 65 and p.nfree == 1635063  # all nodes but the 4 pinned corners
    assert p.f.sum() == pytest.approx(-64 * 32, rel=1e-14)
    q = W.with_mixed_degree(W.bridge(64, 32, 32, degree=2, n_mr=3, seed=0), 0.5, 11)
    assert np.array_equal(p.elem_q1, q.elem_q1) and np.array_equal(p.x, q.x)  # seeded


def test_smooth_field_resampling():
    rng = np.random.default_rng(0)
    # same resolution: the cell-centred resampling is the identity
    c = rng.uniform(size=(3, 4, 5))
    out = c
    for axis, n in enumerate(c.shape):
        out = W._upsample_axis(out, axis, n)
    np.testing.assert_array_equal(out, c)
    # linear data stays linear between the first and last coarse centres
    a = np.arange(4, dtype=np.float64)
    up = W._upsample_axis(a, 0, 16)
    src = (np.arange(16) + 0.5) * (4 / 16) - 0.5
    np.testing.assert_allclose(up, np.clip(src, 0, 3), atol=1e-15)
    # the C1 field: clipped to [0.001, 1], 96 x 48 x 48 cells
    p = W.cantilever(48, 24, 24, n_mr=2, rmin=1.5, density="smooth", seed=0)
    assert p.x.size == 96 * 48 * 48 and p.x.min() >= 0.001 and p.x.max() <= 1.0
    assert p.nfree == 90000


def test_batch_of_64_as_benchmarked():
    b = W.batched_instances(64, 2024, mult=16)
    assert len(b) == 64
    assert all(32 <= p.nx <= 128 and p.nx % 16 == 0 and p.ny == p.nz == p.nx // 2 for p in b)
    assert sum(p.nrhs for p in b) == 116 and all(1 <= p.nrhs <= 3 for p in b)
    assert sum(p.nfree * p.nrhs for p in b) == 62419200 and max(p.nfree for p in b) == 1622400
    for p in b[:8]:
        i, j, l = _nodes(p)
        Lx, Ly, Lz = p.lattice
        for r in range(p.nrhs):
            f = p.f[r].reshape(-1, 3)
            assert np.linalg.norm(f.sum(axis=0)) == pytest.approx(1.0, rel=1e-12)  # unit total load
            on = np.abs(f).sum(axis=1) > 0
            assert (i[on] == Lx - 1).all()  # on the face x = nx ...
            edge_y = (l[on] == 0).all() or (l[on] == Lz - 1).all()
            edge_z = (j[on] == 0).all() or (j[on] == Ly - 1).all()
            assert edge_y or edge_z  # ... along one of its edges
            d = f[on] / np.linalg.norm(f[on], axis=1, keepdims=True)
            np.testing.assert_allclose(d, np.broadcast_to(d[0], d.shape), atol=1e-12)  # one direction


def test_serendipity_and_design_grid_variants():
    p = W.cantilever(4, 2, 3, degree=2, n_mr=2, seed=0)  # edge load: no face-centre loads
    s = W.with_serendipity(p)
    with pytest.raises(ValueError):  # a top pressure loads face centres the element does not have
        W.with_serendipity(W.bridge(4, 2, 3, degree=2, n_mr=2, seed=0))
    i, j, l = _nodes(p)
    interior = (i % 2 == 1).astype(int) + (j % 2 == 1) + (l % 2 == 1) >= 2  # face and cell centres
    held = s.mask.reshape(-1, 3).all(axis=1)
    assert (held[interior]).all() and s.family == "serendipity"
    assert (s.mask.reshape(-1, 3)[~interior] == p.mask.reshape(-1, 3)[~interior]).all()
    g = W.with_design_grid(p, 1, 3)
    assert g.d_mr == 1 and g.x.size == 4 * 2 * 3 and g.n_mr == 2
    with pytest.raises(ValueError):
        W.with_design_grid(p, 3, 0)
