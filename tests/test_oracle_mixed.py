"""Pins of the mixed trilinear / triquadratic oracle (oracle/mixed.py).

Each pin fixes the coupling rule against something outside it: the plain
trilinear and triquadratic oracles (all elements of one kind), the exact
trilinear element matrix, a linear displacement field, and the energy
identities.
"""
import numpy as np
import pytest

import workloads
from oracle import fe, fem, mesh, mixed


def _bridge(degree, n=1, seed=1, shape=(4, 2, 2)):
    return workloads.bridge(*shape, degree=degree, n_mr=n, seed=seed)


def test_all_trilinear_equals_the_trilinear_problem():
    q = workloads.with_mixed_degree(_bridge(2, n=2), 1.0, 0)
    p1 = _bridge(1, n=2)
    r1 = fe.Model(p1).run(method="dense")
    rq = mixed.MixedModel(q).run(method="dense")
    Lx, Ly, _ = q.lattice
    vert = [2 * i + Lx * (2 * j + Ly * 2 * l) for l in range(3) for j in range(3) for i in range(5)]
    uv = rq["u"][0].reshape(-1, 3)[vert].reshape(-1)
    assert np.abs(uv - r1["u"][0]).max() <= 1e-12 * np.abs(r1["u"][0]).max()
    assert abs(rq["c"][0] - r1["c"][0]) <= 1e-12 * r1["c"][0]
    assert np.abs(rq["g_x"] - r1["g_x"]).max() <= 1e-11 * np.abs(r1["g_x"]).max()


def test_all_quadratic_is_the_quadratic_problem():
    p2 = _bridge(2, n=2, seed=3)
    q = workloads.with_mixed_degree(p2, 0.0, 0)
    assert not mixed.slaved_nodes(q).any()
    r2 = fe.Model(p2).run(method="dense")
    rq = mixed.MixedModel(q).run(method="dense")
    np.testing.assert_allclose(rq["u"], r2["u"], rtol=0, atol=1e-13 * np.abs(r2["u"]).max())
    np.testing.assert_allclose(rq["g_x"], r2["g_x"], rtol=1e-12)


def test_embedded_trilinear_element_has_the_trilinear_matrix():
    q = workloads.with_mixed_degree(_bridge(2, shape=(1, 1, 1)), 1.0, 0)
    m = mixed.MixedModel(q)
    K = m.assemble(np.ones((1, 1)))
    Kr = (m.T.T @ K @ m.T).toarray()
    Lx, Ly, _ = q.lattice
    # trilinear local node a = ix + 2 (iy + 2 iz) sits at lattice (2ix, 2iy, 2iz)
    dofs = []
    for iz in range(2):
        for iy in range(2):
            for ix in range(2):
                node = 2 * ix + Lx * (2 * iy + Ly * 2 * iz)
                dofs += [3 * node, 3 * node + 1, 3 * node + 2]
    K1 = fem.subcell_stiffness(1, 1, q.nu)[0]
    np.testing.assert_allclose(Kr[np.ix_(dofs, dofs)], K1, rtol=0, atol=1e-14 * np.abs(K1).max())
    # the slaved rows and columns are empty
    slv = np.repeat(mixed.slaved_nodes(q), 3)
    assert np.abs(Kr[slv]).max() == 0.0 and np.abs(Kr[:, slv]).max() == 0.0


def test_mixed_patch_test_reproduces_linear_field():
    p = workloads.bridge(3, 3, 2, degree=2, n_mr=1, seed=2)
    q = workloads.with_mixed_degree(p, 0.5, 7)
    assert 0 < q.elem_q1.sum() < q.elem_q1.size
    m = mixed.MixedModel(q)
    K = m.assemble(m.weights(np.full(q.x.size, 0.6)))
    X = mesh.node_coords(q.nx, q.ny, q.nz, 2)
    G = np.array([[1e-3, 2e-3, -1e-3], [0.5e-3, -2e-3, 1e-3], [3e-3, 1e-3, 2e-3]])
    exact = (X @ G.T).reshape(-1)
    Lx, Ly, Lz = q.lattice
    ii = np.arange(q.nnodes)
    i, j, l = ii % Lx, (ii // Lx) % Ly, ii // (Lx * Ly)
    bnd = np.repeat((i == 0) | (i == Lx - 1) | (j == 0) | (j == Ly - 1) | (l == 0) | (l == Lz - 1), 3)
    slv = m.slaved
    free = ~bnd & ~slv
    # u = T u_r with u_r = exact on boundary vertices / free nodes
    Kr = (m.T.T @ K @ m.T).tocsr()
    known = bnd & ~slv
    ur = np.zeros(q.ndof)
    ur[known] = exact[known]
    rhs = -(Kr[free][:, known] @ ur[known])
    ur[free] = np.linalg.solve(Kr[free][:, free].toarray(), rhs)
    u = m.T @ ur
    np.testing.assert_allclose(u, exact, rtol=0, atol=1e-13)


@pytest.mark.parametrize("frac,seed", [(0.5, 1), (0.25, 4)])
def test_mixed_energy_identities(frac, seed):
    q = workloads.with_mixed_degree(_bridge(2, n=2, seed=seed, shape=(4, 2, 2)), frac, seed)
    m = mixed.MixedModel(q)
    out = m.run(method="dense")
    u, c = out["u"][0], out["c"][0]
    K = m.assemble(out["w"])
    assert abs(u @ (K @ u) - c) < 1e-11 * c
    assert abs((out["w"] * m.subcell_energies(u)).sum() - c) < 1e-11 * c
    assert (out["g_rho"] <= 1e-15).all()
