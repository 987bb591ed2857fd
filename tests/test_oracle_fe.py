"""Pins of the oracle's assembled solve, compliance and gradient (oracle/fe.py).

  * rigid-body modes are in the kernel of the unconstrained assembled K for
    any densities (superposition of PSD element matrices, Eq. matrixK_mr);
  * patch test: with uniform density and a linear displacement field imposed
    on the boundary, the solve reproduces the field at every interior node
    (k = 1, 2) -- fixes assembly, DOF numbering and the Dirichlet treatment;
  * uniform density: c(rho) = c(1) E0 / w(rho) exactly (K linear in w);
  * energy identities f^T u = u^T K u and sum_{e,i} w_{e,i} s_{e,i} = c
    (Section 3.4);
  * dense Cholesky, SuperLU and CG agree on small meshes;
  * the gradient of Section 3.4 matches central finite differences of the
    compliance through the filter, and d c / d rho <= 0 everywhere.
"""
import numpy as np
import pytest

import workloads
from oracle import fe, fem, mesh


def _model(nx=4, ny=2, nz=2, k=1, n=1, rmin=0.0, seed=0, **kw):
    p = workloads.cantilever(nx, ny, nz, degree=k, n_mr=n, rmin=rmin, seed=seed, **kw)
    return p, fe.Model(p)


@pytest.mark.parametrize("k,n", [(1, 1), (1, 2), (2, 1)])
def test_rigid_modes_in_kernel_of_assembled_K(k, n):
    p, m = _model(3, 2, 2, k, n, seed=3)
    K = m.assemble(m.weights(m.densities(p.x)))
    X = mesh.node_coords(p.nx, p.ny, p.nz, k)
    modes = []
    for t in range(3):
        v = np.zeros(p.ndof); v[t::3] = 1.0; modes.append(v)
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    for a, b in ((x, y), (y, z), (z, x)):
        v = np.zeros(p.ndof)
        # rotation in the (a, b) plane: (-b, a)
        ia = {id(x): 0, id(y): 1, id(z): 2}[id(a)]
        ib = {id(x): 0, id(y): 1, id(z): 2}[id(b)]
        v[ia::3] = -b; v[ib::3] = a
        modes.append(v)
    for v in modes:
        assert np.abs(K @ v).max() < 1e-12 * np.abs(K).max() * max(1.0, np.abs(v).max())


@pytest.mark.parametrize("k", [1, 2])
def test_patch_test_reproduces_linear_field(k):
    p, m = _model(3, 3, 2, k, 1, density="solid")
    w = m.weights(m.densities(p.x))
    K = m.assemble(w)
    X = mesh.node_coords(p.nx, p.ny, p.nz, k)
    G = np.array([[1e-3, 2e-3, -1e-3], [0.5e-3, -2e-3, 1e-3], [3e-3, 1e-3, 2e-3]])
    exact = (X @ G.T).reshape(-1)  # u(x) = G x, DOF-interleaved
    Lx, Ly, Lz = p.lattice
    ii = np.arange(p.nnodes)
    i, j, l = ii % Lx, (ii // Lx) % Ly, ii // (Lx * Ly)
    bnd = (i == 0) | (i == Lx - 1) | (j == 0) | (j == Ly - 1) | (l == 0) | (l == Lz - 1)
    fixed = np.repeat(bnd, 3)
    free = ~fixed
    assert free.sum() > 0
    Kff = K[free][:, free].toarray()
    rhs = -K[free][:, fixed] @ exact[fixed]
    uf = np.linalg.solve(Kff, rhs)
    np.testing.assert_allclose(uf, exact[free], rtol=0, atol=1e-14)


def test_uniform_density_scaling():
    p, m = _model(4, 2, 2, 1, 1, density="solid")
    f = p.f[0]
    u1 = m.solve(m.weights(np.ones(p.x.size)), f)
    c1 = m.compliance(f, u1, p.mask)
    rho = np.full(p.x.size, 0.37)
    w = fe.simp_weights(0.37, p.E0, p.Emin, p.penal)
    u = m.solve(m.weights(rho), f)
    c = m.compliance(f, u, p.mask)
    assert abs(c - c1 * p.E0 / w) < 1e-12 * c


@pytest.mark.parametrize("k,n,rmin", [(1, 1, 0.0), (1, 2, 1.0), (2, 2, 0.8)])
def test_energy_identities(k, n, rmin):
    p, m = _model(4, 2, 2, k, n, rmin=rmin, seed=5)
    out = m.run()
    u, c = out["u"][0], out["c"][0]
    K = m.assemble(out["w"])
    assert abs(u @ (K @ u) - c) < 1e-11 * c
    s = m.subcell_energies(u)
    assert abs((out["w"] * s).sum() - c) < 1e-11 * c
    assert (out["g_rho"] <= 0).all()


def test_direct_solvers_agree():
    p, m = _model(4, 3, 2, 1, 2, rmin=0.9, seed=7, Emin=1e-6)
    w = m.weights(m.densities(p.x))
    f = p.f[0]
    ud = m.solve(w, f, method="dense")
    us = m.solve(w, f, method="splu")
    uc = m.solve(w, f, method="cg", tol=1e-14)
    assert np.linalg.norm(us - ud) <= 1e-11 * np.linalg.norm(ud)
    assert np.linalg.norm(uc - ud) <= 1e-8 * np.linalg.norm(ud)


def test_gradient_matches_central_differences():
    p, m = _model(4, 2, 2, 1, 2, rmin=0.75, seed=11, Emin=1e-3)
    out = m.run()
    g = out["g_x"]
    rng = np.random.default_rng(0)
    for kidx in rng.choice(p.x.size, 6, replace=False):
        h = 1e-5
        xp, xm = p.x.copy(), p.x.copy()
        xp[kidx] += h
        xm[kidx] -= h
        cp = m.run(xp)["c"][0]
        cm = m.run(xm)["c"][0]
        fd = (cp - cm) / (2 * h)
        assert abs(fd - g[kidx]) <= 1e-6 * abs(g[kidx]) + 1e-12


def test_multiple_load_cases_sum_gradient():
    p, m = _model(4, 2, 2, 1, 1, seed=2)
    f2 = np.zeros_like(p.f)
    Lx, Ly, Lz = p.lattice
    nd = (Lx - 1) + Lx * (0 + Ly * (Lz - 1))
    f2[0, 3 * nd + 1] = 1.0
    p.f = np.concatenate([p.f, f2])
    out = m.run()
    g_sum = np.zeros_like(out["g_x"])
    for r in range(2):
        q, mm = _model(4, 2, 2, 1, 1, seed=2)
        q.f = p.f[r: r + 1]
        o = mm.run()
        assert abs(o["c"][0] - out["c"][r]) < 1e-12 * o["c"][0]
        g_sum += o["g_x"]
    np.testing.assert_allclose(out["g_x"], g_sum, rtol=1e-12, atol=0)
