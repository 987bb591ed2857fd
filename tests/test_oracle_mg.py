"""Pins of the oracle's multigrid (oracle/mg.py).

  * Galerkin identity: for Lagrange Q1 with nested meshes the coarse
    operator re-discretised from the density field equals P^T A P on the
    free DOFs (clamped face: the coarse space is a subspace of the fine one);
    this pins the coarse element tables, the density-cell bookkeeping of the
    coarse levels and the interpolation P at once;
  * P reproduces trilinear fields exactly;
  * a cycle with eta1 = eta2 and the same Jacobi smoother is a symmetric
    operator (Algorithm 1 pre/post structure);
  * with a single level the cycle is the exact (Cholesky) solve;
  * MG-PCG converges to the direct solution;
  * Chebyshev smoothing: k steps take the error to p_k(D^-1 A) e0, the
    scaled Chebyshev polynomial evaluated independently (numpy's Chebyshev
    series on the eigenvalues of D^-1 A); one step is damped Jacobi with
    omega = 1/theta; the Lanczos estimate is a lower bound of lambda_max
    within 10 % (exact on a diagonal matrix with as many steps as
    eigenvalues); the cycle stays symmetric; PCG reaches the direct solution
    in fewer iterations than with Jacobi.
"""
import numpy as np
import pytest

import workloads
from oracle import fe, mg, mesh


def _setup(nx, ny, nz, n, levels, rmin=0.0, seed=0, k=1):
    p = workloads.cantilever(nx, ny, nz, degree=k, n_mr=n, rmin=rmin, seed=seed)
    m = fe.Model(p)
    rho = m.densities(p.x)
    return p, m, rho, mg.Hierarchy(p, rho, levels)


@pytest.mark.parametrize("n", [1, 2])
def test_coarse_operator_is_galerkin_product(n):
    p, m, rho, h = _setup(8, 4, 4, n, 3, seed=4)
    for l in range(2):
        F, C = h.levels[l], h.levels[l + 1]
        G = (F.P.T @ F.A @ F.P).toarray()
        freec = C.mask == 0
        A = C.A.toarray()
        Gf = G[np.ix_(freec, freec)]
        Af = A[np.ix_(freec, freec)]
        assert np.abs(Gf - Af).max() <= 1e-12 * np.abs(Af).max()


def test_prolongation_reproduces_trilinear_fields():
    lat_f = (9, 5, 5)
    P = mg.prolongation(lat_f)
    Xc = mesh.node_coords(4, 2, 2, 1) * 2.0
    Xf = mesh.node_coords(8, 4, 4, 1)
    f = lambda X: 1 + 2 * X[:, 0] - X[:, 1] + 0.5 * X[:, 2] + 0.25 * X[:, 0] * X[:, 1] * X[:, 2]
    vc = np.zeros(3 * len(Xc)); vc[1::3] = f(Xc)
    vf = P @ vc
    np.testing.assert_allclose(vf[1::3], f(Xf), atol=1e-13)
    assert np.abs(vf[0::3]).max() == 0 and np.abs(vf[2::3]).max() == 0


@pytest.mark.parametrize("gamma", [1, 2])
def test_cycle_is_symmetric(gamma):
    p, m, rho, h = _setup(8, 4, 4, 2, 3, rmin=1.0, seed=9)
    free = h.levels[0].mask == 0
    rng = np.random.default_rng(3)
    x = np.where(free, rng.normal(size=free.size), 0.0)
    y = np.where(free, rng.normal(size=free.size), 0.0)
    a = y @ mg.vcycle(h, x, gamma=gamma)
    b = x @ mg.vcycle(h, y, gamma=gamma)
    assert abs(a - b) <= 1e-10 * abs(a)


def test_single_level_cycle_is_exact_solve():
    p, m, rho, h = _setup(4, 2, 2, 1, 1, seed=1)
    f = np.where(p.mask == 0, p.f[0], 0.0)
    z = mg.vcycle(h, f)
    u = m.solve(m.weights(rho), f)
    np.testing.assert_allclose(z, u, rtol=0, atol=1e-12 * np.abs(u).max())


def test_mg_pcg_converges_to_direct_solution():
    p, m, rho, h = _setup(8, 4, 4, 2, 3, rmin=1.0, seed=6)
    f = np.where(p.mask == 0, p.f[0], 0.0)
    u, its, hist = mg.pcg(h, f, rtol=1e-12)
    ud = m.solve(m.weights(rho), f)
    assert hist[-1] <= 1e-12 and its < 200
    assert np.linalg.norm(u - ud) <= 1e-8 * np.linalg.norm(ud)


def test_run_with_mg_matches_direct_run():
    p = workloads.cantilever(8, 4, 4, degree=1, n_mr=2, rmin=1.0, seed=12, mg_levels=3)
    m = fe.Model(p)
    a = m.run(method="mg", rtol=1e-13)
    b = m.run(method="dense")
    assert np.linalg.norm(a["u"] - b["u"]) <= 1e-9 * np.linalg.norm(b["u"])
    assert abs(a["c"][0] - b["c"][0]) <= 1e-11 * b["c"][0]
    assert np.linalg.norm(a["g_x"] - b["g_x"]) <= 1e-9 * np.linalg.norm(b["g_x"])


@pytest.mark.parametrize("family,n", [("lagrange", 1), ("lagrange", 2), ("serendipity", 1), ("serendipity", 2)])
def test_degree2_shape_transfers_give_galerkin_coarse_operators(family, n):
    """Degree 2 with the coarse shape functions as P: the quadratic spaces
    are nested (the serendipity monomials are closed under per-axis affine
    maps), so the re-discretised coarse operator is P^T A P on the free
    DOFs, for both families."""
    p = workloads.cantilever(8, 4, 4, degree=2, n_mr=n, seed=4)
    if family == "serendipity":
        p = workloads.with_serendipity(p)
    m = fe.Model(p)
    h = mg.Hierarchy(p, m.densities(p.x), 3)
    for l in range(2):
        F, C = h.levels[l], h.levels[l + 1]
        G = (F.P.T @ F.A @ F.P).toarray()
        freec = C.mask == 0
        A = C.A.toarray()
        Gf = G[np.ix_(freec, freec)]
        Af = A[np.ix_(freec, freec)]
        assert np.abs(Gf - Af).max() <= 1e-12 * np.abs(Af).max()
    # the paper's linear lattice interpolation is not Galerkin for degree 2
    if family == "lagrange":
        hl = mg.Hierarchy(p, m.densities(p.x), 2, transfer="linear")
        F, C = hl.levels[0], hl.levels[1]
        freec = C.mask == 0
        G = (F.P.T @ F.A @ F.P).toarray()[np.ix_(freec, freec)]
        assert np.abs(G - C.A.toarray()[np.ix_(freec, freec)]).max() > 1e-3 * np.abs(G).max()


def test_degree2_shape_prolongation_reproduces_quadratics():
    lat_f = (17, 9, 9)  # 8x4x4 degree-2 lattice; coarse 4x2x2
    Xc = mesh.node_coords(4, 2, 2, 2) * 2.0
    Xf = mesh.node_coords(8, 4, 4, 2)
    q = lambda X: 1 + X[:, 0] - 2 * X[:, 1] + X[:, 0] ** 2 * X[:, 1] ** 2 * X[:, 2] ** 2 - X[:, 1] * X[:, 2]
    P = mg.prolongation_shape(lat_f, "lagrange")
    vc = np.zeros(3 * len(Xc)); vc[2::3] = q(Xc)
    np.testing.assert_allclose((P @ vc)[2::3], q(Xf), atol=1e-12)
    # serendipity: a field in its space (x^2 y z, not x^2 y^2), at the nodes it has
    s = lambda X: 1 + X[:, 0] * X[:, 1] - X[:, 2] ** 2 + X[:, 0] ** 2 * X[:, 1] * X[:, 2]
    Ps = mg.prolongation_shape(lat_f, "serendipity")
    vc = np.zeros(3 * len(Xc)); vc[0::3] = s(Xc)
    vc[mg.serendipity_absent((9, 5, 5))] = 0.0
    vf = (Ps @ vc)[0::3]
    present = ~mg.serendipity_absent(lat_f)[0::3]
    np.testing.assert_allclose(vf[present], s(Xf)[present], atol=1e-12)


@pytest.mark.parametrize("family", ["lagrange", "serendipity"])
def test_degree3_p_coarsening_is_galerkin_and_converges(family):
    """Degree 3: level 1 is the degree-2 mesh of the same family on the same
    elements, P the degree-2 shape functions at the degree-3 nodes.  The
    degree-2 space lies in the degree-3 one (serendipity: superlinear degree
    2 within 3), so the re-discretised level-1 operator is P^T A P; MG-PCG
    reaches the direct solution."""
    p = workloads.cantilever(4, 2, 2, degree=3, n_mr=2, seed=3)
    if family == "serendipity":
        p = workloads.with_serendipity(p)
    m = fe.Model(p)
    h = mg.Hierarchy(p, m.densities(p.x), 3 if family == "lagrange" else 2)
    F, C = h.levels[0], h.levels[1]
    fc = C.mask == 0
    G = (F.P.T @ F.A @ F.P).toarray()[np.ix_(fc, fc)]
    A = C.A.toarray()[np.ix_(fc, fc)]
    assert np.abs(G - A).max() <= 1e-12 * np.abs(A).max()
    f = p.f[0].copy()
    f[p.mask.astype(bool)] = 0.0
    u, its, _ = mg.pcg(h, f, rtol=1e-11)
    ref = m.run(method="splu")
    assert np.linalg.norm(u - ref["u"][0]) <= 1e-8 * np.linalg.norm(ref["u"][0])


# ---- Chebyshev smoothing ------------------------------------------------------

def _cheb_case(deg=2, family="lagrange", levels=2, k=2):
    p = workloads.cantilever(4, 2, 2, degree=deg, n_mr=2, rmin=0.0, seed=6, mg_levels=levels)
    if family == "serendipity":
        p = workloads.with_serendipity(p)
    m = fe.Model(p)
    h = mg.Hierarchy(p, m.densities(p.x), levels, smoother="chebyshev", cheb_degree=k)
    return p, h


def _scaled_eigen(L):
    """Eigenpairs of D^-1 A through the symmetric D^-1/2 A D^-1/2."""
    A = L.A.toarray()
    dh = np.sqrt(L.Dinv)
    lam, Q = np.linalg.eigh(dh[:, None] * A * dh[None, :])
    return lam, Q, dh


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_chebyshev_error_is_the_scaled_chebyshev_polynomial(k):
    """k smoothing steps map the error e0 to p_k(D^-1 A) e0 with
    p_k(t) = T_k((theta - t) / delta) / T_k(theta / delta), evaluated here
    by numpy's Chebyshev series on the eigenvalues of D^-1 A."""
    from numpy.polynomial import chebyshev as C

    p, h = _cheb_case(k=k)
    L = h.levels[0]
    _, _, theta, delta = mg.chebyshev_coefficients(L.lmax, k)
    lam, Q, dh = _scaled_eigen(L)
    rng = np.random.default_rng(5)
    xs = rng.normal(size=L.A.shape[0])
    x0 = rng.normal(size=L.A.shape[0])
    b = L.A @ xs
    e = mg.chebyshev_smooth(L, b, x0) - xs
    Tk = np.zeros(k + 1)
    Tk[k] = 1.0
    pk = C.chebval((theta - lam) / delta, Tk) / C.chebval(theta / delta, Tk)
    # D^-1 A = D^-1/2 S D^1/2, S = Q diag(lam) Q^T
    ref = (Q * pk) @ (Q.T @ ((x0 - xs) / dh)) * dh
    np.testing.assert_allclose(e, ref, atol=1e-11 * np.abs(x0 - xs).max())


def test_chebyshev_degree_one_is_damped_jacobi():
    p, h = _cheb_case(k=1)
    L = h.levels[0]
    rng = np.random.default_rng(2)
    b, x = rng.normal(size=L.A.shape[0]), rng.normal(size=L.A.shape[0])
    omega = L.cheb[0]
    np.testing.assert_allclose(mg.chebyshev_smooth(L, b, x), x + omega * L.Dinv * (b - L.A @ x), rtol=1e-14)


def test_lanczos_estimate_is_a_close_lower_bound():
    p, h = _cheb_case()
    for L in h.levels[:-1]:
        lam = _scaled_eigen(L)[0]
        assert L.lmax <= lam.max() * (1 + 1e-12)
        assert L.lmax >= 0.9 * lam.max()
        # the smoothing interval's upper end covers the spectrum
        assert 1.1 * L.lmax >= lam.max()


def test_lanczos_is_exact_on_a_small_diagonal_matrix():
    """With as many steps as distinct eigenvalues, the largest Ritz value is
    the largest eigenvalue (here of diag(1..6) scaled by D = 2 I)."""
    import scipy.sparse as sp

    A = sp.diags(2.0 * np.arange(1.0, 7.0)).tocsr()
    Dinv = np.full(6, 0.5)
    est = mg.lanczos_lmax(A, Dinv, np.zeros(6, dtype=np.uint8), 6)
    assert abs(est - 6.0) <= 1e-12


@pytest.mark.parametrize("deg,family", [(2, "lagrange"), (2, "serendipity"), (3, "lagrange")])
def test_chebyshev_cycle_is_symmetric(deg, family):
    p, h = _cheb_case(deg=deg, family=family, levels=2 if deg == 2 else 3)
    free = h.levels[0].mask == 0
    rng = np.random.default_rng(8)
    x = np.where(free, rng.normal(size=free.size), 0.0)
    y = np.where(free, rng.normal(size=free.size), 0.0)
    a, b = y @ mg.vcycle(h, x), x @ mg.vcycle(h, y)
    assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)


@pytest.mark.parametrize("deg,family", [(2, "lagrange"), (2, "serendipity"), (3, "serendipity")])
def test_chebyshev_pcg_converges_to_direct_solution_in_fewer_iterations(deg, family):
    p = workloads.cantilever(8, 4, 4, degree=deg, n_mr=2 * deg, rmin=0.0, seed=1, mg_levels=2)
    if family == "serendipity":
        p = workloads.with_serendipity(p)
    m = fe.Model(p)
    rho = m.densities(p.x)
    f = p.f[0].copy()
    f[p.mask.astype(bool)] = 0.0
    levels = 2 if deg == 2 else 3
    ref = m.run(method="splu")["u"][0]
    u_c, its_c, _ = mg.pcg(mg.Hierarchy(p, rho, levels, smoother="chebyshev"), f, rtol=1e-10)
    u_j, its_j, _ = mg.pcg(mg.Hierarchy(p, rho, levels), f, rtol=1e-10)
    assert np.linalg.norm(u_c - ref) <= 1e-7 * np.linalg.norm(ref)
    assert its_c < its_j
