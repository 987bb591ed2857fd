"""Pins of the oracle's element library (oracle/fem.py).

What pins what:
  * exact symbolic integration of the elasticity bilinear form
    a(u, v) = int lambda div u div v + 2 mu eps(u):eps(v) over the unit cube
    (and over its eight half-size sub-cubes) -- a different formula (tensor,
    not Voigt B^T D B) integrated exactly (not by Gauss points); catches
    errors in D, B, the node order, the Jacobian and the subcell intervals;
  * rank(K^(e)) = 3 n_e - 6 with the six rigid-body modes as null space
    (Section 3.5, Table bounds: m max = 18, 75, 186 for Lagrange k = 1, 2, 3);
  * sum of the subcell matrices = whole-element matrix (Section 3.3);
  * K scales linearly with the element edge h (3D elasticity: h^3 / h^2).
"""
import numpy as np
import pytest

from oracle import fem


def test_lagrange_basis_interpolates_and_sums_to_one():
    for k in (1, 2, 3):
        nodes, _, _ = fem.lagrange_1d(k)
        for m, xm in enumerate(nodes):
            N, _ = fem.shape_1d(k, xm)
            np.testing.assert_allclose(N, np.eye(k + 1)[m], atol=1e-14)
        for xi in np.linspace(-1, 1, 7):
            N, dN = fem.shape_1d(k, xi)
            assert abs(N.sum() - 1.0) < 1e-14
            assert abs(dN.sum()) < 1e-12


def _symbolic_q1_stiffness(nu, box):
    """Exact K over a sub-box of the unit cube [0,1]^3 for trilinear shape
    functions, from the tensor form of the bilinear form."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    X = (x, y, z)
    nu = sp.Rational(nu).limit_denominator(1000)
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1 / (2 * (1 + nu))
    N = []
    for iz in range(2):
        for iy in range(2):
            for ix in range(2):
                fx = x if ix else 1 - x
                fy = y if iy else 1 - y
                fz = z if iz else 1 - z
                N.append(sp.expand(fx * fy * fz))
    G = [[sp.diff(Na, X[p]) for p in range(3)] for Na in N]
    bounds = [tuple(sp.Rational(v) for v in ab) for ab in box]

    def integ(expr):
        # exact: expand into monomials and integrate each in closed form
        total = sp.Integer(0)
        for powers, coeff in sp.Poly(expr, *X).terms():
            term = coeff
            for (lo, hi), a in zip(bounds, powers):
                term *= (hi ** (a + 1) - lo ** (a + 1)) / (a + 1)
            total += term
        return float(total)

    K = np.zeros((24, 24))

    for a in range(8):
        for b in range(8):
            for i in range(3):
                for j in range(3):
                    # u = N_b e_j, v = N_a e_i:
                    # lambda d_i N_a d_j N_b + mu (d_j N_a d_i N_b + delta_ij grad N_a . grad N_b)
                    e = lam * G[a][i] * G[b][j] + mu * G[a][j] * G[b][i]
                    if i == j:
                        e += mu * sum(G[a][p] * G[b][p] for p in range(3))
                    K[3 * a + i, 3 * b + j] = integ(sp.expand(e))
    return K


def test_q1_unit_cube_matches_exact_symbolic_integral():
    K = fem.element_stiffness(1, 0.3)
    Kx = _symbolic_q1_stiffness(0.3, ((0, 1), (0, 1), (0, 1)))
    np.testing.assert_allclose(K, Kx, rtol=0, atol=1e-14)
    # a hand-derived entry: K_00 = (lambda + 4 mu) / 9 for node 0, x-DOF
    lam = 0.3 / (1.3 * 0.4)
    mu = 1 / 2.6
    assert abs(K[0, 0] - (lam + 4 * mu) / 9) < 1e-14
    # and the x-y coupling at node 0: (lambda + mu) / 12
    assert abs(K[0, 1] - (lam + mu) / 12) < 1e-14


def test_q1_subcells_match_exact_symbolic_subbox_integrals():
    Ks = fem.subcell_stiffness(1, 2, 0.3)
    for c in range(2):
        for b in range(2):
            for a in range(2):
                i = a + 2 * (b + 2 * c)
                box = ((a / 2, (a + 1) / 2), (b / 2, (b + 1) / 2), (c / 2, (c + 1) / 2))
                Kx = _symbolic_q1_stiffness(0.3, box)
                np.testing.assert_allclose(Ks[i], Kx, rtol=0, atol=1e-14)


@pytest.mark.parametrize("k,rank", [(1, 18), (2, 75), (3, 186)])
def test_element_rank_and_rigid_body_null_space(k, rank):
    K = fem.element_stiffness(k, 0.3)
    np.testing.assert_allclose(K, K.T, atol=1e-13)
    ev = np.linalg.eigvalsh(K)
    tol = 1e-10 * ev.max()
    assert int((ev > tol).sum()) == rank
    assert int((np.abs(ev) <= tol).sum()) == 6
    assert ev.min() > -tol
    R = fem.rigid_body_modes(k)
    assert np.abs(K @ R.T).max() < 1e-12


@pytest.mark.parametrize("k,n", [(1, 1), (1, 2), (1, 3), (1, 4), (2, 2), (2, 3), (3, 2)])
def test_subcells_sum_to_whole_element(k, n):
    Ks = fem.subcell_stiffness(k, n, 0.3)
    assert Ks.shape == (n ** 3, 3 * (k + 1) ** 3, 3 * (k + 1) ** 3)
    np.testing.assert_allclose(Ks.sum(axis=0), fem.element_stiffness(k, 0.3), atol=1e-12)
    # each subcell matrix is itself PSD with the rigid modes in its kernel
    R = fem.rigid_body_modes(k)
    for Ki in Ks[: min(len(Ks), 8)]:
        assert np.abs(Ki @ R.T).max() < 1e-12
        assert np.linalg.eigvalsh(Ki).min() > -1e-12


def test_stiffness_scales_with_edge_length():
    np.testing.assert_allclose(fem.subcell_stiffness(1, 2, 0.3, h=4.0),
                               4.0 * fem.subcell_stiffness(1, 2, 0.3, h=1.0), rtol=1e-13,
                               atol=1e-14)


def test_elasticity_D_is_hookes_law():
    # uniaxial stress check: strain (1, -nu, -nu, 0, 0, 0) gives stress (E, 0, 0, ...)
    nu = 0.3
    D = fem.elasticity_D(nu, E=2.0)
    s = D @ np.array([1.0, -nu, -nu, 0, 0, 0])
    np.testing.assert_allclose(s, [2.0, 0, 0, 0, 0, 0], atol=1e-14)
    # pure shear: engineering gamma gives tau = mu * gamma
    s = D @ np.array([0, 0, 0, 1.0, 0, 0])
    assert abs(s[3] - 2.0 / (2 * (1 + nu))) < 1e-14
