"""Pins of the serendipity elements in the oracle (oracle/fem.py, Sec. 2.1):
the 20-node element on the degree-2 lattice and the 32-node element on the
degree-3 lattice (the same checks, the second set at the end).

* The shape functions: Kronecker delta at the 20 nodes, zero at the face
  and cell centres, partition of unity, and exact reproduction of the 20
  monomials that span the serendipity space (a wrong sign or factor in any
  shape function breaks one of them); gradients against finite differences.
* The element matrix: rank 54 (60 DOFs less the 6 rigid modes), the rigid
  modes as its kernel, subcell sums equal to the whole element, and two
  entries integrated exactly (sympy, rational arithmetic) from the tensor
  form of the bilinear form, independently of the Voigt B^T D B code.
* The assembled serendipity mesh: a linear displacement field passes the
  patch test (interior residual zero).
"""
import itertools

import numpy as np
import pytest

import workloads
from oracle import fe, fem

NU = 0.3
NODES = [(ix - 1, iy - 1, iz - 1) for iz in range(3) for iy in range(3) for ix in range(3)]


def test_kronecker_and_absent_nodes():
    present = fem.serendipity2_present()
    assert present.sum() == 20
    for b, xb in enumerate(NODES):
        N, _ = fem.serendipity2_shape(*xb)
        if present[b]:
            want = np.zeros(27)
            want[b] = 1.0
            assert np.allclose(N, want, atol=1e-15)
        assert np.all(N[~present] == 0.0)


def test_completeness_over_the_serendipity_monomials():
    mons = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0),
            (0, 1, 1), (1, 0, 1), (2, 1, 0), (2, 0, 1), (1, 2, 0), (0, 2, 1), (1, 0, 2), (0, 1, 2),
            (1, 1, 1), (2, 1, 1), (1, 2, 1), (1, 1, 2)]
    rng = np.random.default_rng(0)
    present = fem.serendipity2_present()
    for _ in range(10):
        x = rng.uniform(-1, 1, size=3)
        N, _ = fem.serendipity2_shape(*x)
        assert abs(N.sum() - 1.0) < 1e-14
        for m in mons:
            vals = np.array([np.prod([c ** e for c, e in zip(xb, m)]) for xb in NODES])
            vals[~present] = 0.0
            assert abs(N @ vals - np.prod(x ** np.array(m))) < 1e-14, m
    # a monomial outside the space is not reproduced
    x = np.array([0.3, -0.4, 0.7])
    N, _ = fem.serendipity2_shape(*x)
    vals = np.array([xb[0] ** 2 * xb[1] ** 2 for xb in NODES])
    assert abs(N @ vals - x[0] ** 2 * x[1] ** 2) > 1e-3


def test_gradients_against_finite_differences():
    x = np.array([0.21, -0.63, 0.44])
    _, dN = fem.serendipity2_shape(*x, h=2.0)  # h = 2: physical = reference gradient
    e = 1e-6
    for q in range(3):
        xp, xm = x.copy(), x.copy()
        xp[q] += e
        xm[q] -= e
        fd = (fem.serendipity2_shape(*xp)[0] - fem.serendipity2_shape(*xm)[0]) / (2 * e)
        assert np.allclose(dN[:, q], fd, atol=1e-9)


def test_element_rank_kernel_and_subcells():
    K = fem.subcell_stiffness(2, 1, NU, family="serendipity")[0]
    assert np.abs(K - K.T).max() < 1e-15
    assert np.linalg.matrix_rank(K, tol=1e-10) == 54
    R = fem.rigid_body_modes(2)
    assert np.abs(K @ R.T).max() < 1e-14
    absent = np.repeat(~fem.serendipity2_present(), 3)
    assert np.all(K[absent] == 0.0) and np.all(K[:, absent] == 0.0)
    for n in (2, 3):
        Kn = fem.subcell_stiffness(2, n, NU, family="serendipity")
        assert np.abs(Kn.sum(axis=0) - K).max() < 1e-13


def test_two_entries_exactly():
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    nu = sympy.Rational(3, 10)
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1 / (2 * (1 + nu))
    X = [2 * x - 1, 2 * y - 1, 2 * z - 1]  # unit cube [0, 1]^3 -> [-1, 1]^3 (h = 1)

    def shape(c):
        mids = [q for q in range(3) if c[q] == 0]
        if not mids:
            f = sympy.Integer(1)
            for q in range(3):
                f *= 1 + X[q] * c[q]
            return f * (X[0] * c[0] + X[1] * c[1] + X[2] * c[2] - 2) / 8
        m = mids[0]
        f = sympy.Integer(1)
        for q in range(3):
            f *= (1 - X[q] ** 2) if q == m else (1 + X[q] * c[q])
        return f / 4

    V = [x, y, z]

    def entry(ca, ia, cb, ib):
        """int sigma(u)_ij eps(v)_ij for u = N_a e_ia, v = N_b e_ib (tensor form)."""
        Na, Nb = shape(ca), shape(cb)
        ga = [sympy.diff(Na, v) for v in V]
        gb = [sympy.diff(Nb, v) for v in V]
        # eps(u) = sym(e_ia (x) grad Na); sigma = lam tr(eps) I + 2 mu eps
        integrand = lam * ga[ia] * gb[ib] + mu * (ga[ib] * gb[ia] + (sum(ga[q] * gb[q] for q in range(3)) if ia == ib else 0))
        return sympy.integrate(integrand, (x, 0, 1), (y, 0, 1), (z, 0, 1))

    K = fem.subcell_stiffness(2, 1, NU, family="serendipity")[0]
    cases = [((-1, -1, -1), 0, (-1, -1, -1), 0), ((0, -1, -1), 1, (1, 1, 0), 2)]
    for ca, ia, cb, ib in cases:
        a = NODES.index(ca)
        b = NODES.index(cb)
        exact = float(entry(ca, ia, cb, ib))
        assert abs(K[3 * a + ia, 3 * b + ib] - exact) <= 1e-14 * max(1.0, abs(exact))


def test_patch_test_on_a_serendipity_mesh():
    p = workloads.with_serendipity(workloads.cantilever(3, 2, 2, degree=2, n_mr=2, density="solid", seed=0))
    m = fe.Model(p)
    K = m.assemble(m.weights(m.densities(p.x))).toarray()
    Lx, Ly, Lz = p.lattice
    nn = Lx * Ly * Lz
    n = np.arange(nn)
    i, j, l = n % Lx, (n // Lx) % Ly, n // (Lx * Ly)
    absent = workloads.serendipity_absent_nodes(p)
    u = np.zeros(3 * nn)
    u[0::3] = 0.01 * i + 0.02 * j
    u[1::3] = -0.03 * l
    u[2::3] = 0.005 * i - 0.01 * l
    u[np.repeat(absent, 3)] = 0.0
    r = K @ u
    interior = (i > 0) & (i < Lx - 1) & (j > 0) & (j < Ly - 1) & (l > 0) & (l < Lz - 1) & ~absent
    assert interior.any()
    assert np.abs(r[np.repeat(interior, 3)]).max() < 1e-12


# ---- the 32-node cubic serendipity element -----------------------------------

POS3 = (-1.0, -1.0 / 3.0, 1.0 / 3.0, 1.0)
NODES3 = [(POS3[i % 4], POS3[(i // 4) % 4], POS3[i // 16]) for i in range(64)]


def test_s3_kronecker_and_completeness():
    present = fem.serendipity_present(3)
    assert present.sum() == 32
    for b, xb in enumerate(NODES3):
        N, _ = fem.serendipity3_shape(*xb)
        if present[b]:
            want = np.zeros(64)
            want[b] = 1.0
            assert np.allclose(N, want, atol=1e-14)
        assert np.all(N[~present] == 0.0)
    # the 32 monomials of superlinear degree <= 3 (the total degree less the
    # number of variables that appear linearly): reproduced exactly
    mons = [m for m in itertools.product(range(4), repeat=3) if sum(m) - sum(1 for e in m if e == 1) <= 3]
    assert len(mons) == 32, len(mons)
    rng = np.random.default_rng(3)
    for _ in range(8):
        x = rng.uniform(-1, 1, size=3)
        N, _ = fem.serendipity3_shape(*x)
        assert abs(N.sum() - 1.0) < 1e-13
        for m in mons:
            vals = np.array([np.prod([c ** e for c, e in zip(xb, m)]) for xb in NODES3])
            vals[~present] = 0.0
            assert abs(N @ vals - np.prod(x ** np.array(m))) < 1e-13, m
    x = np.array([0.3, -0.4, 0.7])
    N, _ = fem.serendipity3_shape(*x)
    vals = np.array([xb[0] ** 2 * xb[1] ** 2 for xb in NODES3])  # superlinear degree 4
    assert abs(N @ vals - x[0] ** 2 * x[1] ** 2) > 1e-3


def test_s3_gradients_rank_and_subcells():
    x = np.array([0.37, -0.52, 0.11])
    _, dN = fem.serendipity3_shape(*x, h=2.0)
    e = 1e-6
    for q in range(3):
        xp, xm = x.copy(), x.copy()
        xp[q] += e
        xm[q] -= e
        fd = (fem.serendipity3_shape(*xp)[0] - fem.serendipity3_shape(*xm)[0]) / (2 * e)
        assert np.allclose(dN[:, q], fd, atol=1e-8)
    K = fem.subcell_stiffness(3, 1, NU, family="serendipity")[0]
    assert np.linalg.matrix_rank(K, tol=1e-9) == 90
    assert np.abs(K @ fem.rigid_body_modes(3).T).max() < 1e-13
    K2 = fem.subcell_stiffness(3, 2, NU, family="serendipity")
    assert np.abs(K2.sum(axis=0) - K).max() < 1e-12


def test_s3_patch_test():
    p = workloads.with_serendipity(workloads.cantilever(2, 2, 2, degree=3, n_mr=1, density="solid", seed=0))
    m = fe.Model(p)
    K = m.assemble(m.weights(m.densities(p.x))).toarray()
    Lx, Ly, Lz = p.lattice
    n = np.arange(Lx * Ly * Lz)
    i, j, l = n % Lx, (n // Lx) % Ly, n // (Lx * Ly)
    absent = workloads.serendipity_absent_nodes(p)
    u = np.zeros(3 * len(n))
    u[0::3] = 0.01 * i - 0.02 * l
    u[1::3] = 0.03 * j
    u[2::3] = -0.01 * i + 0.005 * j
    u[np.repeat(absent, 3)] = 0.0
    r = K @ u
    interior = (i > 0) & (i < Lx - 1) & (j > 0) & (j < Ly - 1) & (l > 0) & (l < Lz - 1) & ~absent
    assert interior.any()
    assert np.abs(r[np.repeat(interior, 3)]).max() < 1e-12
