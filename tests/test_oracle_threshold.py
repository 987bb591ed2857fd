"""Pins of the thresholding and Heaviside oracle (oracle/threshold.py, Sec. 5).

* Strategy 1 against numpy's stable argsort, with its count and order
  properties; ties by index.
* The angle condition on hand-computed directions.
* Strategy 2 on a hand-worked case, and against an independent
  construction: every candidate step evaluated at once with prefix sums
  over the sorted steps (the form a parallel implementation takes).
* The Heaviside projection: the bounds the section states (h(rho, beta, 0)
  >= rho, h(rho, beta, 1) <= rho), h -> rho as beta -> 0, the derivative
  against finite differences, and Newton's eta against scipy's brentq.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import threshold as th


def test_round_extremes():
    r = th.round_extremes(np.array([0.0, 0.05, 0.051, 0.5, 0.949, 0.95, 1.0]))
    assert list(r) == [0.0, 0.0, 0.051, 0.5, 0.949, 1.0, 1.0]


@pytest.mark.parametrize("n,vfrac", [(1, 0.5), (10, 0.3), (101, 0.25), (64, 1.0)])
def test_by_density_is_a_stable_descending_sort(n, vfrac):
    rng = np.random.default_rng(n)
    rho = np.round(rng.random(n), 1)  # many ties
    out = th.by_density(rho, vfrac)
    k = math.floor(vfrac * n)
    assert out.sum() == k
    idx = np.argsort(-rho, kind="stable")
    want = np.zeros(n)
    want[idx[:k]] = 1.0
    assert np.array_equal(out, want)
    if 0 < k < n:
        assert rho[out == 1].min() >= rho[out == 0].max()


def test_angle_condition_by_hand():
    g = np.array([1.0, -2.0, 0.5])
    assert th.angle_condition(g, -g)
    assert not th.angle_condition(g, g)
    assert not th.angle_condition(g, np.array([2.0, 1.0, 0.0]))  # orthogonal
    assert not th.angle_condition(g, np.zeros(3))
    # just inside 89.9 degrees: cos = 0.002 > cos(89.9 deg) = 0.001745
    d = np.array([1.0, 0.0, 0.0]) * -0.002 + np.array([0.0, 1.0, 0.0]) * math.sqrt(1 - 0.002 ** 2)
    assert th.angle_condition(np.array([1.0, 0.0, 0.0]), d)
    d2 = np.array([1.0, 0.0, 0.0]) * -0.0015 + np.array([0.0, 1.0, 0.0]) * math.sqrt(1 - 0.0015 ** 2)
    assert not th.angle_condition(np.array([1.0, 0.0, 0.0]), d2)


def test_by_gradient_by_hand():
    # alpha = (0.5, 0.5): both reach their bound together, d = (-0.5, 0.5)
    # is exactly -grad / 2: accepted.
    out, a = th.by_gradient(np.array([0.5, 0.5]), np.array([1.0, -1.0]))
    assert a == 0.5 and list(out) == [0.0, 1.0]
    # a density of 0.2 may not be rounded to 1 (safeguard 0.3): its step
    # 0.8 caps alpha below it; the first component (step 0.4) is fine.
    out, a = th.by_gradient(np.array([0.4, 0.2]), np.array([1.0, -1.0]))
    assert a == 0.4 and np.allclose(out, [0.0, 0.6])
    # zero gradient: nothing moves
    out, a = th.by_gradient(np.array([0.4, 0.6]), np.zeros(2))
    assert a == 0.0 and list(out) == [0.4, 0.6]


def _by_gradient_prefix(rho, grad, vu_min=0.3, vl_max=0.7, theta=89.9):
    """Independent construction: candidates sorted once; at candidate j the
    components 0..j have reached their bound t, the others move by -alpha g.
    grad^T d = S1_j - alpha G_j and ||d||^2 = S2_j + alpha^2 G_j with S1, S2
    prefix sums over the reached ones and G the sum of g^2 over the rest."""
    alpha = th.step_to_bound(rho, grad)
    order = np.lexsort((np.arange(rho.size), alpha))
    a = alpha[order]
    g = grad[order]
    r = rho[order]
    t = np.where(g > 0, 0.0, 1.0)
    fin = np.isfinite(a)
    S1 = np.cumsum(np.where(fin, g * (t - r), 0.0))
    S2 = np.cumsum(np.where(fin, (t - r) ** 2, 0.0))
    G = np.sum(g * g) - np.cumsum(g * g)
    bad = np.cumsum(((g < 0) & (r < vu_min)) | ((g > 0) & (r > vl_max))) > 0
    ng = np.linalg.norm(grad)
    with np.errstate(invalid="ignore", divide="ignore"):  # a = inf where g = 0
        gd = S1 - a * G
        dd = np.sqrt(np.maximum(S2 + a * a * G, 0.0))
        ok = fin & ~bad & (dd > 0) & (-gd / (ng * dd) > math.cos(math.radians(theta)))
    if not ok.any():
        return 0.0
    return float(a[np.nonzero(ok)[0].max()])


@pytest.mark.parametrize("seed", range(6))
def test_by_gradient_matches_prefix_construction(seed):
    rng = np.random.default_rng(seed)
    n = 40
    rho = rng.random(n)
    grad = rng.normal(size=n) * (rng.random(n) < 0.9)
    if seed % 2:
        rho = np.round(rho, 1)
    _, a = th.by_gradient(rho, grad)
    assert a == pytest.approx(_by_gradient_prefix(rho, grad), rel=0, abs=0)


def test_heaviside_bounds_and_limits():
    rho = np.linspace(0.0, 1.0, 101)
    for beta in (0.5, 1.0, 8.0, 100.0):
        assert (th.heaviside(rho, beta, 0.0) >= rho - 1e-15).all()
        assert (th.heaviside(rho, beta, 1.0) <= rho + 1e-15).all()
        for eta in (0.2, 0.5, 0.9):
            h = th.heaviside(rho, beta, eta)
            assert abs(h[0]) < 1e-15 and abs(h[-1] - 1.0) < 1e-15
            assert (np.diff(h) >= 0).all()
            assert h[int(100 * eta) + 3] > h[int(100 * eta) - 3]  # rises around eta
    assert np.allclose(th.heaviside(rho, 1e-6, 0.37), rho, atol=1e-10)


@pytest.mark.parametrize("beta", [1.0, 4.0, 32.0])
def test_heaviside_eta_is_the_zero_of_f(beta):
    rng = np.random.default_rng(int(beta))
    rho = rng.random(500) ** 2
    v = np.full(rho.size, 1.0 / rho.size)
    for eta in (0.1, 0.5, 0.8):
        e = 1e-6
        fd = (th.heaviside_f(rho, v, beta, eta + e) - th.heaviside_f(rho, v, beta, eta - e)) / (2 * e)
        assert th.heaviside_df(rho, v, beta, eta) == pytest.approx(fd, rel=1e-6, abs=1e-9)
    eta, its = th.heaviside_eta(rho, v, beta)
    ref = brentq(lambda z: th.heaviside_f(rho, v, beta, z), 1e-12, 1 - 1e-12, xtol=1e-15)
    assert abs(eta - ref) <= 1e-10 and its < 30
    assert abs(v @ th.heaviside(rho, beta, eta) - v @ rho) <= 1e-12
