"""Thresholding and the Heaviside projection on the GPU (Sec. 5) against the
oracle (oracle/threshold.py).

* Heaviside: eta to 1e-12 (the Newton sums are reductions in another
  order), the projected densities to 1e-12 (dh/deta is at most beta / 2),
  the Newton iteration count exactly.
* Strategy 1: the 0/1 vector bit for bit (an integer selection on the same
  FP64 values, ties by index on both sides), the angle decision equal.
* Strategy 2: the chosen step alpha bit for bit (it is one of the inputs'
  quotients), the projected densities to 1 ulp (the GPU may fuse the
  multiply-add), on sizes the direct oracle handles and, at the density
  grid of the benchmark cantilever (221,184 cells), against the prefix-sum
  construction pinned to the oracle in tests/test_oracle_threshold.py.
"""
import math

import numpy as np
import pytest

from oracle import threshold as th
from tests.gpu_helpers import lib
from tests.test_oracle_threshold import _by_gradient_prefix

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda:0")


def _scratch(T, n):
    import torch

    return torch.empty(max(T.tosolve_threshold_scratch_bytes(n), 1), dtype=torch.uint8, device="cuda:0")


@pytest.mark.parametrize("n,beta", [(1, 1.0), (1000, 1.0), (12345, 8.0), (100003, 64.0)])
def test_heaviside(n, beta):
    import torch

    T = lib()
    rho = np.random.default_rng(n).random(n) ** 2
    out = torch.empty(n, dtype=torch.float64, device="cuda:0")
    eta, its = T.tosolve_heaviside(_dev(rho), beta, out, _scratch(T, n))
    v = np.full(n, 1.0 / n)
    eta_ref, its_ref = th.heaviside_eta(rho, v, beta)
    assert abs(eta - eta_ref) <= 1e-12
    assert its == its_ref
    np.testing.assert_allclose(out.cpu().numpy(), th.heaviside(rho, beta, eta_ref), rtol=0, atol=1e-12)
    assert abs(out.sum().item() - rho.sum()) <= 1e-10 * n


@pytest.mark.parametrize("n,vfrac,ties", [(1, 0.5, False), (7, 0.3, True), (4097, 0.3, True),
                                          (50000, 0.25, False), (2048, 1.0, True), (300, 0.0, False)])
def test_threshold_density(n, vfrac, ties):
    import torch

    T = lib()
    rng = np.random.default_rng(n)
    rho = rng.random(n)
    if ties:
        rho = np.round(rho, 1)
    g = rng.normal(size=n)
    out = torch.empty(n, dtype=torch.float64, device="cuda:0")
    acc = T.tosolve_threshold_density(_dev(rho), vfrac, _dev(g), out, _scratch(T, n))
    r = th.round_extremes(rho)
    ref = th.by_density(r, vfrac)
    assert np.array_equal(out.cpu().numpy(), ref)
    d = ref - r
    if np.linalg.norm(d) > 0:
        cosv = -(g @ d) / (np.linalg.norm(g) * np.linalg.norm(d))
        if abs(cosv - math.cos(math.radians(89.9))) > 1e-12:
            assert acc == th.angle_condition(g, d)
    else:
        assert not acc


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (300, 2), (1500, 3), (1500, 4)])
def test_threshold_gradient_small(n, seed):
    import torch

    T = lib()
    rng = np.random.default_rng(seed)
    rho = rng.random(n)
    if seed % 2:
        rho = np.round(rho, 1)
    g = rng.normal(size=n) * (rng.random(n) < 0.9)
    out = torch.empty(n, dtype=torch.float64, device="cuda:0")
    alpha = T.tosolve_threshold_gradient(_dev(rho), _dev(g), out, _scratch(T, n))
    r = th.round_extremes(rho)
    ref, a_ref = th.by_gradient(r, g)
    assert alpha == a_ref
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=2.3e-16)


def test_threshold_gradient_full_grid():
    """The density grid of the 48x24x24, n = 2 cantilever (96x48x48 cells),
    with gradient and densities shaped like a late optimisation iterate:
    most densities near 0 or 1, small gradients of both signs."""
    import torch

    T = lib()
    n = 96 * 48 * 48
    rng = np.random.default_rng(42)
    rho = np.clip(rng.beta(0.3, 0.3, size=n), 0.0, 1.0)
    g = rng.normal(scale=1e-3, size=n) - 2e-4 * (rho - 0.5)
    out = torch.empty(n, dtype=torch.float64, device="cuda:0")
    alpha = T.tosolve_threshold_gradient(_dev(rho), _dev(g), out, _scratch(T, n))
    r = th.round_extremes(rho)
    a_ref = _by_gradient_prefix(r, g)
    assert alpha == a_ref
    np.testing.assert_allclose(out.cpu().numpy(), th.projected(r, g, a_ref), rtol=0, atol=2.3e-16)


def test_edge_cases_and_errors():
    import torch

    T = lib()
    e = torch.empty(0, dtype=torch.float64, device="cuda:0")
    s = _scratch(T, 0)
    assert T.tosolve_threshold_gradient(e, e, e, s) == 0.0
    assert T.tosolve_threshold_density(e, 0.5, e, e, s) is False
    # zero gradient: nothing moves past the rounding
    rho = _dev([0.2, 0.5, 0.97])
    out = torch.empty(3, dtype=torch.float64, device="cuda:0")
    assert T.tosolve_threshold_gradient(rho, _dev([0.0, 0.0, 0.0]), out, _scratch(T, 3)) == 0.0
    assert out.cpu().numpy().tolist() == [0.2, 0.5, 1.0]
    with pytest.raises(T.TosolveError):
        T.tosolve_heaviside(rho, 0.0, out, _scratch(T, 3))
    with pytest.raises(T.TosolveError):
        T.tosolve_threshold_density(rho, 1.5, rho, out, _scratch(T, 3))
    with pytest.raises(T.TosolveError):
        T.tosolve_threshold_gradient(rho, rho, out, _scratch(T, 3), theta_max_deg=180.0)
    small = torch.empty(16, dtype=torch.uint8, device="cuda:0")
    with pytest.raises(T.TosolveError):
        T.tosolve_threshold_gradient(rho, rho, out, small)
