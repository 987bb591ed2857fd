"""Density projection (thresholding) and the Heaviside projection (oracle).

Section 5.  With n densities rho_i of volumes v_i and a volume fraction
v_frac:
  * first, densities >= 0.95 are rounded to 1 and densities <= 0.05 to 0;
  * strategy 1 (density values): the floor(v_frac n) largest densities
    become 1, the others 0; the result is accepted when d = rho~ - rho makes
    an angle below theta_max with -grad L (Eq. angle);
  * strategy 2 (gradient of the Lagrangian): rho~(alpha) is the projection
    of rho - alpha grad L onto [0, 1]; alpha_i is the step at which
    component i reaches its bound (0 when grad_i L > 0, 1 when < 0); alpha~
    is the largest alpha_i at which rho~ satisfies the angle condition and
    the safeguards (a component may reach 1 only if its density is at least
    v_min^u, and 0 only if at most v_max^l);
  * the Heaviside projection h(rho, beta, eta) = (tanh(beta eta) +
    tanh(beta (rho - eta))) / (tanh(beta eta) + tanh(beta (1 - eta))) with
    eta the zero of f(eta) = sum v_i h(rho_i, beta, eta) - sum v_i rho_i,
    found by Newton's method.

Readings (the section does not fix them):
  * the safeguards test the densities before the projection (the projected
    values of the components that reach a bound are 0 or 1 by construction);
  * among equal densities, strategy 1 makes the ones with the lower index 1
    (a stable sort in descending order), and strategy 2 orders equal
    alpha_i by index as well; components with grad_i L = 0 never reach a
    bound;
  * with d = 0 the angle condition fails (0 > cos(theta_max) is false);
  * if no alpha_i qualifies, alpha~ = 0 and the densities stay as rounded;
  * Newton starts from eta = 1/2 and stops when |f| <= 1e-12 sum v_i or the
    step is below 1e-14; a step that would leave (0, 1) is halved until it
    does not (f has a zero in (0, 1), Sec. 5).

Test infrastructure only: nothing on the product path imports this module.
"""
from __future__ import annotations

import math

import numpy as np


def round_extremes(rho: np.ndarray, lo: float = 0.05, hi: float = 0.95) -> np.ndarray:
    """The first step of both strategies."""
    r = np.array(rho, dtype=np.float64)
    r[r >= hi] = 1.0
    r[r <= lo] = 0.0
    return r


def angle_condition(grad: np.ndarray, d: np.ndarray, theta_max_deg: float = 89.9) -> bool:
    """Eq. angle: -grad^T d / (||grad|| ||d||) > cos(theta_max)."""
    ng, nd = float(np.linalg.norm(grad)), float(np.linalg.norm(d))
    if ng == 0.0 or nd == 0.0:
        return False
    return -float(grad @ d) / (ng * nd) > math.cos(math.radians(theta_max_deg))


def by_density(rho: np.ndarray, vfrac: float) -> np.ndarray:
    """Strategy 1: the floor(vfrac n) largest densities to 1, the rest to 0."""
    n = rho.size
    k = int(math.floor(vfrac * n))
    order = sorted(range(n), key=lambda i: (-rho[i], i))
    out = np.zeros(n)
    out[order[:k]] = 1.0
    return out


def step_to_bound(rho: np.ndarray, grad: np.ndarray) -> np.ndarray:
    """alpha_i at which rho_i - alpha grad_i reaches 0 (grad_i > 0) or 1
    (grad_i < 0); +inf when grad_i = 0."""
    a = np.full(rho.size, np.inf)
    pos, neg = grad > 0, grad < 0
    a[pos] = rho[pos] / grad[pos]
    a[neg] = (rho[neg] - 1.0) / grad[neg]
    return a


def projected(rho: np.ndarray, grad: np.ndarray, alpha: float) -> np.ndarray:
    return np.clip(rho - alpha * grad, 0.0, 1.0)


def by_gradient(rho: np.ndarray, grad: np.ndarray, vu_min: float = 0.3, vl_max: float = 0.7,
                theta_max_deg: float = 89.9) -> tuple[np.ndarray, float]:
    """Strategy 2: returns (rho~, alpha~).  Every candidate alpha_i is
    checked directly (O(n^2): small inputs only)."""
    alpha = step_to_bound(rho, grad)
    best = 0.0
    order = sorted(range(rho.size), key=lambda i: (alpha[i], i))
    for j, i in enumerate(order):
        a = alpha[i]
        if not np.isfinite(a):
            break
        # safeguards on every component that has reached its bound at a
        reached = order[:j + 1]
        ok = True
        for q in reached:
            if grad[q] < 0 and rho[q] < vu_min:
                ok = False
            if grad[q] > 0 and rho[q] > vl_max:
                ok = False
        if not ok:
            break  # a larger alpha keeps this component at its bound
        if angle_condition(grad, projected(rho, grad, a) - rho, theta_max_deg):
            best = a
    return projected(rho, grad, best), best


def heaviside(rho: np.ndarray, beta: float, eta: float) -> np.ndarray:
    t = math.tanh(beta * eta)
    return (t + np.tanh(beta * (rho - eta))) / (t + math.tanh(beta * (1.0 - eta)))


def heaviside_f(rho: np.ndarray, v: np.ndarray, beta: float, eta: float) -> float:
    return float(v @ heaviside(rho, beta, eta) - v @ rho)


def heaviside_df(rho: np.ndarray, v: np.ndarray, beta: float, eta: float) -> float:
    """d f / d eta from the quotient rule (sech^2 = 1 - tanh^2)."""
    tn = math.tanh(beta * eta)
    t1 = math.tanh(beta * (1.0 - eta))
    tr = np.tanh(beta * (rho - eta))
    num = tn + tr
    den = tn + t1
    dnum = beta * (1.0 - tn * tn) - beta * (1.0 - tr * tr)
    dden = beta * (1.0 - tn * tn) - beta * (1.0 - t1 * t1)
    return float(v @ ((dnum * den - num * dden) / (den * den)))


def heaviside_eta(rho: np.ndarray, v: np.ndarray, beta: float, maxit: int = 100) -> tuple[float, int]:
    """Newton's method for f(eta) = 0 (volume-preserving eta)."""
    eta = 0.5
    scale = float(np.sum(v))
    for it in range(1, maxit + 1):
        f = heaviside_f(rho, v, beta, eta)
        if abs(f) <= 1e-12 * scale:
            return eta, it - 1
        step = f / heaviside_df(rho, v, beta, eta)
        while not (0.0 < eta - step < 1.0):
            step *= 0.5
        eta -= step
        if abs(step) < 1e-14:
            return eta, it
    return eta, maxit
