"""Sequential linear programming over the solver (host side, Sec. 4).

The topology problem (Problem topopt) as the SLP of Sec. 4: minimise the
compliance f(x) = f^T u(x) subject to the linear volume constraint
v^T H x <= Vmax and 0 <= x <= 1.  Each iteration solves the LP of
Problem Pstar (linearised objective, trust region ||s||_inf <= delta) on
the host, accepts or rejects the step by the merit-function test, updates
the trust region and the penalty parameter theta, and stops on the
KKT-based criteria of Sec. 4.3.  f and grad f come from the GPU solver
through the C ABI (one tosolve_step_host per trial point, warm-started from
the previous displacements, Sec. 7.2.1).

Readings (the paper is terse here):
  * the volume constraint is an inequality; it enters the LP as one row
    and the infeasibility measure is phi(x) = 1/2 max(0, v^T H x - Vmax)^2;
  * P_red^opt in the theta rule is the predicted decrease of f,
    -grad f^T s (with the sign as printed theta would collapse to 0 at a
    feasible point and every step would be accepted);
  * the objective-change test uses the relative change |df| / |f|.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import linprog


class SLP:
    """Drives one design through Algorithm 2 (SLP).

    evaluate(x) -> (f, grad_f) runs one solve and gradient for design x.
    volume_row: the row a with volume = a^T x (= H^T v).
    """

    def __init__(self, evaluate, volume_row: np.ndarray, vmax: float, x0: np.ndarray,
                 delta0: float = 0.1, delta_min: float = 1e-4, N: float = 1e6,
                 eps_s: float = 1e-4, eps_f: float = 5e-2, eps_g: float = 1e-3,
                 max_iter: int = 500):
        self.evaluate = evaluate
        self.a = np.asarray(volume_row, dtype=np.float64)
        self.vmax = float(vmax)
        self.x = np.clip(np.asarray(x0, dtype=np.float64), 0.0, 1.0)
        self.delta = float(delta0)
        self.delta_min = float(delta_min)
        self.N = float(N)
        self.eps = (eps_s, eps_f, eps_g)
        self.max_iter = max_iter
        self.f, self.g = evaluate(self.x)
        self.theta_hist = []
        self.theta_max = 1.0
        self.k = 0
        self.history = [dict(k=0, f=self.f, volume=float(self.a @ self.x), delta=self.delta)]
        self._streak_fg = 0
        self._streak_s = 0

    def _c(self, x):  # constraint residual (positive = violated)
        return max(0.0, float(self.a @ x) - self.vmax)

    def _phi(self, x):
        return 0.5 * self._c(x) ** 2

    def _lp(self, delta):
        """Problem Pstar: min g^T s, a^T s <= Vmax - a^T x, s in the box."""
        sl = np.maximum(-delta, -self.x)
        su = np.minimum(delta, 1.0 - self.x)
        res = linprog(self.g, A_ub=self.a[None, :], b_ub=[self.vmax - float(self.a @ self.x)],
                      bounds=np.stack([sl, su], axis=1), method="highs")
        if res.status != 0:
            return None, 0.0
        lam = -float(res.ineqlin.marginals[0]) if res.ineqlin is not None else 0.0
        return res.x, lam

    def _lp_feasibility(self, delta):
        """Problem Pstar2 with one artificial slack z >= 0 on the volume row
        (the box shrunk to 0.8 delta)."""
        n = self.x.size
        sl = np.maximum(-0.8 * delta, -self.x)
        su = np.minimum(0.8 * delta, 1.0 - self.x)
        cost = np.concatenate([np.zeros(n), [1.0]])
        A = np.concatenate([self.a, [-1.0]])[None, :]
        b = [self.vmax - float(self.a @ self.x)]
        bounds = np.concatenate([np.stack([sl, su], axis=1), [[0.0, None]]])
        res = linprog(cost, A_ub=A, b_ub=b, bounds=bounds, method="highs")
        return res.x[:n]

    def step(self) -> dict:
        """One pass of the loop of Algorithm 2 (an accepted or a rejected
        step); returns what happened."""
        s, lam = self._lp(self.delta)
        if s is None:
            s = self._lp_feasibility(self.delta)
            lam = 0.0
        # penalty parameter
        M0 = self._phi(self.x)
        Ms = 0.5 * max(0.0, float(self.a @ (self.x + s)) - self.vmax) ** 2
        p_fsb = M0 - Ms
        p_opt = -float(self.g @ s)
        t_min = min(self.theta_hist) if self.theta_hist else 1.0
        t_large = (1.0 + self.N / (self.k + 1) ** 1.1) * t_min
        t_sup = 0.5 * p_fsb / (p_fsb - p_opt) if (p_opt <= 0.5 * p_fsb and p_fsb != p_opt) else 1.0
        theta = min(t_large, t_sup, self.theta_max)
        self.theta_hist.append(theta)
        x_new = np.clip(self.x + s, 0.0, 1.0)
        f_new, g_new = self.evaluate(x_new)
        a_red = theta * (self.f - f_new) + (1.0 - theta) * (self._phi(self.x) - self._phi(x_new))
        p_red = theta * p_opt + (1.0 - theta) * p_fsb
        s_inf = float(np.abs(s).max()) if s.size else 0.0
        if a_red < 0.1 * p_red:  # reject
            self.delta = min(0.25 * s_inf, 0.1 * self.delta)
            self.theta_max = theta
            return dict(accepted=False, f_trial=f_new, delta=self.delta)
        f_old = self.f
        self.x, self.f, self.g = x_new, f_new, g_new
        if a_red >= 0.5 * p_red:
            self.delta = min(2.0 * self.delta, 1.0)
        self.delta = max(self.delta, self.delta_min)
        self.theta_max = 1.0
        self.k += 1
        # stopping criteria (Sec. 4.3): projected Lagrangian gradient
        grad_l = self.g + lam * self.a
        gp = np.clip(self.x - grad_l, 0.0, 1.0) - self.x
        eps_s, eps_f, eps_g = self.eps
        kkt = float(np.abs(gp).max())
        df = abs(self.f - f_old) / max(abs(self.f), 1e-300)
        self._streak_fg = self._streak_fg + 1 if (kkt < eps_g and df < eps_f) else 0
        self._streak_s = self._streak_s + 1 if s_inf < eps_s else 0
        rec = dict(k=self.k, f=self.f, volume=float(self.a @ self.x), delta=self.delta, kkt=kkt,
                   step=s_inf, theta=theta, accepted=True)
        self.history.append(rec)
        return rec

    def done(self) -> bool:
        return self._streak_fg >= 3 or self._streak_s >= 3 or self.k >= self.max_iter

    def run(self, iterations: int | None = None):
        n = 0
        while not self.done() and (iterations is None or n < iterations):
            self.step()
            n += 1
        return self.history


def volume_row(shape, n_mr: int, rmin: float) -> np.ndarray:
    """a with a^T x = sum_i v_i rho_i for rho = H x (unit total volume,
    equal cells): a = H^T v, H the normalised Gaussian filter of Sec. 2.2
    (ball dist <= r in element units, sigma = r/3, truncated at the domain
    boundary).  shape = (Dz, Dy, Dx)."""
    Dz, Dy, Dx = shape
    N = Dx * Dy * Dz
    v = np.full(N, 1.0 / N)
    if rmin <= 0.0:
        return v
    R = int(np.floor(rmin * n_mr + 1e-9))
    rc2 = (rmin * n_mr) ** 2
    sig = rmin / 3.0
    offs = [(i, j, k) for k in range(-R, R + 1) for j in range(-R, R + 1) for i in range(-R, R + 1)
            if i * i + j * j + k * k <= rc2 * (1.0 + 1e-12)]
    wts = [np.exp(-((i * i + j * j + k * k) / float(n_mr * n_mr)) / (2.0 * sig * sig)) for i, j, k in offs]
    z, y, x = np.meshgrid(np.arange(Dz), np.arange(Dy), np.arange(Dx), indexing="ij")
    omega = np.zeros((Dz, Dy, Dx))
    for (i, j, k), w in zip(offs, wts):
        ok = (x + i >= 0) & (x + i < Dx) & (y + j >= 0) & (y + j < Dy) & (z + k >= 0) & (z + k < Dz)
        omega += w * ok
    vr = (v.reshape(Dz, Dy, Dx) / omega)
    a = np.zeros((Dz, Dy, Dx))
    for (i, j, k), w in zip(offs, wts):  # a_c = sum_i w_ic v_i / omega_i over the ball of c
        src = np.zeros((Dz, Dy, Dx))
        zs, ys, xs = slice(max(k, 0), Dz + min(k, 0)), slice(max(j, 0), Dy + min(j, 0)), slice(max(i, 0), Dx + min(i, 0))
        zd, yd, xd = slice(max(-k, 0), Dz + min(-k, 0)), slice(max(-j, 0), Dy + min(-j, 0)), slice(max(-i, 0), Dx + min(-i, 0))
        src[zd, yd, xd] = vr[zs, ys, xs]
        a += w * src
    return a.reshape(-1)


def gpu_evaluator(T, h, f_host: np.ndarray, nrhs: int, rtol: float = 1e-8, maxit: int = 5000):
    """evaluate(x) -> (compliance summed over load cases, dc/dx) through
    tosolve_step_host; every solve after the first starts from the previous
    displacements."""
    f_host = np.ascontiguousarray(f_host, dtype=np.float64)
    state = {"warm": 0}

    def evaluate(x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        g = np.zeros(x.size)
        c, _ = T.tosolve_step_host(h, x, f_host, nrhs, rtol, maxit, state["warm"], None, g)
        state["warm"] = 1
        return float(np.sum(c)), g

    return evaluate
