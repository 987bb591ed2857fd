"""Host SLP loop (Sec. 4, Algorithm 2) on a small cantilever, driven by the
CPU oracle (no GPU): accepted steps decrease the compliance, the volume and
box constraints hold, the volume row is the filter transpose of the cell
volumes."""
import numpy as np

import workloads
from oracle import fe
from paper_2311_05595_gb300.slp import SLP, volume_row


def _oracle_eval(p):
    m = fe.Model(p)

    def ev(x):
        out = m.run(x=x, method="dense")
        return float(out["c"].sum()), out["g_x"]

    return m, ev


def test_volume_row_is_filter_transpose():
    p = workloads.cantilever(4, 2, 2, n_mr=2, rmin=1.5, seed=0)
    m = fe.Model(p)
    a = volume_row(p.density_shape, p.n_mr, p.rmin)
    v = np.full(p.x.size, 1.0 / p.x.size)
    np.testing.assert_allclose(a, m.H.T @ v, rtol=1e-12)


def test_slp_decreases_compliance_within_constraints():
    p = workloads.cantilever(6, 3, 3, n_mr=1, rmin=1.5, density="solid", seed=0)
    p.x = np.full(p.x.size, 0.3)
    m, ev = _oracle_eval(p)
    a = volume_row(p.density_shape, p.n_mr, p.rmin)
    slp = SLP(ev, a, 0.3, p.x, delta0=0.1)
    hist = slp.run(iterations=12)
    fs = [h["f"] for h in hist]
    assert all(f1 <= f0 * (1 + 1e-12) for f0, f1 in zip(fs, fs[1:]))
    assert fs[-1] < 0.8 * fs[0]
    assert float(a @ slp.x) <= 0.3 + 1e-9
    assert slp.x.min() >= 0.0 and slp.x.max() <= 1.0
