"""The host SLP loop (Sec. 4) driven by the GPU solver through the C ABI
(tosolve_step_host, warm starts) against the same loop driven by the CPU
oracle: the compliance histories agree (the solves match to 1e-7; the LP
steps are the same vertices), and both stay feasible."""
import numpy as np
import pytest

import workloads
from oracle import fe
from paper_2311_05595_gb300.slp import SLP, gpu_evaluator, volume_row
from tests.gpu_helpers import Run

pytestmark = pytest.mark.gpu


def test_gpu_slp_follows_the_oracle_slp():
    p = workloads.cantilever(12, 6, 6, n_mr=2, rmin=1.5, density="solid", seed=0, mg_levels=2)
    p.x = np.full(p.x.size, 0.3)
    a = volume_row(p.density_shape, p.n_mr, p.rmin)
    m = fe.Model(p)

    def oracle_eval(x):
        out = m.run(x=x, method="splu")
        return float(out["c"].sum()), out["g_x"]

    R = Run(p, 3)
    gpu_eval = gpu_evaluator(R.T, R.h, np.asarray(p.f), p.nrhs, rtol=1e-11)
    ref = SLP(oracle_eval, a, 0.3, p.x, delta0=0.1).run(iterations=8)
    got = SLP(gpu_eval, a, 0.3, p.x, delta0=0.1).run(iterations=8)
    R.close()
    assert len(got) == len(ref)
    f_ref = np.array([h["f"] for h in ref])
    f_got = np.array([h["f"] for h in got])
    np.testing.assert_allclose(f_got, f_ref, rtol=1e-5)
    assert f_got[-1] < 0.7 * f_got[0]
    assert all(h["volume"] <= 0.3 + 1e-9 for h in got)
