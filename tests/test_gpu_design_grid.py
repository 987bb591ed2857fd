"""Coarser design grid (d_mr < n_mr, Sec. 3.2 Eq. projdsgn) on the GPU vs
the oracle: densities (FP64 rounding, 1e-14 relative), and the whole path
(displacement 1e-6, compliance 1e-7, design gradient 1e-6 at rtol 1e-11)."""
import numpy as np
import pytest

import workloads
from oracle import fe
from tests.gpu_helpers import Run, rel

pytestmark = pytest.mark.gpu

FP64, FP32X2 = 0, 3


@pytest.mark.parametrize("n,d,r", [(3, 2, 0.6), (2, 1, 0.9), (4, 2, 0.6)])
def test_projected_densities_match_oracle(n, d, r):
    import torch

    p = workloads.with_design_grid(workloads.cantilever(6, 4, 4, n_mr=n, rmin=r, seed=2, mg_levels=2), d, 5)
    R = Run(p, FP64)
    R.set_densities()
    rho = torch.zeros(n ** 3 * 96, dtype=torch.float64, device=R.dev)
    R.T.tosolve_densities(R.h, rho, None)
    R.stream.synchronize()
    ref = fe.Model(p).densities(p.x)
    assert rel(rho.cpu().numpy(), ref) <= 1e-14
    R.close()


@pytest.mark.parametrize("precision", [FP64, FP32X2])
def test_coarser_design_grid_whole_path(precision):
    p = workloads.with_design_grid(
        workloads.cantilever(12, 6, 6, n_mr=3, rmin=0.6, seed=1, mg_levels=2), 2, 7)
    ref = fe.Model(p).run(method="splu")
    R = Run(p, precision)
    R.set_densities()
    u, info = R.solve(rtol=1e-11)
    assert rel(u.cpu().numpy()[0], ref["u"][0]) <= 1e-6
    import torch

    gx = torch.zeros(p.x.size, dtype=torch.float64, device=R.dev)
    gr = torch.zeros(27 * 432, dtype=torch.float64, device=R.dev)
    with torch.cuda.stream(R.stream):
        c = R.T.tosolve_compliance_grad(R.h, u, R.f[:1].contiguous(), 1, gx, gr)
    R.stream.synchronize()
    assert abs(c[0] - ref["c"][0]) <= 1e-7 * abs(ref["c"][0])
    assert rel(gr.cpu().numpy(), ref["g_rho"]) <= 1e-6
    assert rel(gx.cpu().numpy(), ref["g_x"]) <= 1e-6
    R.close()
