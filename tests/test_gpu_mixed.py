"""Mixed trilinear / triquadratic meshes (tosolve_create_mixed) vs the mixed
oracle (oracle/mixed.py).  Tolerances as for uniform degree: the reduced
FP64 operator to FP64 rounding (1e-13), solves at rtol 1e-11 to displacement
1e-6, compliance 1e-7, gradient 1e-6.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import fe, mixed
from tests.gpu_helpers import Run, rel

pytestmark = pytest.mark.gpu

FP64, FP32, FP32X2 = 0, 1, 3


def _mixed_bridge(frac=0.5, seed=3, shape=(8, 4, 4), n=2, levels=3):
    p = workloads.bridge(*shape, degree=2, n_mr=n, seed=seed, mg_levels=levels)
    return workloads.with_mixed_degree(p, frac, seed)


def test_mixed_operator_and_unknowns_match_oracle():
    q = _mixed_bridge()
    m = mixed.MixedModel(q)
    w = m.weights(m.densities(q.x))
    A = (m.T.T @ m.assemble(w) @ m.T).tocsr()
    held = (q.mask != 0) | m.slaved
    keep = sp.diags((~held).astype(float))
    A = (keep @ A @ keep + sp.diags(held.astype(float))).tocsr()
    x = np.random.default_rng(0).normal(size=q.ndof)
    R = Run(q, FP32X2)
    R.set_densities()
    assert rel(R.apply(0, FP64, x), A @ x) <= 1e-13
    assert R.T.tosolve_free_dofs(R.h) == m.free.size
    R.close()


@pytest.mark.parametrize("precision", [FP64, FP32, FP32X2])
@pytest.mark.parametrize("frac", [0.5, 0.2])
def test_mixed_bridge_matches_oracle(precision, frac):
    q = _mixed_bridge(frac=frac)
    ref = mixed.MixedModel(q).run(method="splu")
    R = Run(q, precision)
    R.set_densities()
    u, info = R.solve(rtol=1e-11)
    assert info.rel_residual <= 1e-11
    assert rel(u.cpu().numpy()[0], ref["u"][0]) <= 1e-6
    c, gx, gr = R.grad(u)
    assert abs(c[0] - ref["c"][0]) <= 1e-7 * abs(ref["c"][0])
    assert rel(gr, ref["g_rho"]) <= 1e-6
    assert rel(gx, ref["g_x"]) <= 1e-6
    R.close()


def test_all_trilinear_mixed_equals_degree_one_path():
    """All elements trilinear: the vertex values are the degree-1 solution.
    (The coarse levels of a mixed hierarchy are triquadratic, so the cycle
    is weaker here than on a genuinely mixed mesh: rtol 1e-10.)"""
    q = _mixed_bridge(frac=1.0, shape=(8, 4, 4), n=1, levels=3)
    p1 = workloads.bridge(8, 4, 4, degree=1, n_mr=1, seed=3, mg_levels=3)
    Rq = Run(q, FP64)
    Rq.set_densities()
    uq, _ = Rq.solve(rtol=1e-10)
    cq, gq, _ = Rq.grad(uq)
    R1 = Run(p1, FP64)
    R1.set_densities()
    u1, _ = R1.solve(rtol=1e-10)
    c1, g1, _ = R1.grad(u1)
    Lx, Ly, Lz = q.lattice
    vert = [2 * i + Lx * (2 * j + Ly * 2 * l) for l in range(5) for j in range(5) for i in range(9)]
    uv = uq.cpu().numpy()[0].reshape(-1, 3)[vert].reshape(-1)
    assert rel(uv, u1.cpu().numpy()[0]) <= 1e-6
    assert abs(cq[0] - c1[0]) <= 1e-7 * c1[0]
    assert rel(gq, g1) <= 1e-6
    Rq.close()
    R1.close()
