"""tosolve_compliance_noalloc (no device allocation, fixed scratch array) vs
tosolve_compliance_grad's compliance, through the C ABI.

Both sum f_r[d] u_r[d] over the free DOFs in FP64 in different orders, so
they agree to FP64 rounding: relative 1e-13, the tolerance the parity tests
use for FP64 reductions.  Two calls follow each other with different sizes,
so a stale partial sum left in the shared array by the first call would show
in the second.
"""
import numpy as np
import pytest

import workloads
from tests.gpu_helpers import Run

pytestmark = pytest.mark.gpu

FP32 = 1


def _problem(shape, seed, nrhs):
    p = workloads.cantilever(*shape, seed=seed, mg_levels=2)
    if nrhs > 1:
        rng = np.random.default_rng(seed)
        f = np.zeros((nrhs, p.ndof))
        f[0] = p.f[0]
        f[1:] = rng.normal(size=(nrhs - 1, p.ndof))
        p.f = f
    return p


def _solve_and_reference(p):
    R = Run(p, FP32)
    R.set_densities()
    u, _ = R.solve(rtol=1e-10)
    c_ref, _, _ = R.grad(u)
    return R, u, c_ref


def test_noalloc_compliance_matches_handle_two_calls():
    torch = pytest.importorskip("torch")
    cases = [_problem((12, 6, 6), 3, 3), _problem((6, 4, 2), 5, 1)]
    for p in cases:
        R, u, c_ref = _solve_and_reference(p)
        T = R.T
        mask = torch.tensor(p.mask, dtype=torch.uint8, device=R.dev)
        c = torch.full((p.nrhs,), float("nan"), dtype=torch.float64, device=R.dev)
        with torch.cuda.stream(R.stream):
            T.tosolve_compliance_noalloc(R.f, u, mask, p.ndof, p.nrhs, c, R.stream)
        R.stream.synchronize()
        np.testing.assert_allclose(c.cpu().numpy(), c_ref, rtol=1e-13, atol=0.0)
        R.close()


def test_noalloc_rejects_too_many_load_cases():
    torch = pytest.importorskip("torch")
    from tests.gpu_helpers import lib

    T = lib()
    n = 30
    dev = torch.device("cuda:0")
    f = torch.ones((T.NOALLOC_MAX_RHS + 1, n), dtype=torch.float64, device=dev)
    mask = torch.zeros(n, dtype=torch.uint8, device=dev)
    c = torch.zeros(T.NOALLOC_MAX_RHS + 1, dtype=torch.float64, device=dev)
    with pytest.raises(T.TosolveError) as e:
        T.tosolve_compliance_noalloc(f, f, mask, n, T.NOALLOC_MAX_RHS + 1, c)
    assert e.value.status == T.EINVAL and "16" in str(e.value)
    T.tosolve_compliance_noalloc(f, f, mask, n, T.NOALLOC_MAX_RHS, c)
    torch.cuda.synchronize()
    assert np.all(c.cpu().numpy()[: T.NOALLOC_MAX_RHS] == n)


def test_noalloc_grid_stride_sixteen_load_cases():
    """ndof above 608 blocks x 256 threads, so every block strides over the
    vector several times; 16 load cases with a random mask against the
    float64 sum over the free DOFs (numpy, pairwise order)."""
    torch = pytest.importorskip("torch")
    from tests.gpu_helpers import lib

    T = lib()
    n, nrhs = 200_003, T.NOALLOC_MAX_RHS
    rng = np.random.default_rng(41)
    f = rng.normal(size=(nrhs, n))
    u = rng.normal(size=(nrhs, n))
    mask = (rng.random(n) < 0.3).astype(np.uint8)
    ref = (f * u)[:, mask == 0].sum(axis=1)
    dev = torch.device("cuda:0")
    fd, ud = torch.tensor(f, device=dev), torch.tensor(u, device=dev)
    md = torch.tensor(mask, device=dev)
    c = torch.full((nrhs,), float("nan"), dtype=torch.float64, device=dev)
    T.tosolve_compliance_noalloc(fd, ud, md, n, nrhs, c)
    torch.cuda.synchronize()
    # sum of |f u| bounds the rounding of either order
    scale = np.abs(f * u)[:, mask == 0].sum(axis=1)
    np.testing.assert_array_less(np.abs(c.cpu().numpy() - ref), 1e-13 * scale)
