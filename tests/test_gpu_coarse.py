"""The coarsest level's direct solve on the GPU (Sec. 7.2) against the
oracle's Cholesky solve (oracle/mg.py).  With one multigrid level, one
V-cycle is exactly the coarse solve z = A_c^{-1} b, so the preconditioner
call returns the GPU's explicit inverse applied to b.

The inverse is formed by blocked symmetric Gauss-Jordan sweeps, 16-wide
pivot blocks up to 640 unknowns and 32-wide above, one block sweeping the
next pivot block ahead of the others.  The sizes cover ragged last pivot
blocks and exact multiples for both widths:

* densities iid U[0.01, 1]: FP64 to 1e-11 (the inverse's error is about
  cond(A_c) * 1e-16 and these matrices are well conditioned);
* the I-beam density on the 9x6x5 mesh (void regions at E_min = 1e-9,
  condition number 1.8e10): to 3e-5, within a small multiple of cond * eps;
* the FP32 preconditioner: the FP64 inverse applied to the FP32 right-hand
  side, rounded to FP32 (3e-7).
"""
import numpy as np
import pytest

import workloads
from oracle import fe, mg
from tests.gpu_helpers import Run, rel

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1

# elements -> coarse unknowns (pivot blocks): 2x1x1 -> 36 (16-wide, 3, ragged);
# 3x3x2 -> 144 (16-wide, 9); 4x3x2 -> 180 (16-wide, 12, ragged); 7x3x3 -> 384
# (16-wide, 24); 7x6x3 -> 672 (32-wide, 21); 9x6x5 -> 1260 (32-wide, 40, ragged)
SHAPES = [(2, 1, 1), (3, 3, 2), (4, 3, 2), (7, 3, 3), (7, 6, 3), (9, 6, 5)]


def _case(shape, density, seed):
    p = workloads.cantilever(*shape, n_mr=2, rmin=0.0, density=density, seed=seed, mg_levels=1)
    rho = fe.Model(p).densities(p.x)
    h = mg.Hierarchy(p, rho, 1)
    rng = np.random.default_rng(seed)
    b = np.where(np.asarray(p.mask) == 0, rng.normal(size=p.ndof), 0.0)
    return p, h, b


@pytest.mark.parametrize("shape", SHAPES)
def test_coarse_solve_fp64(shape):
    p, h, b = _case(shape, "uniform", 3)
    R = Run(p, FP64)
    R.set_densities()
    z = R.precondition(b)
    assert rel(z, mg.vcycle(h, b)) <= 1e-11
    R.close()


def test_coarse_solve_void_regions():
    p, h, b = _case((9, 6, 5), "ibeam", 5)
    R = Run(p, FP64)
    R.set_densities()
    z = R.precondition(b)
    assert rel(z, mg.vcycle(h, b)) <= 3e-5
    R.close()


@pytest.mark.parametrize("shape", [(4, 3, 2), (9, 6, 5)])
def test_coarse_solve_fp32(shape):
    p, h, b = _case(shape, "uniform", 7)
    R = Run(p, FP32)
    R.set_densities()
    z = R.precondition(b)
    b32 = b.astype(np.float32).astype(np.float64)
    assert rel(z, mg.vcycle(h, b32)) <= 3e-7
    R.close()
