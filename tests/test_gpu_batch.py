"""Batched solve (tosolve_batch_*) vs the CPU oracle and vs one-handle solves.

Workload: an uneven batch of Q1 cantilever instances (nx log-uniform, ny = nz
= nx/2, 1..3 load cases each, design variables iid U[0.01, 1]), the small
counterpart of the 64-instance batch.  Tolerances as in the single-handle
parity tests: displacement relative L2 error <= 1e-6 at rtol = 1e-11; and
because a batch branch runs the same kernels with the same fixed-order
reductions as tosolve_solve, its result equals the one-handle result bit for
bit.
"""
import numpy as np
import pytest

import workloads
from oracle import fe
from tests.gpu_helpers import Run, rel

pytestmark = pytest.mark.gpu

FP64, FP32, TF32 = 0, 1, 2


def _setup(probs, precisions):
    runs = [Run(p, prec) for p, prec in zip(probs, precisions)]
    for R in runs:
        R.set_densities()
    return runs


def test_batch_matches_oracle_and_single_solves():
    probs = workloads.batched_instances(5, seed=4, min_nx=8, max_nx=24, mult=4)
    precisions = [FP32, TF32, FP64, FP32, TF32]
    runs = _setup(probs, precisions)
    T = runs[0].T
    torch = runs[0].torch
    us = [torch.zeros((p.nrhs, p.ndof), dtype=torch.float64, device=R.dev) for p, R in zip(probs, runs)]
    b = T.tosolve_batch_create([R.h for R in runs], [p.nrhs for p in probs], [R.f for R in runs], us)
    try:
        infos = T.tosolve_batch_solve(b, 1e-11, 2000, len(runs))
        for p, R, u, inf in zip(probs, runs, us, infos):
            assert inf.status == T.OK and inf.rel_residual <= 1e-11
            ref = fe.Model(p).run(method="splu")
            un = u.cpu().numpy()
            for r in range(p.nrhs):
                assert rel(un[r], ref["u"][r]) <= 1e-6
            u1, inf1 = R.solve(rtol=1e-11)
            assert torch.equal(u1, u), p.name
            assert inf1.total_iterations == inf.total_iterations
        # second run warm-starts from the first result: nothing left to do
        infos = T.tosolve_batch_solve(b, 1e-11, 2000, len(runs))
        assert all(i.total_iterations == 0 and i.status == T.OK for i in infos)
    finally:
        T.tosolve_batch_destroy(b)
        for R in runs:
            R.close()


def test_batch_new_densities_zero_load_and_errors():
    probs = workloads.batched_instances(3, seed=11, min_nx=8, max_nx=16, mult=4, max_rhs=2)
    runs = _setup(probs, [FP32] * 3)
    T = runs[0].T
    torch = runs[0].torch
    runs[1].f.zero_()
    us = [torch.zeros((p.nrhs, p.ndof), dtype=torch.float64, device=R.dev) for p, R in zip(probs, runs)]
    hs = [R.h for R in runs]
    nr = [p.nrhs for p in probs]
    fs = [R.f for R in runs]
    with pytest.raises(T.TosolveError) as e:  # a handle twice
        T.tosolve_batch_create([hs[0], hs[0]], nr[:1] * 2, fs[:1] * 2, us[:1] * 2)
    assert e.value.status == T.EINVAL
    with pytest.raises(T.TosolveError) as e:  # more load cases than max_rhs
        T.tosolve_batch_create(hs, [p.nrhs + 1 for p in probs], fs, us)
    assert e.value.status == T.EINVAL
    b = T.tosolve_batch_create(hs, nr, fs, us)
    try:
        with pytest.raises(T.TosolveError) as e:
            T.tosolve_batch_solve(b, 0.0, 10, 3)
        assert e.value.status == T.EINVAL
        us[1].fill_(1.0)
        infos = T.tosolve_batch_solve(b, 1e-8, 2000, 3)
        assert infos[1].total_iterations == 0 and float(us[1].abs().max()) == 0.0
        # new densities on instance 2, then the same graph solves the new operator
        rng = np.random.default_rng(5)
        p2 = probs[2]
        x2 = rng.uniform(0.2, 1.0, size=p2.x.shape)
        runs[2].set_densities(torch.tensor(x2, device=runs[2].dev))
        us[2].zero_()
        infos = T.tosolve_batch_solve(b, 1e-11, 2000, 3)
        assert infos[2].status == T.OK
        p2.x = x2
        ref = fe.Model(p2).run(method="splu")
        un = us[2].cpu().numpy()
        for r in range(p2.nrhs):
            assert rel(un[r], ref["u"][r]) <= 1e-6
        # maxit too small: ENOTCONV reported per instance
        for u in us:
            u.zero_()
        infos = T.tosolve_batch_solve(b, 1e-11, 1, 3, raise_on_error=False)
        assert infos[0].status == T.ENOTCONV and infos[2].status == T.ENOTCONV
        assert infos[1].status == T.OK
    finally:
        T.tosolve_batch_destroy(b)
        for R in runs:
            R.close()


def test_tune_times_candidates_and_skips_those_not_offered():
    """tosolve_tune on a small cantilever: FP32X2 and FP32 candidates get
    finite, positive solve times; a candidate the library does not offer
    (Chebyshev smoothing at degree 1) records +inf; the pick is one of the
    finite ones."""
    import torch

    from tests.gpu_helpers import desc_for, lib

    T = lib()
    p = workloads.cantilever(16, 8, 8, seed=4)
    dev = torch.device("cuda:0")
    x = torch.tensor(p.x, device=dev)
    f = torch.tensor(np.asarray(p.f), device=dev)
    cands = [desc_for(T, p, 3), desc_for(T, p, 1), desc_for(T, p, 1, smoother=1)]
    ms = T.tosolve_tune(cands, p.mask, x, f, p.nrhs, 1e-8, 500, 3)
    assert ms.shape == (3, 3)
    assert np.all(np.isfinite(ms[:2])) and np.all(ms[:2] > 0)
    assert np.all(np.isinf(ms[2]))
    c = T.tosolve_tune_pick(ms[None], 0.05)
    assert c[0] in (0, 1)
