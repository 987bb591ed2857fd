"""Serving runtime (tosolve_server_*): results alone vs in the mix, HBM
admission with eviction, parity of a served request with the oracle.

A served request is one SLP iteration of a design: x -> densities, a solve
warm-started from the design's previous displacements, compliance and
gradient.  Every kernel uses fixed-order reductions and launch shapes that
do not depend on what else runs, so a request's result in a mix of
concurrent designs (or after its design was evicted and rebuilt with the
saved warm start) must equal the result of the same request sequence run
alone, bit for bit.
"""
import numpy as np
import pytest

import workloads
from oracle import fe
from tests.gpu_helpers import desc_for, lib, rel

pytestmark = pytest.mark.gpu

FP32, FP32X2 = 1, 3
GiB = 1 << 30


def _designs():
    probs = workloads.batched_instances(4, seed=21, min_nx=8, max_nx=24, mult=8, max_rhs=2)
    probs.append(workloads.cantilever(16, 8, 8, n_mr=2, rmin=1.0, density="smooth", seed=3,
                                      mg_levels=3))
    precisions = [FP32X2, FP32, FP32X2, FP32, FP32X2]
    return probs, precisions


def _sequences(probs, n_iter, seed=5):
    """Per design, n_iter design vectors: the problem's x, then SLP-like
    drifts x <- clip(x + U(-0.05, 0.05), 0.001, 1)."""
    rng = np.random.default_rng(seed)
    seqs = []
    for p in probs:
        xs = [np.array(p.x, dtype=np.float64)]
        for _ in range(n_iter - 1):
            xs.append(np.clip(xs[-1] + rng.uniform(-0.05, 0.05, size=p.x.shape), 0.001, 1.0))
        seqs.append(xs)
    return seqs


def _design_bytes(T, p, precision):
    d = desc_for(T, p, precision)
    ncell = p.x.size
    return T.tosolve_footprint(d) + (2 * ncell + 2 * p.nrhs * p.ndof) * 8


def _serve(T, probs, precisions, seqs, order, slots, budget, rtol=1e-10):
    """Runs the requests (design, step) in `order`; returns {(design, step):
    (result, dcdx)} and the final stats."""
    s = T.tosolve_server_create(slots, budget, rtol, 2000)
    try:
        for k, (p, prec) in enumerate(zip(probs, precisions)):
            T.tosolve_server_add_design(s, k, desc_for(T, p, prec), p.mask, np.asarray(p.f), p.nrhs)
        grads, key_of = {}, {}
        for k, step in order:
            g = np.full(probs[k].x.size, np.nan)
            rid = T.tosolve_server_submit(s, k, seqs[k][step], g)
            grads[(k, step)] = g
            key_of[rid] = (k, step)
        import time

        out, done = {}, []
        deadline = time.monotonic() + 300.0
        while len(done) < len(order):
            assert time.monotonic() < deadline, "requests did not finish"
            got = T.tosolve_server_poll(s, 64, 2000)
            st = T.tosolve_server_stats(s)
            assert got or st.running + st.pending > 0
            done += got
        for r in done:
            key = key_of[r.request]
            out[key] = (r, grads[key])
        return out, T.tosolve_server_stats(s), done
    finally:
        T.tosolve_server_destroy(s)


def test_served_results_equal_alone_and_in_order():
    T = lib()
    probs, precisions = _designs()
    n_iter = 3
    seqs = _sequences(probs, n_iter)
    alone = {}
    for k in range(len(probs)):
        res, _, _ = _serve(T, [probs[k]], [precisions[k]], [seqs[k]],
                           [(0, i) for i in range(n_iter)], 1, 8 * GiB)
        for i in range(n_iter):
            alone[(k, i)] = res[(0, i)]
    order = [(k, i) for i in range(n_iter) for k in range(len(probs))]  # interleaved
    mix, stats, done = _serve(T, probs, precisions, seqs, order, 4, 8 * GiB)
    for key, (r, g) in mix.items():
        ra, ga = alone[key]
        assert r.status == T.OK and ra.status == T.OK, key
        assert r.rel_residual <= 1e-10
        assert r.compliance == ra.compliance, key
        assert np.array_equal(g, ga), key
        assert r.iterations == ra.iterations, key
        assert r.t_submit <= r.t_start <= r.t_end
    # requests of one design finish in submission order; warm starts help
    for k in range(len(probs)):
        ends = [mix[(k, i)][0].t_end for i in range(n_iter)]
        assert ends == sorted(ends)
        assert mix[(k, 1)][0].iterations <= mix[(k, 0)][0].iterations
    assert stats.builds == len(probs) and stats.evictions == 0


def test_admission_evicts_idle_designs_and_restores_warm_starts():
    T = lib()
    probs, precisions = _designs()
    n_iter = 3
    seqs = _sequences(probs, n_iter, seed=9)
    need = [_design_bytes(T, p, q) for p, q in zip(probs, precisions)]
    budget = int(max(need) * 1.5)  # about one design resident at a time
    order = [(k, i) for i in range(n_iter) for k in range(len(probs))]
    roomy, _, _ = _serve(T, probs, precisions, seqs, order, 2, 8 * GiB)
    tight, stats, _ = _serve(T, probs, precisions, seqs, order, 2, budget)
    assert stats.evictions > 0 and stats.builds > len(probs)
    for key in order:
        r, g = tight[key]
        r0, g0 = roomy[key]
        assert r.status == T.OK
        assert r.compliance == r0.compliance, key
        assert np.array_equal(g, g0), key
    # a design larger than the whole budget is refused, not queued forever
    s = T.tosolve_server_create(1, 1 << 20, 1e-8, 100)
    try:
        p = probs[0]
        T.tosolve_server_add_design(s, 0, desc_for(T, p, FP32), p.mask, np.asarray(p.f), p.nrhs)
        T.tosolve_server_submit(s, 0, p.x)
        got = T.tosolve_server_poll(s, 4, 5000)
        assert len(got) == 1 and got[0].status == T.ENOMEM
        msgs = T.tosolve_server_failures(s)
        assert len(msgs) == 1 and "status 2" in msgs[0] and "design 0" in msgs[0]
    finally:
        T.tosolve_server_destroy(s)


def test_failed_requests_are_logged_with_their_reason():
    """maxit = 1: every request ends ENOTCONV; the failure log holds the
    newest 64, newest first, each with its status, iterations and residual."""
    T = lib()
    p = workloads.cantilever(8, 4, 4, seed=2, mg_levels=2)
    s = T.tosolve_server_create(2, 4 * GiB, 1e-10, 1)
    try:
        T.tosolve_server_add_design(s, 7, desc_for(T, p, FP32X2), p.mask, np.asarray(p.f), p.nrhs)
        ids = [T.tosolve_server_submit(s, 7, p.x) for _ in range(70)]
        done = []
        while len(done) < len(ids):
            done += T.tosolve_server_poll(s, 64, 5000)
        assert all(r.status == T.ENOTCONV and r.iterations == 1 for r in done)
        msgs = T.tosolve_server_failures(s)
        assert len(msgs) == 64
        assert msgs[0].startswith(f"request {ids[-1]} design 7 status 3 its 1")
        assert all("status 3" in m and "maxit" in m for m in msgs)
    finally:
        T.tosolve_server_destroy(s)


def test_served_request_matches_oracle():
    T = lib()
    p = workloads.cantilever(12, 6, 6, n_mr=2, rmin=1.0, seed=4, mg_levels=2)
    ref = fe.Model(p).run(method="splu")
    res, _, _ = _serve(T, [p], [FP32X2], [[p.x]], [(0, 0)], 1, 8 * GiB, rtol=1e-11)
    r, g = res[(0, 0)]
    assert r.status == T.OK and r.cold == 1
    assert abs(r.compliance - ref["c"].sum()) <= 1e-7 * abs(ref["c"].sum())
    assert rel(g, ref["g_x"]) <= 1e-6
