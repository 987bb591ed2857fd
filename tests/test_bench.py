"""Host logic of bench.py that needs no GPU.

* kernel_launches is the fallback estimate of our kernels per step (the
  bench line counts them from a traced step when it can).  For the
  multiresolution cantilever 48x24x24, n = 2, 4 levels, 24 PCG iterations
  with the FP32 V-cycle it equals the ncu launch list of one step: 416
  launches, three of them PyTorch fill kernels (the L2 flush and two zeroed
  vectors), 413 ours.
* Its per-iteration term follows the V-cycle's structure: 4 kernels per
  non-coarsest level, the coarse solve, then direction, q = K p and update
  (the first reduction rides on the finest post-smoothing step); the TF32
  path runs its finest pre and post steps as two kernels each and keeps the
  separate reduction.
* Variant labels name the preconditioner's precision and the inner FP32
  PCG iterations; only the combinations the library accepts are timed.
"""
import pytest

import bench
import workloads


def test_launch_count_matches_the_launch_list():
    assert bench.kernel_launches(4, 24) == 413


def test_launch_count_per_iteration():
    one = bench.kernel_launches(4, 1)
    two = bench.kernel_launches(4, 2)
    assert two - one == 4 * 3 + 1 + 3
    assert bench.kernel_launches(4, 2, tc=True) - bench.kernel_launches(4, 1, tc=True) == 4 * 3 + 1 + 3 + 3
    # triquadratic: pre, post (product + gather each), restriction (element-wise + gather),
    # prolongation per level; reduction, direction, q = K p (three kernels), update
    assert bench.kernel_launches(5, 2, degree=2) - bench.kernel_launches(5, 1, degree=2) == 7 * 4 + 1 + 6


def test_variant_labels():
    assert bench.parse_variant("f16x3+i16") == ("f16x3", 16)
    assert bench.parse_variant("fp32") == ("fp32", 0)
    assert bench.parse_variant("bf16+i8") == ("bf16", 8)
    assert bench.parse_variant("f16x3+i16+c2") == ("f16x3", 16) and bench.cheb_of("f16x3+i16+c2") == 2
    assert bench.cheb_of("fp32+i4") == 0
    for bad in ("f16", "fp32+i", "fp32+ix", "int8", "fp32+", "fp32+x2"):
        with pytest.raises(ValueError):
            bench.parse_variant(bad)
    for wl, text in bench.DEFAULT_VARIANTS.items():
        for v in text.split(","):
            bench.parse_variant(v)


def test_variants_offered_per_problem():
    q1 = workloads.cantilever(8, 4, 4, n_mr=2)
    q2 = workloads.bridge(4, 2, 2, degree=2, n_mr=3)
    mixed = workloads.with_mixed_degree(q2, 0.5, 1)
    assert bench.variant_ok("tf32", q1) and bench.variant_ok("fp32x2", q1)
    assert not bench.variant_ok("f16x3", q1) and not bench.variant_ok("fp32+i4", q1)
    for p in (q2, mixed):
        for v in ("f16x3+i16", "bf16x3", "bf16+i8", "tf32", "fp32+i4", "fp32"):
            assert bench.variant_ok(v, p), v
        assert not bench.variant_ok("fp32x2+i4", p)
        assert bench.variant_ok("f16x3+i16+c2", p) and not bench.variant_ok("fp32x2+c2", p)
    assert not bench.variant_ok("fp32+c2", q1)
    # the default workload's variants are all offered on it
    p = bench.problem(bench.SPECS[bench.DEFAULT_WORKLOAD], sample=True)
    assert all(bench.variant_ok(v, p) for v in bench.DEFAULT_VARIANTS[bench.DEFAULT_WORKLOAD].split(","))


def test_percentiles():
    v = list(range(1, 101))
    assert bench.pct(v, 0.5) == 50 and bench.pct(v, 0.99) == 99 and bench.pct([3.0], 0.99) == 3.0
