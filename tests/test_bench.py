"""Host logic of bench.py that needs no GPU.

* The claimed kernel count of one benchmark step equals the ncu launch list
  of the multiresolution cantilever 48x24x24, n = 2, 4 levels, 24 PCG
  iterations with the FP32 V-cycle: 416 launches in one step, three of them
  PyTorch fill kernels (the L2 flush and two zeroed vectors), 413 ours.
* The per-iteration term follows the V-cycle's structure: 4 kernels per
  non-coarsest level, the coarse solve, then direction, q = K p and update
  (the first reduction rides on the finest post-smoothing step); the TF32
  path runs its finest pre and post steps as two kernels each and keeps the
  separate reduction.
"""
import bench


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
