"""The autotuner's choice (tosolve_tune_pick, host only: no device is
touched) on synthetic timings: per class the median of the finite repeats,
the fastest candidate, ties to the lower index, and the default (candidate
0) kept unless the winner is faster by more than min_gain."""
import numpy as np
import pytest

from tests.gpu_helpers import lib

INF = float("inf")


def _pick(ms, gain=0.05):
    T = lib()
    return list(T.tosolve_tune_pick(np.array(ms, dtype=np.float64), gain))


def test_fastest_candidate_wins():
    ms = [[[10, 10, 10], [7, 7, 7], [8, 8, 8]],  # 30 % faster: candidate 1
          [[5, 5, 5], [6, 6, 6], [9, 9, 9]]]       # default fastest
    assert _pick(ms) == [1, 0]


def test_default_kept_below_the_minimum_gain():
    ms = [[[10, 10, 10], [9.7, 9.7, 9.7]],  # 3 % < 5 %: keep the default
          [[10, 10, 10], [9.4, 9.4, 9.4]]]  # 6 % > 5 %
    assert _pick(ms, 0.05) == [0, 1]
    assert _pick(ms, 0.0) == [1, 1]


def test_median_ignores_one_outlier_repeat():
    ms = [[[10, 10, 10], [5, 50, 5]]]  # median 5: one slow repeat does not count
    assert _pick(ms) == [1]
    ms = [[[10, 10, 10], [50, 5, 50]]]  # median 50: one fast repeat does not either
    assert _pick(ms) == [0]


def test_failed_candidates_and_classes():
    ms = [[[INF, INF, INF], [8, 8, 8], [7, 7, 7]],  # the default failed: fastest finite
          [[INF, INF, INF], [INF, INF, INF], [INF, INF, INF]],  # nothing ran
          [[10, 10, 10], [1, INF, INF], [9, 9, 9]]]  # 1 finite of 3: not a median
    assert _pick(ms) == [2, -1, 2]


def test_ties_go_to_the_lower_index():
    ms = [[[10, 10, 10], [6, 6, 6], [6, 6, 6]]]
    assert _pick(ms) == [1]


def test_arguments_are_checked():
    T = lib()
    with pytest.raises(T.TosolveError):
        T.tosolve_tune_pick(np.ones((1, 2, 3)), 1.0)
    with pytest.raises(T.TosolveError):
        T.tosolve_tune_pick(np.ones((1, 65, 3)), 0.1)
