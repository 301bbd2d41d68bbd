"""Host helpers of the inversion driver (no GPU): the time-to-misfit clock, the held-out tear
sizes and the summary statistics."""
import numpy as np

from paper_2311_05322_gb300 import inversion


def test_first_time_below_stops_at_the_first_reaching_iterate():
    J = [1.0, 0.5, 0.31, 0.30002, 0.29]
    secs = [0.0, 1.0, 2.0, 3.0, 4.0]
    assert inversion.first_time_below(J, secs, 0.3) == 4.0
    # within the band of the solves' tolerance the fourth iterate already counts
    assert inversion.first_time_below(J, secs, 0.3 * (1 + inversion.TARGET_REL_BAND)) == 3.0
    assert inversion.first_time_below(J, secs, 0.1) is None
    assert 0 < inversion.TARGET_REL_BAND <= 1e-3


def test_held_out_tears_span_the_size_range():
    n = 6
    means = []
    for k in range(n):
        t = inversion.held_out_tear(3, k, n)
        assert all(0.002 - 1e-12 <= a <= 0.010 + 1e-12 for a in t.semi_axes)
        means.append(sum(t.semi_axes) / 3)
    assert means == sorted(means)                      # sizes grow with k
    assert means[0] < 0.004 and means[-1] > 0.007      # the 2-10 mm range, both ends
    # the same tear for the same seed and index (the target of a given run is reproducible)
    a, b = inversion.held_out_tear(3, 2, n), inversion.held_out_tear(3, 2, n)
    assert a.center == b.center and a.semi_axes == b.semi_axes


def test_stats_skip_missing_times():
    st = inversion._stats([1.0, None, 3.0])
    assert st["n"] == 2 and st["mean"] == 2.0 and st["min"] == 1.0 and st["max"] == 3.0
    assert abs(st["std"] - np.std([1.0, 3.0], ddof=1)) < 1e-15
    assert inversion._stats([None]) == {"n": 0}
