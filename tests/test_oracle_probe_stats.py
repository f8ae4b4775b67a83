"""Time statistics of probe signals (Sec. 3.2: dp~ = dp - its time mean, and the RMS of dp~
plotted on rings in Sec. 3.3 and 4) in the oracle, pinned to closed forms and to the standard
library's exactly rounded population standard deviation; the Doppler ring of Sec. 3.3."""
import math
import statistics

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00182_gb300 import workloads as W



@pytest.mark.parametrize("N", [3, 7, 64, 1000])
def test_sampled_sinusoid_over_whole_periods(N):
    # sum_t sin^2(2 pi t / N + phi) = N / 2 for N > 2: mean c, RMS A / sqrt(2)
    t = np.arange(N)
    c = np.array([0.0, 3.0, -1e3])
    A = np.array([1.0, 1e-4, 2.5])
    phi = np.array([0.3, 1.1, -2.0])
    h = c + A * np.sin(2.0 * math.pi * t[:, None] / N + phi)
    mean, rms = O.probe_stats(h)
    assert np.all(np.abs(mean - c) <= 1e-13 * (np.abs(c) + A))
    assert np.allclose(rms, A / math.sqrt(2.0), rtol=1e-12, atol=0.0)


def test_two_samples_and_constant_and_empty():
    mean, rms = O.probe_stats(np.array([[1.0, 5.0, 2.0], [3.0, -1.0, 2.0]]))
    assert np.array_equal(mean, [2.0, 2.0, 2.0])
    assert np.array_equal(rms, [1.0, 3.0, 0.0])
    mean, rms = O.probe_stats(np.zeros((0, 4)))
    assert np.array_equal(mean, np.zeros(4)) and np.array_equal(rms, np.zeros(4))


def test_against_exactly_rounded_library_statistics():
    rng = np.random.default_rng(7)
    # a small fluctuation on a large offset (the case the mean removal exists for)
    h = 1e3 + 1e-3 * rng.standard_normal((500, 6)) + np.linspace(-1, 1, 6)
    mean, rms = O.probe_stats(h)
    for k in range(h.shape[1]):
        col = [float(v) for v in h[:, k]]
        # a float sum of n terms errs by at most (n - 1) eps sum|x|, so the mean by (n - 1) eps max|x|
        assert abs(mean[k] - statistics.fmean(col)) <= len(col) * 2.0 ** -52 * max(map(abs, col))
        assert abs(rms[k] / statistics.pstdev(col) - 1.0) <= 1e-9


def test_mean_removal_is_shift_invariant():
    rng = np.random.default_rng(3)
    h = rng.standard_normal((200, 5))
    m0, r0 = O.probe_stats(h)
    m1, r1 = O.probe_stats(h + 0.5)
    assert np.allclose(m1, m0 + 0.5, rtol=0, atol=1e-15)
    assert np.allclose(r1, r0, rtol=1e-13, atol=0)


def test_doppler_ring():
    R, M = 75.0, 0.2
    xp = W.doppler_ring_probes(8, R, M, center=(1.0, -2.0))
    r = np.hypot(xp[0] - 1.0, xp[1] + 2.0)
    th = np.arctan2(xp[1] + 2.0, xp[0] - 1.0)
    assert np.allclose(r, R * (1.0 - M * np.cos(th)), rtol=1e-14)
    assert math.isclose(r[0], R * (1 - M)) and math.isclose(r[4], R * (1 + M))
    assert math.isclose(r[2], R) and math.isclose(r[6], R)
