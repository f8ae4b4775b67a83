"""The IB + fluid coupling of the oracle against linear acoustics: Sec. 3.1's Gaussian pulse
scattered by a rigid cylinder (Eqs. 6-11 with the penalty law of Eq. 7).  The exact solution
(tests/acoustic_scattering.py, derived there) is first pinned to what fixes it -- the initial
pulse at t = 0, the free-space solution as R -> 0, a vanishing normal derivative on the
cylinder -- and then the oracle's probe histories are compared with it at D/h = 12.8."""
import math

import numpy as np
import pytest

from oracle import oracle as O

from tests import cases
from tests.acoustic_scattering import scattered_pulse

pytest.importorskip("scipy.special")


def _free_space(r, t, eps=1e-3, b2=0.04):
    from scipy import special
    a = math.log(2.0) / b2
    k = np.linspace(0.0, 12.0 * math.sqrt(a), 40001)
    f = np.exp(-k * k / (4.0 * a)) * k
    return np.array([eps / (2.0 * a) * np.trapezoid(f * np.cos(k * t) * special.j0(k * rr), k)
                     for rr in np.atleast_1d(r)])


def test_exact_scattering_solution_is_pinned():
    # t = 0: the initial pulse, cylinder or not
    xp = np.array([[4.0, 4.1, 3.8], [0.0, 0.1, -0.15]])
    p0 = scattered_pulse(xp, [0.0], nk=2500)[0]
    np.testing.assert_allclose(p0, 1e-3 * np.exp(-math.log(2.0) * ((xp[0] - 4) ** 2 + xp[1] ** 2)
                                                 / 0.04), rtol=1e-6)
    # R -> 0: the free-space solution (Hankel transform of the pulse)
    xq = np.array([[2.0, 2.0], [0.0, 2.0]])
    ts = np.array([2.0, 2.8, 4.0])
    small = scattered_pulse(xq, ts, R=1e-3, nk=2500)
    free = np.array([_free_space(np.hypot(xq[0] - 4.0, xq[1]), t) for t in ts])
    assert np.max(np.abs(small - free)) <= 1e-6 * 1e-3   # signal peak ~8e-5
    # rigid wall: dp/dr = 0 on r = R while the pulse passes (one-sided second-order difference)
    th = np.array([0.0, 0.7, 2.0])
    d = 1e-4
    ring = [scattered_pulse(np.array([(0.5 + j * d) * np.cos(th), (0.5 + j * d) * np.sin(th)]),
                            [3.6, 4.5], nk=2500) for j in range(3)]
    dpdr = (-3.0 * ring[0] + 4.0 * ring[1] - ring[2]) / (2.0 * d)
    assert np.max(np.abs(dpdr)) <= 1e-3 * np.max(np.abs(ring[0])) / 0.2


def _oracle_history(case):
    Q, xi = case["Q"], None
    out = []
    for _ in range(case["samples"]):
        Q, xi = O.rk3(case["spec"], Q, case["dt"], case["every"], case["X"], case["U"],
                      case["dS"], xi)
        out.append(O.probe(case["spec"], Q, case["probes"]))
    return np.array(out)


def test_oracle_scatters_the_pulse_off_the_cylinder():
    case = cases.cylinder_scattering(12.8)
    got = _oracle_history(case)
    t = case["sample"] * np.arange(1, case["samples"] + 1)
    want = scattered_pulse(case["probes"], t, nk=2500)
    err = np.sqrt(np.sum((got - want) ** 2) / np.sum(want ** 2))
    # the wave reflected by the cylinder reaches (2, 0) at t ~ 5; without a cylinder this
    # window's error is the whole signal (relative error ~ 1)
    w = (t >= 4.5) & (t <= 6.5)
    err_refl = np.sqrt(np.sum((got[w, 0] - want[w, 0]) ** 2) / np.sum(want[w, 0] ** 2))
    print(f"D/h 12.8: relative RMS of the probe histories {err:.4f}, reflected pulse {err_refl:.4f}")
    assert err <= 0.16, err
    assert err_refl <= 0.4, err_refl
