"""Physics pins of the oracle: what linear acoustics and the penalty method fix.

* Sec. 3.1's initial Gaussian pressure pulse (rho uniform, u = 0) propagates, to linear order,
  by the 2D wave equation with c = 1; its exact solution is the Hankel transform
  p(r, t) = eps/(2a) int_0^inf exp(-k^2/(4a)) cos(k t) J0(k r) k dk, a = ln 2 / 0.04.
  The oracle must converge to it (pins the Euler fluxes, the sound speed and the r^-1/2
  cylindrical spreading).
* The penalty law of Eq. 7 must drive the interpolated fluid velocity at the markers to the
  wall velocity: a cylinder spun up impulsively in fluid at rest loses its slip.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00182_gb300 import workloads as W


def _exact_pulse(r, t, eps=1e-3, b2=0.04):
    special = pytest.importorskip("scipy.special")
    a = math.log(2.0) / b2
    k = np.linspace(0.0, 12.0 * math.sqrt(a), 40001)
    f = np.exp(-k * k / (4.0 * a)) * k
    return np.array([eps / (2.0 * a) * np.trapezoid(f * np.cos(k * t) * special.j0(k * rr), k)
                     for rr in np.atleast_1d(r)])


def test_exact_solution_quadrature_reproduces_the_initial_pulse():
    r = np.array([0.0, 0.1, 0.2, 0.35])
    np.testing.assert_allclose(_exact_pulse(r, 0.0), 1e-3 * np.exp(-math.log(2.0) * r * r / 0.04),
                               rtol=1e-6, atol=1e-15)


def _pulse_error(n):
    spec = W.GridSpec(dim=2, n=(n, n, 1), lo=(-4, -4, 0), hi=(4, 4, 1), Re=0.0,
                      qinf=W.freestream(2, 1.4), scheme=W.WENO5JS)
    Q = W.gaussian_pulse_state(spec, (0.0, 0.0))
    h = spec.h[0]
    dt = 0.5 / (2.0 / h)
    xp = np.array([[1.0, 0.0, 1.5 / math.sqrt(2.0), -1.5], [0.0, 1.0, 1.5 / math.sqrt(2.0), 0.0]])
    rp = np.hypot(xp[0], xp[1])
    every = int(round(0.1 / dt))
    err, peak = 0.0, 0.0
    for s in range(int(round(2.0 / dt))):
        Q, _ = O.rk3(spec, Q, dt, 1)
        if (s + 1) % every == 0:
            want = _exact_pulse(rp, (s + 1) * dt)
            err = max(err, np.max(np.abs(O.probe(spec, Q, xp) - want)))
            peak = max(peak, np.max(np.abs(want)))
    return err / peak


def test_acoustic_pulse_converges_to_linear_acoustics():
    coarse, fine = _pulse_error(80), _pulse_error(160)
    # 2 and 4 points per half-width; at 4 the probe histories are within 5 % of the peak
    assert fine <= 0.05, fine
    assert coarse / fine >= 3.0, (coarse, fine)


def test_penalty_law_enforces_no_slip():
    n = 64
    spec = W.GridSpec(dim=2, n=(n, n, 1), lo=(-1.5, -1.5, 0), hi=(1.5, 1.5, 1), Re=1000.0,
                      qinf=W.freestream(2, 1.4), scheme=W.TENO5, max_markers=100)
    h = spec.h[0]
    dt = 0.5 / (2.0 / h)
    spec.alpha_pen, spec.beta_pen = W.penalty_defaults(h, dt)
    X, U, dS = W.circle_markers(100, 0.5, omega=0.2)
    Q = W.random_smooth_state(spec, 1, amp=0.0)
    xi = None
    slip = []
    for s in range(60):
        Q, xi = O.rk3(spec, Q, dt, 1, X, U, dS, xi)
        if s % 10 == 9:
            _, _, rate, _ = O.rhs(spec, Q, X, U, dS, xi, return_markers=True)
            slip.append(np.sqrt((rate ** 2).sum(0).mean() / (U ** 2).sum(0).mean()))
    assert all(b < a for a, b in zip(slip[:4], slip[1:4])), slip
    assert slip[-1] < 0.01, slip
