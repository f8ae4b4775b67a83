"""Pins of two small parts of the oracle that other pins do not reach.

* The sponge (an absorbing layer of S cells; reading R16): on a periodic box whose state differs
  from the free stream by a constant, every flux difference and viscous term vanishes, so each
  cell's right-hand side is its relaxation -sigma(m) (Q - Q_inf): one rate for all variables,
  sigma_max at the walls, zero from S cells in, successive rates in the ratio of the cubes of
  the remaining fractions, equal wherever the nearest wall is equally far, and nothing on the
  free stream itself.
* The global Lax-Friedrichs speeds (reading R2): alpha_d must be the largest spectral radius over
  the interior of the flux Jacobian along d, here taken from finite differences of the fluxes
  and numpy's eigenvalue routine (not from the formula |u_d| + c).
"""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1905_00182_gb300 import workloads as W  # noqa: E402

G = 1.4


def test_sponge_relaxes_each_cell_at_its_cubic_rate():
    S, smax = 5, 3.0
    spec = W.GridSpec(dim=2, n=(17, 13, 1), lo=(0, 0, 0), hi=(1.7, 1.3, 1), gamma=G, Re=50.0,
                      qinf=W.freestream(2, G, vel=(0.2, -0.1, 0.0)), scheme=W.TENO5,
                      bc=((2, 2), (2, 2), (0, 0)), sponge_cells=S, sponge_sigma=smax)
    # the free stream itself is left alone: the layer acts on Q - Q_inf
    assert np.all(O.rhs(spec, W.rest_state(spec)) == 0.0)
    # a constant offset on a periodic box: no flux difference, no viscous term, only the layer
    dq = np.array([1e-3, -2e-3, 5e-4, 3e-3])
    Q = W.rest_state(spec) + dq[:, None, None, None]
    rate = -O.rhs(spec, Q) / dq[:, None, None, None]
    assert np.all(np.abs(rate - rate[0]) <= 1e-12 * smax)   # one rate per cell, all variables
    r = rate[0, 0]
    nx, ny = spec.n[0], spec.n[1]
    m = np.minimum.outer(np.minimum(np.arange(ny), ny - 1 - np.arange(ny)),
                         np.minimum(np.arange(nx), nx - 1 - np.arange(nx)))
    assert np.allclose(r[m == 0], smax, rtol=1e-14)           # full strength at the walls
    assert np.all(r[m >= S] == 0.0)                           # nothing S cells in
    for k in range(S - 1):                                    # the cube of the remaining fraction
        ratio = r[m == k][0] / r[m == k + 1][0]
        assert math.isclose(ratio, ((S - k) / (S - k - 1)) ** 3, rel_tol=1e-13), (k, ratio)
    for k in range(S):                                        # the nearest wall decides
        assert np.allclose(r[m == k], r[m == k][0], rtol=1e-14)


def test_split_speeds_are_the_largest_jacobian_spectral_radius():
    spec = W.GridSpec(dim=3, n=(7, 6, 5), lo=(0, 0, 0), hi=(1, 1, 1), gamma=G, Re=0.0,
                      qinf=W.freestream(3, G), scheme=W.TENO5)
    Q = W.random_smooth_state(spec, seed=9, amp=0.2, vel0=(0.3, -0.5, 0.1))
    alpha = O.wavespeeds(spec, Q)

    def flux(q, a):
        rho, m, E = q[0], q[1:4], q[4]
        u = m / rho
        p = (G - 1.0) * (E - 0.5 * np.dot(m, u))
        F = np.empty(5)
        F[0] = m[a]
        F[1:4] = m * u[a]
        F[1 + a] += p
        F[4] = (E + p) * u[a]
        return F

    for a in range(3):
        best = 0.0
        for idx in np.ndindex(*Q.shape[1:]):
            q = Q[(slice(None),) + idx]
            J = np.empty((5, 5))
            for k in range(5):
                h = 1e-6 * max(1.0, abs(q[k]))
                e = np.zeros(5)
                e[k] = h
                J[:, k] = (flux(q + e, a) - flux(q - e, a)) / (2 * h)
            best = max(best, float(np.max(np.abs(np.linalg.eigvals(J)))))
        assert math.isclose(alpha[a], best, rel_tol=1e-7), (a, alpha[a], best)
