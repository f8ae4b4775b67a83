"""Pins of the periodic Gaussian pressure source (Sec. 3.6, Eq. 16) in the oracle.

The source enters the energy equation as A_p / (gamma - 1), A_p = amp exp(-b ln2 r^2) cos(w t).
In a periodic box at rest every flux difference vanishes, so (i) the energy right-hand side is
the source alone and sums to the Gaussian integral amp cos(w t) (pi / (b ln2))^(d/2) / (gamma-1);
(ii) the box's total energy obeys dE/dt = I cos(w t) exactly, and SSP-RK3 with its stage times
t, t + dt, t + dt/2 and weights 1/6, 1/6, 2/3 integrates it as Simpson's rule does, within
Simpson's error bound of the exact I sin(w T) / w."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00182_gb300 import workloads as W


def _box(dim, n, amp=-0.01, b=8.0, omega=2.0 * math.pi, xc=(0.1, -0.2, 0.05)):
    g = 1.4
    spec = W.GridSpec(dim=dim, n=(n, n, n if dim == 3 else 1), lo=(-2.0, -2.0, -2.0),
                      hi=(2.0, 2.0, 2.0 if dim == 3 else 1.0), gamma=g, Re=100.0,
                      qinf=W.freestream(dim, g), scheme=W.TENO5,
                      bc=((2, 2), (2, 2), (2, 2) if dim == 3 else (0, 0)))
    spec.src_amp, spec.src_b, spec.src_omega, spec.src_xc = amp, b, omega, xc
    return spec


@pytest.mark.parametrize("dim,n", [(2, 64), (3, 32)])
def test_source_is_the_gaussian_integral(dim, n):
    spec = _box(dim, n)
    Q = W.rest_state(spec)
    t = 0.37
    L = O.rhs(spec, Q, t=t)
    assert np.all(L[: spec.nv - 1] == 0.0)
    vol = float(np.prod(spec.h))
    total = L[spec.nv - 1].sum() * vol
    exact = spec.src_amp * math.cos(spec.src_omega * t) / (spec.gamma - 1.0) * \
        (math.pi / (spec.src_b * math.log(2.0))) ** (dim / 2.0)
    assert abs(total - exact) <= 1e-8 * abs(exact)
    # first moment: the source is centred on xc
    xs = W.node_coords(spec)
    for a in range(dim):
        shape = [1] * 3
        shape[2 - a] = -1
        m1 = (L[spec.nv - 1] * xs[a].reshape(shape)).sum() * vol / total
        assert abs(m1 - spec.src_xc[a]) <= 1e-8


def test_rk3_integrates_the_source_as_simpsons_rule():
    spec = _box(2, 48, amp=-0.01, b=8.0, omega=3.0)
    Q = W.rest_state(spec)
    dt, n, t0 = 0.05, 12, 0.2
    vol = float(np.prod(spec.h))
    E0 = Q[spec.nv - 1].sum() * vol
    Q1, _ = O.rk3(spec, Q, dt, nsteps=n, t=t0)
    dE = Q1[spec.nv - 1].sum() * vol - E0
    I = spec.src_amp / (spec.gamma - 1.0) * math.pi / (spec.src_b * math.log(2.0))
    w, T = spec.src_omega, n * dt
    exact = I * (math.sin(w * (t0 + T)) - math.sin(w * t0)) / w
    bound = T * dt ** 4 * w ** 4 * abs(I) / 2880.0  # Simpson: (b-a) h^4 max|f''''| / 2880
    err = abs(dE - exact)
    assert err <= 1.05 * bound + 1e-13
    # a first-order clock (every stage at the step start) would miss by far more
    assert 0.5 * abs(I) * w * dt * T / 2 > 20 * bound
    # mass and momentum of the box are untouched
    for c in range(spec.nv - 1):
        assert abs((Q1[c] - Q[c]).sum() * vol) <= 1e-10 * abs(exact)
