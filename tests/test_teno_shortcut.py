"""The all-kept shortcut of the fast forms' TENO5, checked against the oracle's TENO5 (Sec. 2,
the TENO5 reconstruction with its cut-off; reading R3) on the CPU.

TENO5 keeps every stencil when tau5 <= 4 (min beta + eps): each gamma_k = (1 + tau5/beta_k)^6
then lies in [1, 5^6], so chi_k >= 1/(3 5^6) = 2.1e-5 > C_T = 1e-5, and the reconstruction is
the optimal linear one.  The FP64 fast form evaluates this sufficient test in FP32, from the
stencil's four FP64 first differences rounded to FP32 (t0 = d2 - d1, u0 = 3 d2 - d1, ...); the
FP32 form evaluates it on its FP32 perturbations.  What must hold is one direction only: a
stencil the test passes is a stencil on which the oracle's TENO5 (every step in FP64) returns
the linear reconstruction.  The test rule is written out here in float32 numpy (each operation
rounded, as the kernels' unfused form would be at worst) and run on smooth, rough and tiny
stencils and on a family constructed at TENO5's cut-off (a test kept too loose -- a threshold
of 6 instead of 4 -- fails here).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402

F = np.float32


def _fp32_test(v):
    """the fast forms' sufficient all-kept test, in float32"""
    d = [F(v[k + 1] - v[k]) for k in range(4)]   # FP64 differences rounded to FP32
    d1, d2, d3, d4 = d
    t = [d2 - d1, d3 - d2, d4 - d3]
    u = [F(3) * d2 - d1, d2 + d3, d4 - F(3) * d3]
    k13 = F(13.0 / 3.0)
    b = [k13 * t[k] * t[k] + u[k] * u[k] for k in range(3)]
    return bool(abs(b[0] - b[2]) <= F(4) * min(b) + F(1.6e-29))


def _linear(v):
    return (2 * v[0] - 13 * v[1] + 47 * v[2] + 27 * v[3] - 3 * v[4]) / 60.0


def _stencils(rng):
    out = []
    x = np.arange(5, dtype=np.float64)
    for _ in range(4000):   # smooth: low-order polynomials plus noise, offsets and scales
        off, scale = rng.normal() * 10.0 ** rng.uniform(-2, 2), 10.0 ** rng.uniform(-14, 0)
        c = rng.normal(size=4)
        out.append(off + scale * (c[0] * x + c[1] * x ** 2 + c[2] * x ** 3
                                  + 10.0 ** rng.uniform(-6, 0) * rng.normal(size=5)))
    for _ in range(3000):   # rough: independent values, steps and spikes
        out.append(rng.normal(size=5) * 10.0 ** rng.uniform(-12, 1))
        s = np.zeros(5)
        s[rng.integers(1, 5):] = 10.0 ** rng.uniform(-12, 0)
        out.append(rng.normal() + s)
    for _ in range(4000):
        # at the cut-off itself: v = (a, 1, 2, 3, e) has beta_1 = 1 (a linear middle), beta_0 =
        # 13/12 a^2 + (a + 2)^2/4 large, and e solves beta_2 = beta_0 + r, so tau5/min beta = r
        # exactly while the two outer gammas stay near 1 -- the configuration in which TENO5
        # cuts soonest (at r = (1e5 - 2)^(1/6) - 1 = 5.81); r spans both sides of the test's 4
        # and of the cut-off
        a = rng.uniform(10.0, 100.0) * rng.choice([-1.0, 1.0])
        r = rng.uniform(3.0, 7.0)
        b0 = 13.0 / 12.0 * a * a + 0.25 * (a + 2.0) ** 2
        # 13/12 (e - 4)^2 + (e - 6)^2 / 4 = b0 + r  ->  (4/3) e^2 - (35/3) e + (79/3 - b0 - r) = 0
        A, B, C = 4.0 / 3.0, -35.0 / 3.0, 79.0 / 3.0 - b0 - r
        e = (-B + np.sqrt(B * B - 4 * A * C)) / (2 * A)
        off, scale = rng.normal(), 10.0 ** rng.uniform(-6, 0)
        out.append(off + scale * np.array([a, 1.0, 2.0, 3.0, e]))
    return out


def test_stencils_the_fp32_test_keeps_are_kept_by_teno5():
    rng = np.random.default_rng(7)
    kept = cut_by_test = 0
    for v in _stencils(rng):
        v = np.asarray(v, dtype=np.float64)
        if not _fp32_test(v):
            cut_by_test += 1
            continue
        kept += 1
        # the oracle's TENO5 keeps all three stencils: its value is the linear reconstruction
        scale = np.max(np.abs(v)) + 1e-300
        assert abs(O.teno5(v) - _linear(v)) <= 1e-14 * scale, v
    # the check is not vacuous: both outcomes occur
    assert kept > 5000 and cut_by_test > 2000, (kept, cut_by_test)


def test_the_test_keeps_smooth_stencils():
    """where data are smooth on the stencil the test passes (the shortcut is the common path)"""
    rng = np.random.default_rng(8)
    x = np.arange(5, dtype=np.float64)
    n = 0
    for _ in range(500):
        v = 1.0 + 1e-3 * np.sin(0.05 * (x + rng.uniform(0, 100)))
        n += _fp32_test(v)
    assert n == 500
