"""The exact solution of tests/sphere_scattering.py (Sec. 3.6: the periodic Gaussian source of
Eq. 16 scattered by a rigid sphere) pinned to what fixes it: the closed-form far field of a
Gaussian source, the time-domain retarded integral (a second route, real arithmetic, no complex
convention), the Helmholtz equation with the source, the Neumann condition on the sphere, the
series' convergence and the small-sphere limit."""
import math

import numpy as np
import pytest

pytest.importorskip("scipy.special")

from tests import sphere_scattering as S  # noqa: E402

R = 0.5
W_ = 2.0 * math.pi / R          # omega of the workload, k = omega (c = 1)
AMP = -0.01
B = 16.0 / (R * R)
A = B * math.log(2.0)
XC = (2.0 * R, 0.0, 0.0)


def test_far_field_matches_the_closed_form():
    # beyond the source: (G * g)(rho) = exp(ik rho)/(k rho) int_0^inf s exp(-a s^2) sin(k s) ds
    # and that integral is sqrt(pi) k / (4 a^1.5) exp(-k^2 / (4a))
    rho = np.array([1.5, 2.7, 4.0])
    U, dU = S.free_field(rho, W_, A)
    m = math.sqrt(math.pi) * W_ / (4.0 * A ** 1.5) * math.exp(-W_ * W_ / (4.0 * A))
    want = np.exp(1j * W_ * rho) / (W_ * rho) * m
    np.testing.assert_allclose(U, want, rtol=1e-10)
    np.testing.assert_allclose(dU, want * (1j * W_ - 1.0 / rho), rtol=1e-10)


@pytest.mark.parametrize("rho,t", [(0.05, 7.3), (0.3, 6.9), (1.1, 8.05), (2.4, 9.6)])
def test_time_domain_retarded_integral(rho, t):
    U, _ = S.free_field([rho], W_, A)
    P = -1j * W_ * AMP * U[0]
    want = S.free_field_time(rho, t, W_, AMP, A)
    scale = abs(P)
    assert abs((P * np.exp(-1j * W_ * t)).real - want) <= 1e-10 * scale


def test_centre_is_the_limit():
    U, dU = S.free_field(np.array([0.0, 1e-6]), W_, A)
    assert abs(U[0] - U[1]) <= 1e-8 * abs(U[0]) and dU[0] == 0.0 and abs(dU[1]) <= 1e-3 * abs(U[0])


@pytest.mark.parametrize("rho", [0.04, 0.12, 0.25])
def test_helmholtz_equation_with_the_source(rho):
    # radial form: U'' + 2 U'/rho + k^2 U = -exp(-a rho^2)
    d = 1e-3
    U, dU = S.free_field(np.array([rho - d, rho, rho + d]), W_, A)
    U2 = (U[2] - 2.0 * U[1] + U[0]) / (d * d)
    res = U2 + 2.0 * dU[1] / rho + W_ * W_ * U[1] + math.exp(-A * rho * rho)
    assert abs(res) <= 1e-4 * math.exp(-A * rho * rho), res
    # the derivative returned is the derivative of the value
    assert abs((U[2] - U[0]) / (2 * d) - dU[1]) <= 1e-4 * abs(dU[1])


def test_neumann_condition_on_the_sphere():
    th = np.array([0.0, 0.4, 1.1, 1.9, 2.6, math.pi])
    d = 1e-5
    pts = lambda r: np.stack([r * np.cos(th), r * np.sin(th) * 0.6, r * np.sin(th) * 0.8])  # noqa: E731
    Pp = S.sphere_source_field(pts(R + d), R, W_, AMP, B, XC)
    Pm = S.sphere_source_field(pts(R - d), R, W_, AMP, B, XC)
    _, g = S.incident(pts(R), W_, AMP, A, XC)
    dinc = np.sum(g * pts(R), axis=0) / R
    dtot = (Pp - Pm) / (2 * d)
    assert np.max(np.abs(dtot)) <= 1e-6 * np.max(np.abs(dinc))
    assert np.max(np.abs(dinc)) > 0


def test_series_converged_and_small_sphere_limit():
    x = np.array([[-2.0, -0.8, 0.7, 1.6, 0.0, 0.0], [0.0, 0.1, 0.0, 0.0, 0.9, 2.5],
                  [0.0, 0.0, 0.2, 0.0, 0.0, 0.0]])
    a40 = S.sphere_source_field(x, R, W_, AMP, B, XC, nterms=40)
    a60 = S.sphere_source_field(x, R, W_, AMP, B, XC, nterms=60)
    assert np.max(np.abs(a40 - a60)) <= 1e-12 * np.max(np.abs(a40))
    free = S.sphere_source_field(x, 0.0, W_, AMP, B, XC)
    # scattering by a sphere of radius R_s << wavelength falls like (k R_s)^3
    small = S.sphere_source_field(x, 1e-3, W_, AMP, B, XC, nterms=8)
    assert np.max(np.abs(small - free)) <= 1e-6 * np.max(np.abs(free))
    # and the rigid sphere of the workload scatters at order one
    assert np.max(np.abs(a40 - free)) >= 0.1 * np.max(np.abs(free))
