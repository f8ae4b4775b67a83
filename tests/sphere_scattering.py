"""Time-harmonic sound of the periodic Gaussian source of Eq. 16 scattered by a rigid sphere
(Sec. 3.6): an exact linear-acoustics solution derived here from the wave equation (no
published data set).

Problem, in the solver's units (rho = c = 1 at rest).  The source adds A(x) cos(w t)/(gamma-1)
to the energy equation, which is A(x) cos(w t) in the linearised pressure equation, so
    p_tt - lap p = d/dt [H(t) A(x) cos(w t)],   A(x) = amp exp(-a |x - x_c|^2),  a = b ln 2,
outside the sphere r = R (centre at the origin) with dp/dr = 0 on it.  In 3D the retarded
solution forgets the switch-on once every retarded time is positive, and the sphere's creeping
waves decay exponentially, so the field settles to p = Re[P(x) exp(-i w t)] with
    lap P + k^2 P = i w A(x),  k = w,   P = P_inc + P_sc,
    P_inc = -i w amp (G * g),  g(y) = exp(-a |y - x_c|^2),  G(x) = exp(i k |x|) / (4 pi |x|).

Free field.  The mean of G over the sphere |y - x_c| = s seen from a point at distance rho is
(exp(ik(rho + s)) - exp(ik |rho - s|)) / (2 i k rho s), hence
    (G * g)(rho) = 1 / (2 i k rho) int_0^inf exp(-a s^2) s [exp(ik(rho + s)) - exp(ik |rho - s|)] ds,
integrated by Gauss-Legendre quadrature split at the kink s = rho.

Scattered field, axisymmetric about the line through the centre and the source (x axis):
    P_sc(r, mu) = sum_n c_n h_n(k r) P_n(mu),   mu = cos(angle from +x),  h_n = j_n + i y_n,
    c_n = -(2n + 1) / (2 k h_n'(kR)) int_{-1}^{1} dP_inc/dr (R, mu) P_n(mu) dmu
(the Neumann condition, term by term, with Gauss-Legendre quadrature in mu).

The time-domain form of the free field, used to pin the frequency-domain one:
    p(x, t) = -amp int_0^inf exp(-a s^2) s / (2 rho) [cos(w(t - rho - s)) - cos(w(t - |rho - s|))] ds
for t beyond the last retarded arrival (t > rho + the source's extent).
"""
from __future__ import annotations

import functools

import numpy as np
from numpy.polynomial.legendre import leggauss


@functools.lru_cache(maxsize=None)
def _nodes(n):
    return leggauss(n)


def _gl(lo, hi, n):
    x, w = _nodes(n)
    return 0.5 * (hi - lo) * x + 0.5 * (hi + lo), 0.5 * (hi - lo) * w


def _segments(rho, smax):
    return [(0.0, rho), (rho, smax)] if rho < smax else [(0.0, smax)]


def free_field(rho, k, a, nq=600):
    """(G * exp(-a|.|^2)) at distances rho >= 0 from the Gaussian's centre and its derivative
    in rho (complex arrays)."""
    rho = np.atleast_1d(np.asarray(rho, dtype=np.float64))
    smax = 12.0 / np.sqrt(a)  # exp(-144) beyond
    U = np.empty(rho.shape, dtype=np.complex128)
    dU = np.empty_like(U)
    for i, r in enumerate(rho.flat):
        if r < 1e-9 * smax:  # the centre: the mean of G over |y| = s is exp(iks) / (4 pi s)
            s, w = _gl(0.0, smax, nq)
            U.flat[i] = np.sum(w * np.exp(-a * s * s) * s * np.exp(1j * k * s))
            dU.flat[i] = 0.0
            continue
        I = 0.0 + 0.0j
        dI = 0.0 + 0.0j
        for lo, hi in _segments(r, smax):
            s, w = _gl(lo, hi, nq)
            gs = np.exp(-a * s * s) * s
            e1 = np.exp(1j * k * (r + s))
            e2 = np.exp(1j * k * np.abs(r - s))
            I += np.sum(w * gs * (e1 - e2))
            dI += np.sum(w * gs * (1j * k * e1 - 1j * k * np.sign(r - s) * e2))
        U.flat[i] = I / (2j * k * r)
        dU.flat[i] = -U.flat[i] / r + dI / (2j * k * r)
    return U, dU


def free_field_time(rho, t, w, amp, a, nq=600):
    """The free field's pressure at distance rho and time t from the retarded integral (real,
    time domain; valid once t exceeds rho plus the source's extent)."""
    smax = 12.0 / np.sqrt(a)
    out = 0.0
    for lo, hi in _segments(rho, smax):
        s, wq = _gl(lo, hi, nq)
        f = np.exp(-a * s * s) * s / (2.0 * rho)
        out += np.sum(wq * f * (np.cos(w * (t - rho - s)) - np.cos(w * (t - np.abs(rho - s)))))
    return -amp * out


def incident(x, w, amp, a, xc):
    """P_inc at points x [3][np] and its gradient [3][np]."""
    x = np.asarray(x, dtype=np.float64)
    d = x - np.asarray(xc, dtype=np.float64)[:, None]
    rho = np.sqrt(np.sum(d * d, axis=0))
    U, dU = free_field(rho, w, a)
    P = -1j * w * amp * U
    safe = np.where(rho > 0.0, rho, 1.0)
    grad = np.where(rho > 0.0, -1j * w * amp * dU / safe, 0.0)[None, :] * d
    return P, grad


def _hn(n, z, derivative=False):
    from scipy import special
    return (special.spherical_jn(n, z, derivative=derivative)
            + 1j * special.spherical_yn(n, z, derivative=derivative))


def scattering_coefficients(R, w, amp, a, xc, nterms=40, nmu=160):
    """c_n of the scattered field (x_c on the +x axis)."""
    from scipy import special
    mu, wm = _nodes(nmu)
    xs = np.stack([R * mu, R * np.sqrt(1.0 - mu * mu), np.zeros_like(mu)])
    _, grad = incident(xs, w, amp, a, xc)
    dPdr = np.sum(grad * xs, axis=0) / R
    c = np.empty(nterms, dtype=np.complex128)
    for n in range(nterms):
        proj = np.sum(wm * dPdr * special.eval_legendre(n, mu))
        c[n] = -(2 * n + 1) / (2.0 * w * _hn(n, w * R, derivative=True)) * proj
    return c


def scattered(x, R, w, coef):
    """P_sc at points x [3][np] (outside or on the sphere)."""
    from scipy import special
    x = np.asarray(x, dtype=np.float64)
    r = np.sqrt(np.sum(x * x, axis=0))
    mu = x[0] / r
    P = np.zeros(r.shape, dtype=np.complex128)
    for n, cn in enumerate(coef):
        P += cn * _hn(n, w * r) * special.eval_legendre(n, mu)
    return P


def sphere_source_field(x, R, w, amp, b, xc, nterms=40):
    """Complex amplitude P (p = Re[P exp(-i w t)]) of the settled field at points x [3][np]:
    the Gaussian source amp exp(-b ln2 |x - x_c|^2) cos(w t) of Eq. 16 (x_c on the +x axis) and
    a rigid sphere of radius R at the origin (R = 0: free field)."""
    a = b * np.log(2.0)
    P, _ = incident(x, w, amp, a, xc)
    if R > 0.0:
        P = P + scattered(x, R, w, scattering_coefficients(R, w, amp, a, xc, nterms))
    return P
