"""Linear-acoustic scattering of the Sec. 3.1 Gaussian pressure pulse by a rigid circular
cylinder: an exact solution derived here from the wave equation (no published data set).

Problem: p_tt = lap p (c = 1) outside r = R, dp/dr = 0 on r = R,
p(x, 0) = eps exp(-a |x - x_s|^2), p_t(x, 0) = 0, a = ln 2 / b^2 (b the half-width), the
source at distance r_s on the ray theta = 0.  The initial state of Sec. 3.1 has uniform density,
so besides sound it carries an entropy mode; that mode is stationary and carries no pressure,
so to linear order p obeys the wave equation with exactly these data.

Radial transform per angular mode n with the Neumann condition (generalised Weber transform):
with phi_k(r) = J_n(k r) Y_n'(k R) - Y_n(k r) J_n'(k R), which satisfies phi_k'(R) = 0,
    f_n(r) = int_0^inf F(k) phi_k(r) k dk / (J_n'(kR)^2 + Y_n'(kR)^2),
    F(k)   = int_R^inf f_n(r) phi_k(r) r dr,
where f_n is the cos(n theta) coefficient of the initial pressure; a component of wavenumber k
evolves as cos(k t).  F needs no quadrature: J_n(k r) cos(n theta) and Y_n(k r) cos(n theta)
solve the Helmholtz equation wherever the Gaussian has weight, and a Gaussian of exponent a
integrates such a u to (pi / a) exp(-k^2 / (4a)) u(x_s) (the heat semigroup acting on an
eigenfunction of the Laplacian; the singular centre of Y_n carries weight exp(-a (r_s - R)^2)).
Hence, with e_0 = 1, e_n = 2 and g = J_n'(kR) / Y_n'(kR) (dividing phi_k by Y_n'(kR) keeps every
factor finite),
    p(r, theta, t) = sum_n e_n cos(n theta) eps / (2a) int_0^inf exp(-k^2 / (4a)) cos(k t)
                     [J_n(k r_s) - g Y_n(k r_s)] [J_n(k r) - g Y_n(k r)] k / (1 + g^2) dk.
For R -> 0, g -> 0 and Graf's addition theorem returns the free-space solution
eps / (2a) int exp(-k^2 / (4a)) cos(k t) J_0(k |x - x_s|) k dk.  Midpoint rule in k.
"""
import math

import numpy as np


def _phi(n, k, r, g):
    """J_n(k r) - g Y_n(k r) for wavenumbers k [nk] and radii r [m] -> [nk, m]; g Y_n is zero
    where g underflows (Y_n then overflows at least as fast at the smaller radius R)."""
    from scipy import special
    arg = np.outer(k, r)
    J = special.jv(n, arg)
    Y = special.yv(n, arg)
    gY = np.where(g[:, None] == 0.0, 0.0, g[:, None] * np.where(np.isfinite(Y), Y, 0.0))
    return J - gY


def scattered_pulse(xp, times, R=0.5, rs=4.0, eps=1e-3, b=0.2, kmax=35.0, nk=8000, nmax=400):
    """Pressure perturbation at points xp [2, m] (cylinder centred at the origin, source at
    (rs, 0)) and times [nt]; returns [nt, m]."""
    from scipy import special
    xp = np.asarray(xp, dtype=float)
    times = np.atleast_1d(np.asarray(times, dtype=float))
    rp = np.hypot(xp[0], xp[1])
    thp = np.arctan2(xp[1], xp[0])
    a = math.log(2.0) / (b * b)
    dk = kmax / nk
    k = (np.arange(nk) + 0.5) * dk
    base = eps / (2.0 * a) * np.exp(-k * k / (4.0 * a)) * k * dk
    ct = np.cos(np.outer(times, k))                        # [nt, nk]
    out = np.zeros((times.size, rp.size))
    for n in range(nmax + 1):
        # Y_n' overflows at small k R for high orders (its recurrence then meets inf - inf):
        # those values are masked just below, so the floating-point warning is expected
        with np.errstate(invalid="ignore", over="ignore"):
            yR = special.yvp(n, k * R)
        jR = special.jvp(n, k * R)
        ok = np.isfinite(yR) & (yR != 0.0)
        g = np.where(ok, jR / np.where(ok, yR, 1.0), 0.0)
        src = _phi(n, k, np.array([rs]), g)[:, 0]           # [nk]
        w = (1.0 if n == 0 else 2.0) * base * src / (1.0 + g * g)
        if n > 10 and np.max(np.abs(w)) < 1e-16 * eps:
            break
        out += (ct * w[None, :]) @ _phi(n, k, rp, g) * np.cos(n * thp)[None, :]
    return out
