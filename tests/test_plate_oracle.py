"""Pins of the plate oracle (oracle/plate_oracle.c): the ANCF plate of Eq. 1, its clamp motion
(Eq. 17) and the coupled plate-fluid step, checked against what mechanics fixes independently
of the discretisation: Euler-Bernoulli closed forms, the elastica by shooting, natural
frequencies (k_1 = 1.8751 of Sec. 4.1), matrices by independent quadrature, finite
differences, and conservation laws."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00182_gb300 import workloads as W


def hermite_basis(l):
    """Cubic Hermite basis on [0, l] derived here from its defining conditions (value and
    slope at both ends), as monomial coefficients: basis i has value/slope 1 at condition i."""
    # conditions: p(0), p'(0), p(l), p'(l) for p = c0 + c1 s + c2 s^2 + c3 s^3
    A = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [1, l, l * l, l ** 3], [0, 1, 2 * l, 3 * l * l]],
                 dtype=float)
    return np.linalg.solve(A, np.eye(4))  # column i = coefficients of basis i


def poly_matrix(l, deriv):
    """int_0^l p_i^(deriv) p_j^(deriv) ds for the Hermite basis, by Gauss-Legendre (exact)."""
    C = hermite_basis(l)
    x, w = np.polynomial.legendre.leggauss(8)
    s = 0.5 * l * (x + 1.0)
    w = 0.5 * l * w
    vals = []
    for i in range(4):
        p = np.polynomial.Polynomial(C[:, i]).deriv(deriv)
        vals.append(p(s))
    vals = np.array(vals)
    return (vals * w) @ vals.T


def global_from_scalar(ps, Ms):
    nd = ps.ndof
    M = np.zeros((nd, nd))
    for el in range(ps.n_el):
        for i in range(4):
            for j in range(4):
                for a in range(2):
                    I = 4 * el + 4 * (i // 2) + 2 * (i % 2) + a
                    J = 4 * el + 4 * (j // 2) + 2 * (j % 2) + a
                    M[I, J] += Ms[i, j]
    return M


def test_mass_and_bending_matrices_by_quadrature():
    ps = W.PlateSpec(n_el=5, n_markers=10, length=1.3, rho_s=0.7, K_S=0.0, K_B=2.5, clamped=0)
    e, _ = W.plate_straight(ps, origin=(0.1, -0.2), theta=0.3)
    _, K, M = O.plate_internal(ps, e, tangent=True, mass=True)
    l = ps.length / ps.n_el
    M_ref = global_from_scalar(ps, ps.rho_s * poly_matrix(l, 0))
    K_ref = global_from_scalar(ps, ps.K_B * poly_matrix(l, 2))
    assert np.max(np.abs(M - M_ref)) <= 1e-14 * np.max(np.abs(M_ref))
    assert np.max(np.abs(K - K_ref)) <= 1e-12 * np.max(np.abs(K_ref))
    # total mass: a rigid translation carries rho_s L
    tx = np.zeros(ps.ndof)
    tx[0::4] = 1.0
    assert abs(tx @ M @ tx - ps.rho_s * ps.length) <= 1e-14


def test_cantilever_uniform_load_matches_euler_bernoulli():
    ps = W.PlateSpec(n_el=40, n_markers=800, K_S=1e4, K_B=1.0, clamped=1, newton_tol=1e-10)
    e0, _ = W.plate_straight(ps)
    q = 1e-5
    F = np.zeros((2, ps.n_markers))
    F[1] = q
    e, it = O.plate_static(ps, e0, O.plate_load(ps, F))
    s = np.arange(ps.n_el + 1) * ps.length / ps.n_el
    L, EI = ps.length, ps.K_B
    w = q * s ** 2 * (6 * L * L - 4 * L * s + s * s) / (24 * EI)      # deflection
    th = q * s * (3 * L * L - 3 * L * s + s * s) / (6 * EI)           # slope
    tip = q * L ** 4 / (8 * EI)
    # nodal values of cubic Hermite elements are exact for Euler-Bernoulli; what is left is the
    # marker (midpoint) quadrature of the load and O((w/L)^2) geometric non-linearity
    assert np.max(np.abs(e[1::4] - w)) <= 1e-6 * tip
    assert np.max(np.abs(e[3::4] - th)) <= 1e-6 * q * L ** 3 / (6 * EI)
    assert it <= 5


def test_uniform_stretch_under_end_load():
    ps = W.PlateSpec(n_el=12, n_markers=24, K_S=50.0, K_B=0.3, clamped=1)
    e0, _ = W.plate_straight(ps)
    P = 0.7
    Qf = np.zeros(ps.ndof)
    Qf[4 * ps.n_el] = P                    # axial force on the tip node
    e, _ = O.plate_static(ps, e0, Qf)
    eps = P / ps.K_S                       # tension K_S (|r_s| - 1) = P everywhere
    s = np.arange(ps.n_el + 1) * ps.length / ps.n_el
    assert np.max(np.abs(e[0::4] - s * (1.0 + eps))) <= 1e-13
    assert np.max(np.abs(e[2::4] - (1.0 + eps))) <= 1e-13
    assert np.max(np.abs(e[1::4])) <= 1e-15 and np.max(np.abs(e[3::4])) <= 1e-15


def elastica_tip(P_over_EI, L=1.0):
    """Tip of a clamped elastica under a transverse dead end load, by shooting on
    theta'' = -(P/EI) cos(theta), theta(0) = 0, theta'(L) = 0 (zero end moment)."""
    from scipy.integrate import solve_ivp
    from scipy.optimize import brentq

    def run(k0):
        f = lambda s, y: [y[1], -P_over_EI * math.cos(y[0]), math.cos(y[0]), math.sin(y[0])]
        return solve_ivp(f, (0.0, L), [0.0, k0, 0.0, 0.0], rtol=1e-12, atol=1e-14)

    k0 = brentq(lambda k: run(k).y[1, -1], 0.0, P_over_EI * L * 1.01)
    y = run(k0).y[:, -1]
    return y[2], y[3], y[0]


@pytest.mark.parametrize("load", [1.0, 3.0])
def test_large_deflection_converges_to_the_elastica(load):
    """P L^2 / K_B = 1 and 3 (tip rotations of 27 and 58 degrees).  K_S / K_B = 1e7 keeps the
    stretch below 3e-7; the thin element locks in membrane at coarse meshes, so the error falls
    quickly with refinement (static Newton limited by the conditioning: tolerance 1e-9)."""
    x, y, th = elastica_tip(load)
    errs = []
    for ne in (20, 40, 80):
        ps = W.PlateSpec(n_el=ne, n_markers=2 * ne, K_S=1e7, K_B=1.0, clamped=1,
                         newton_tol=1e-9)
        e, _ = W.plate_straight(ps)
        for frac in np.linspace(0.25, 1.0, 4):  # load stepping
            Qf = np.zeros(ps.ndof)
            Qf[4 * ps.n_el + 1] = frac * load
            e, _ = O.plate_static(ps, e, Qf)
        errs.append(max(abs(e[-4] - x), abs(e[-3] - y), abs(math.atan2(e[-1], e[-2]) - th)))
    assert errs[0] > 8 * errs[1] > 64 * errs[2]
    assert errs[2] <= 5e-7


def periods(ts, ys):
    zc = [ts[i] - ys[i] * (ts[i + 1] - ts[i]) / (ys[i + 1] - ys[i])
          for i in range(len(ys) - 1) if ys[i] * ys[i + 1] < 0]
    return (zc[-1] - zc[0]) / ((len(zc) - 1) / 2.0)


def test_first_bending_frequency_of_cantilever():
    # omega_1 = k_1^2 / L^2 sqrt(K_B / rho_s), k_1 = 1.8751 (Sec. 4.1); start in the mode shape
    k1 = 1.8751040687119611
    ps = W.PlateSpec(n_el=40, n_markers=80, K_S=1e4, K_B=1.0, rho_s=1.0, clamped=1)
    sig = (math.cosh(k1) + math.cos(k1)) / (math.sinh(k1) + math.sin(k1))
    s = np.arange(ps.n_el + 1) / ps.n_el
    e, v = W.plate_straight(ps)
    e = e.reshape(-1, 4)
    e[:, 1] = 1e-4 * (np.cosh(k1 * s) - np.cos(k1 * s) - sig * (np.sinh(k1 * s) - np.sin(k1 * s)))
    e[:, 3] = 1e-4 * k1 * (np.sinh(k1 * s) + np.sin(k1 * s) - sig * (np.cosh(k1 * s) - np.cos(k1 * s)))
    e = e.ravel()
    T = 2 * math.pi / (k1 * k1)
    assert abs(1.8751 ** 2 / (k1 * k1) - 1.0) < 1e-5
    dt = T / 400
    ys = [e[-3]]
    for n in range(1200):
        e, v, _ = O.plate_step(ps, e, v, (n + 1) * dt, dt)
        ys.append(e[-3])
    Tm = periods(np.arange(len(ys)) * dt, np.array(ys))
    # the midpoint rule lengthens the period by (omega dt)^2 / 12 = 2.1e-5
    assert abs(Tm / T - 1.0 - (2 * math.pi / 400) ** 2 / 12) <= 2e-6


def test_first_axial_frequency_of_clamped_free_rod():
    # omega = (pi / 2L) sqrt(K_S / rho_s)
    ps = W.PlateSpec(n_el=40, n_markers=80, K_S=4.0, K_B=1e-6, rho_s=1.0, clamped=1)
    s = np.arange(ps.n_el + 1) / ps.n_el
    e, v = W.plate_straight(ps)
    e = e.reshape(-1, 4)
    amp = 1e-5
    e[:, 0] = s + amp * np.sin(0.5 * math.pi * s)
    e[:, 2] = 1.0 + amp * 0.5 * math.pi * np.cos(0.5 * math.pi * s)
    e = e.ravel()
    om = 0.5 * math.pi * math.sqrt(ps.K_S / ps.rho_s)
    T = 2 * math.pi / om
    dt = T / 400
    xs = [e[-4] - 1.0]
    for n in range(1200):
        e, v, _ = O.plate_step(ps, e, v, (n + 1) * dt, dt)
        xs.append(e[-4] - 1.0)
    Tm = periods(np.arange(len(xs)) * dt, np.array(xs))
    assert abs(Tm / T - 1.0 - (2 * math.pi / 400) ** 2 / 12) <= 5e-6


def deformed_state(ps, seed=5):
    r = W.splitmix64(seed, 2 * ps.ndof)
    e, v = W.plate_straight(ps, origin=(0.2, -0.1), theta=0.4)
    e = e + 0.05 * (r[: ps.ndof] - 0.5)
    v = v + 0.5 * (r[ps.ndof:] - 0.5)
    return e, v


def test_tangent_is_the_derivative_of_the_internal_force():
    ps = W.PlateSpec(n_el=6, n_markers=12, K_S=30.0, K_B=0.2, clamped=0)
    e, _ = deformed_state(ps)
    _, K, _ = O.plate_internal(ps, e, tangent=True)
    h = 1e-6
    Kfd = np.zeros_like(K)
    for j in range(ps.ndof):
        ep, em = e.copy(), e.copy()
        ep[j] += h
        em[j] -= h
        Kfd[:, j] = (O.plate_internal(ps, ep)[0] - O.plate_internal(ps, em)[0]) / (2 * h)
    assert np.max(np.abs(K - Kfd)) <= 1e-7 * np.max(np.abs(K))
    assert np.max(np.abs(K - K.T)) <= 1e-12 * np.max(np.abs(K))


def momenta(ps, e, v):
    _, _, M = O.plate_internal(ps, e, mass=True)
    tx = np.zeros(ps.ndof)
    tx[0::4] = 1.0
    ty = np.zeros(ps.ndof)
    ty[1::4] = 1.0
    px, py = tx @ M @ v, ty @ M @ v
    xi = np.r_[0:ps.ndof:4, 2:ps.ndof:4]
    xi.sort()
    Ms = M[np.ix_(xi, xi)]
    Jz = e[xi] @ Ms @ v[xi + 1] - e[xi + 1] @ Ms @ v[xi]  # int rho (x y_t - y x_t) ds
    return px, py, Jz


def test_free_plate_conserves_momentum_and_angular_momentum():
    ps = W.PlateSpec(n_el=10, n_markers=20, K_S=40.0, K_B=0.05, clamped=0)
    e, v = deformed_state(ps)
    p0 = momenta(ps, e, v)
    e1, v1, _ = O.plate_step(ps, e, v, 0.01, 0.01, nsteps=50)
    p1 = momenta(ps, e1, v1)
    assert np.max(np.abs(e1 - e)) > 0.05            # the plate has moved and deformed
    for a, b in zip(p0, p1):
        assert abs(a - b) <= 1e-12 * (1.0 + abs(a))


def test_free_plate_takes_the_impulse_of_a_uniform_load():
    ps = W.PlateSpec(n_el=10, n_markers=40, K_S=40.0, K_B=0.05, clamped=0)
    e, v = deformed_state(ps)
    F = np.zeros((2, ps.n_markers))
    F[0], F[1] = 0.3, -0.2
    Qf = O.plate_load(ps, F)
    dt, n = 0.01, 20
    px0, py0, _ = momenta(ps, e, v)
    e1, v1, _ = O.plate_step(ps, e, v, dt, dt, Qf=Qf, nsteps=n)
    px1, py1, _ = momenta(ps, e1, v1)
    assert abs((px1 - px0) - n * dt * 0.3 * ps.length) <= 1e-12
    assert abs((py1 - py0) + n * dt * 0.2 * ps.length) <= 1e-12


def test_clamp_motion_follows_eq17_and_its_rates_are_derivatives():
    ps = W.PlateSpec(x0=(0.3, -0.4), theta0=0.2, A0=1.5, freq=0.7, beta=1.1, alpha_m=0.9,
                     phi=0.4)
    for t in (0.0, 0.37, 1.9):
        e4, v4 = O.plate_motion(ps, t)
        w = 2 * math.pi * ps.freq
        X0 = np.array(ps.x0) + 0.5 * ps.A0 * math.cos(w * t) * np.array([math.cos(ps.beta),
                                                                          math.sin(ps.beta)])
        al = 0.5 * ps.alpha_m * math.sin(w * t + ps.phi)
        assert np.allclose(e4, [X0[0], X0[1], math.cos(ps.theta0 + al),
                                math.sin(ps.theta0 + al)], rtol=0, atol=1e-15)
        h = 1e-6
        fd = (O.plate_motion(ps, t + h)[0] - O.plate_motion(ps, t - h)[0]) / (2 * h)
        assert np.max(np.abs(fd - v4)) <= 1e-8


def test_clamped_plate_follows_its_clamp():
    w = W.flapping_plate_2d(n=(64, 32))
    ps = w["plate"]
    e, v = w["e"], w["v"]
    dt = 0.05
    e1, v1, it = O.plate_step(ps, e, v, dt, dt, nsteps=10)
    t = dt
    for _ in range(9):
        t = t + dt  # the clamp time as the steps accumulate it
    ep, vp = O.plate_motion(ps, t)
    # the clamp holds the root position and the direction of the slope, not its length
    assert np.array_equal(e1[:2], ep[:2]) and np.array_equal(v1[:2], vp[:2])
    assert abs(e1[2] * ep[3] - e1[3] * ep[2]) <= 1e-15
    assert 0.0 < e1[2] * ep[2] + e1[3] * ep[3] and abs(np.hypot(e1[2], e1[3]) - 1.0) < 1e-4
    assert it <= 6
    # the plate stays (nearly) inextensible: node spacing within K-proportional strain
    seg = np.hypot(np.diff(e1[0::4]), np.diff(e1[1::4]))
    assert np.max(np.abs(seg / (ps.length / ps.n_el) - 1.0)) < 1e-3


def test_coupled_step_balances_momentum_in_a_periodic_box():
    """Penalty forces pass momentum between fluid and plate only: in a periodic box (no
    boundary fluxes, no sponge) the fluid's total momentum plus the free plate's is constant."""
    g = 1.4
    spec = W.GridSpec(dim=2, n=(48, 40, 1), lo=(-1.5, -1.25, 0.0), hi=(1.5, 1.25, 1.0), gamma=g,
                      Re=300.0, qinf=W.freestream(2, g, vel=(0.1, 0.0, 0.0)), scheme=W.TENO5,
                      bc=((2, 2), (2, 2), (0, 0)), max_markers=40)
    h = spec.h[0]
    dt = 0.5 / (2.2 / h)
    spec.alpha_pen, spec.beta_pen = W.penalty_defaults(h, dt)
    ps = W.PlateSpec(n_el=6, n_markers=40, length=1.0, rho_s=0.5, K_S=50.0, K_B=0.01, clamped=0)
    Q = W.random_smooth_state(spec, seed=7, amp=1e-3, vel0=(0.1, 0.0, 0.0), periodic=True)
    e, v = W.plate_straight(ps, origin=(-0.5, 0.05), theta=0.2, omega=0.05)
    xi = np.zeros((2, ps.n_markers))
    cell = h * spec.h[1]

    def total(Q, e, v):
        px, py, _ = momenta(ps, e, v)
        return np.array([Q[1].sum() * cell + px, Q[2].sum() * cell + py])

    P0 = total(Q, e, v)
    Q1, xi1, e1, v1, t1, iters = O.fsi_step(spec, ps, Q, xi, e, v, 0.0, dt, nsteps=4)
    P1 = total(Q1, e1, v1)
    moved = abs(momenta(ps, e1, v1)[0] - momenta(ps, e, v)[0])
    assert moved > 1e-4                      # the plate was pushed by the stream
    assert np.max(np.abs(P1 - P0)) <= 1e-12 * moved + 1e-15
    assert abs(t1 - 4 * dt) <= 1e-15 and max(iters) <= 6


def test_plate_force_is_the_impulse_the_fluid_loses():
    """Eq. 19 numerators: a uniform load gives force q L and power q.U L; through a coupled step
    in a periodic box the fluid's momentum changes by exactly -dt times the plate force."""
    ps = W.PlateSpec(n_el=5, n_markers=50, clamped=0)
    F = np.zeros((2, 50))
    F[0], F[1] = 0.4, -0.3
    U = np.zeros((2, 50))
    U[0], U[1] = 0.5, 2.0
    f, pw = O.plate_force(ps, F, U)
    assert np.allclose(f, [0.4, -0.3], rtol=0, atol=1e-15) and abs(pw - (0.2 - 0.6)) <= 1e-15
    g = 1.4
    spec = W.GridSpec(dim=2, n=(48, 40, 1), lo=(-1.5, -1.25, 0.0), hi=(1.5, 1.25, 1.0), gamma=g,
                      Re=300.0, qinf=W.freestream(2, g, vel=(0.1, 0.0, 0.0)), scheme=W.TENO5,
                      bc=((2, 2), (2, 2), (0, 0)), max_markers=40)
    h = spec.h[0]
    dt = 0.5 / (2.2 / h)
    spec.alpha_pen, spec.beta_pen = W.penalty_defaults(h, dt)
    ps = W.PlateSpec(n_el=6, n_markers=40, rho_s=0.5, K_S=50.0, K_B=0.01, clamped=0)
    Q = W.random_smooth_state(spec, seed=7, amp=1e-3, vel0=(0.1, 0.0, 0.0), periodic=True)
    e, v = W.plate_straight(ps, origin=(-0.5, 0.05), theta=0.2, omega=0.05)
    X, Uk, _ = O.plate_markers(ps, e, v)
    Q1, _, _, _, _, _ = O.fsi_step(spec, ps, Q, np.zeros((2, 40)), e, v, 0.0, dt, nsteps=1)
    f, pw = O.plate_force(ps, O.fsi_last_load(ps), Uk)
    cell = h * spec.h[1]
    dP = np.array([(Q1[1] - Q[1]).sum() * cell, (Q1[2] - Q[2]).sum() * cell])
    assert np.max(np.abs(dP + dt * f)) <= 1e-12 * np.max(np.abs(dt * f))
    assert abs(pw) > 0
