"""Pins of the FP64 CPU oracle against what arXiv:1905.00182 and the mathematics fix.

Each test checks the oracle against something other than itself: values of Eq. 11 evaluated by
hand, moment identities of Peskin's kernel, adjointness and conservation of Eq. 8/9, closed
forms of the fifth-order reconstructions, convergence orders of the discretisation of Eq. 2-5
(the viscous target is derived symbolically from the continuous equations), free-stream
preservation, the exact amplification polynomial of third-order Runge-Kutta, and the exact
entropy-wave solution of the equations.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00182_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------------------------------
# Peskin kernel (Eq. 10-11)
# ------------------------------------------------------------------------------------------

def test_lambda_golden_values():
    for r, val in _read_golden("peskin_lambda.txt"):
        assert O.lam(float(r)) == pytest.approx(float(val), abs=1e-16, rel=1e-15)


def test_lambda_moment_identities():
    # Peskin's four-point construction: for every shift r, sum_j lambda(r-j) = 1, the first
    # moment vanishes, the even and odd sums are 1/2 each and sum_j lambda(r-j)^2 = 3/8.
    rng = np.random.default_rng(0)
    for r in np.concatenate([rng.random(2000), [0.0, 0.25, 0.5, 0.999999999999]]):
        js = np.arange(-3, 5)
        w = np.array([O.lam(r - j) for j in js])
        assert abs(w.sum() - 1.0) < 1e-15
        assert abs(((r - js) * w).sum()) < 1e-15
        assert abs(w[js % 2 == 0].sum() - 0.5) < 1e-15
        assert abs((w * w).sum() - 0.375) < 1e-15


def test_lambda_continuity_and_support():
    for r in (1.0, 2.0):
        left, right = O.lam(r - 1e-13), O.lam(r + 1e-13)
        assert abs(left - right) < 1e-6
    assert O.lam(2.0) == 0.0 and O.lam(-2.0) == 0.0 and O.lam(3.7) == 0.0
    assert O.lam(0.3) == O.lam(-0.3)


# ------------------------------------------------------------------------------------------
# Interpolation / spreading (Eq. 8-9)
# ------------------------------------------------------------------------------------------

def _ib_spec(dim):
    if dim == 2:
        return W.GridSpec(dim=2, n=(24, 20, 1), lo=(-1.0, -0.8, 0.0), hi=(1.0, 0.9, 1.0))
    return W.GridSpec(dim=3, n=(14, 12, 10), lo=(-1.0, -0.7, -0.5), hi=(1.0, 0.8, 0.6))


def _random_markers(spec, n, seed):
    rng = np.random.default_rng(seed)
    X = np.empty((spec.dim, n))
    for a in range(spec.dim):
        h = spec.h[a]
        X[a] = rng.uniform(spec.lo[a] + 2.6 * h, spec.hi[a] - 2.6 * h, n)
    return X


@pytest.mark.parametrize("dim", [2, 3])
def test_interp_spread_adjoint(dim):
    # <I phi, F dS> = - <phi, S[F]>_{h^d}: Eq. 8 and Eq. 9 share delta_h.
    spec = _ib_spec(dim)
    rng = np.random.default_rng(1)
    X = _random_markers(spec, 37, 2)
    phi = rng.standard_normal(spec.shape()[1:])
    F = rng.standard_normal(37)
    dS = rng.uniform(0.5, 1.5, 37) * 0.01
    lhs = np.sum(O.interp_scalar(spec, phi, X) * F * dS)
    f = O.spread_scalar(spec, X, F, dS)
    rhs = -np.sum(phi * f) * np.prod(spec.h)
    assert abs(lhs - rhs) <= 1e-14 * (abs(lhs) + np.sum(np.abs(F * dS)))


@pytest.mark.parametrize("dim", [2, 3])
def test_spread_conserves_force(dim):
    spec = _ib_spec(dim)
    rng = np.random.default_rng(3)
    X = _random_markers(spec, 50, 4)
    F = rng.standard_normal(50)
    dS = rng.uniform(0.5, 1.5, 50) * 0.01
    f = O.spread_scalar(spec, X, F, dS)
    total = np.sum(f) * np.prod(spec.h)
    assert abs(total + np.sum(F * dS)) <= 1e-14 * np.sum(np.abs(F * dS))


@pytest.mark.parametrize("dim", [2, 3])
def test_interp_exact_for_linear_fields(dim):
    spec = _ib_spec(dim)
    X = _random_markers(spec, 30, 5)
    Xg, Yg, Zg = W.mesh(spec)
    coef = [0.7, -1.3, 2.1][:dim]
    phi = 0.4 + coef[0] * Xg[...] + coef[1] * Yg
    if dim == 3:
        phi = phi + coef[2] * Zg
    got = O.interp_scalar(spec, phi, X)
    want = 0.4 + sum(coef[a] * X[a] for a in range(dim))
    assert np.max(np.abs(got - want)) < 1e-14


def test_markers_out_of_bounds_rejected():
    spec = _ib_spec(2)
    X = np.array([[spec.lo[0] + 1.2 * spec.h[0]], [0.0]])
    with pytest.raises(RuntimeError):
        O.interp_scalar(spec, np.zeros(spec.shape()[1:]), X)


# ------------------------------------------------------------------------------------------
# Fifth-order reconstructions (Sec. 2: WENO of Liu et al. / Jiang-Shu, TENO of Fu et al.)
# ------------------------------------------------------------------------------------------

def test_reconstruction_golden_cases():
    for row in _read_golden("reconstruction_cases.txt"):
        scheme, tol = row[0], float(row[1])
        v = [float(x) for x in row[2:7]]
        want = float(row[7])
        fns = {"weno": [O.weno5js], "teno": [O.teno5], "both": [O.weno5js, O.teno5]}[scheme]
        for fn in fns:
            got = fn(v)
            assert abs(got - want) <= tol * max(1.0, abs(want)), (fn, v, got, want)


def test_reconstruction_shift_and_scale_invariance():
    # candidates are affine with weights summing to one and the indicators depend on
    # differences only: R(a v + b) = a R(v) + b for a > 0
    rng = np.random.default_rng(6)
    for _ in range(200):
        v = rng.standard_normal(5)
        for fn in (O.weno5js, O.teno5):
            base = fn(v)
            assert fn(v + 3.0) == pytest.approx(base + 3.0, abs=1e-13)


@pytest.mark.parametrize("fn", [O.weno5js, O.teno5])
def test_reconstruction_fifth_order(fn):
    # (F_{i+1/2} - F_{i-1/2}) / h -> f'(x_i) at fifth order on a smooth monotone function
    errs = []
    Ns = [16, 32, 64, 128]
    for N in Ns:
        h = 1.0 / N
        M = int(round(0.5 / h))
        xs = 0.2 + (np.arange(-3, M + 3) + 0.5) * h
        f = np.exp(xs)
        Fh = np.array([fn(f[m - 2:m + 3]) for m in range(2, M + 3)])
        d = (Fh[1:] - Fh[:-1]) / h
        errs.append(np.max(np.abs(d - np.exp(xs[3:3 + len(d)]))))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 4.7) and np.all(slopes < 5.3), slopes


# ------------------------------------------------------------------------------------------
# Full right-hand side (Eq. 2-5)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim,scheme", [(2, W.WENO5JS), (2, W.TENO5), (3, W.WENO5JS), (3, W.TENO5)])
def test_free_stream_preserved_bitwise(dim, scheme):
    vel = (0.31, -0.17, 0.23)
    n = (9, 7, 1) if dim == 2 else (7, 6, 5)
    spec = W.GridSpec(dim=dim, n=n, lo=(0, 0, 0), hi=(1, 1.2, 0.8), Re=50.0,
                      qinf=W.freestream(dim, 1.4, rho=1.3, vel=vel, p=0.9), scheme=scheme,
                      bc=((2, 2), (0, 1), (1, 0)))
    Q = np.empty(spec.shape())
    for c in range(spec.nv):
        Q[c] = spec.qinf[c]
    L = O.rhs(spec, Q)
    assert np.all(L == 0.0)


def _viscous_target(dim, Re, N):
    """(1/Re) div tau and (1/Re) div(u.tau) of Eq. 2-5 for a smooth periodic velocity field,
    derived symbolically from the continuous definitions (tau = grad u + grad u^T - 2/3 div u I,
    b_j = u_i tau_ij, no heat flux)."""
    sp = pytest.importorskip("sympy")
    xs = sp.symbols("x y z")[:dim]
    two_pi = 2 * sp.pi
    if dim == 2:
        x, y = xs
        u = [sp.Rational(1, 10) * sp.sin(two_pi * x) * sp.cos(two_pi * y),
             sp.Rational(1, 20) * sp.cos(two_pi * x) + sp.Rational(1, 25) * sp.sin(2 * two_pi * y)]
    else:
        x, y, z = xs
        u = [sp.Rational(1, 10) * sp.sin(two_pi * x) * sp.cos(two_pi * z),
             sp.Rational(1, 20) * sp.cos(two_pi * y) * sp.sin(two_pi * x),
             sp.Rational(1, 25) * sp.sin(two_pi * (y + z))]
    div = sum(sp.diff(u[i], xs[i]) for i in range(dim))
    tau = [[sp.diff(u[i], xs[j]) + sp.diff(u[j], xs[i]) - (sp.Rational(2, 3) * div if i == j else 0)
            for j in range(dim)] for i in range(dim)]
    mom = [sum(sp.diff(tau[i][j], xs[j]) for j in range(dim)) / Re for i in range(dim)]
    b = [sum(u[i] * tau[i][j] for i in range(dim)) for j in range(dim)]
    en = sum(sp.diff(b[j], xs[j]) for j in range(dim)) / Re
    fu = [sp.lambdify(xs, e, "numpy") for e in u]
    fm = [sp.lambdify(xs, e, "numpy") for e in mom]
    fe = sp.lambdify(xs, en, "numpy")
    return fu, fm, fe


@pytest.mark.parametrize("dim", [2, 3])
def test_viscous_operator_fourth_order(dim):
    Re = 20.0
    fu, fm, fe = _viscous_target(dim, Re, None)
    Ns = [12, 24, 48] if dim == 3 else [16, 32, 64]
    errs = []
    for N in Ns:
        n = (N, N, N) if dim == 3 else (N, N, 1)
        spec = W.GridSpec(dim=dim, n=n, lo=(0, 0, 0), hi=(1, 1, 1), Re=Re,
                          qinf=W.freestream(dim, 1.4), bc=((2, 2), (2, 2), (2, 2)))
        X, Y, Z = W.mesh(spec)
        pts = (X, Y) if dim == 2 else (X, Y, Z)
        vel = [np.broadcast_to(f(*pts), X.shape).astype(float) for f in fu]
        Q = W.conservative(spec, np.ones(X.shape), vel, np.full(X.shape, 1.0 / 1.4))
        Lv = O.rhs(spec, Q)
        spec0 = W.GridSpec(**{**spec.__dict__, "Re": 0.0})
        L0 = O.rhs(spec0, Q)
        D = Lv - L0
        err = np.max(np.abs(D[0]))
        for i in range(dim):
            err = max(err, np.max(np.abs(D[1 + i] - np.broadcast_to(fm[i](*pts), X.shape))))
        err = max(err, np.max(np.abs(D[dim + 1] - np.broadcast_to(fe(*pts), X.shape))))
        errs.append(err)
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 3.8), (errs, slopes)


def test_entropy_wave_fifth_order():
    # rho = 1 + 0.2 sin(2 pi (x + y)), u = (0.5, 0.3), p = const is an exact solution of the
    # paper's equations (tau = 0 for uniform u and there is no heat flux): it translates.
    u0, v0, T = 0.5, 0.3, 0.2
    errs = []
    for N in (16, 32, 64):
        spec = W.GridSpec(dim=2, n=(N, N, 1), lo=(0, 0, 0), hi=(1, 1, 1), Re=100.0,
                          qinf=W.freestream(2, 1.4, vel=(u0, v0, 0)), scheme=W.TENO5,
                          bc=((2, 2), (2, 2), (0, 0)))
        X, Y, _ = W.mesh(spec)
        rho = 1.0 + 0.2 * np.sin(2 * math.pi * (X + Y))
        Q = W.conservative(spec, rho, [np.full(X.shape, u0), np.full(X.shape, v0)],
                           np.full(X.shape, 1.0))
        h = 1.0 / N
        steps = int(math.ceil(T / (0.4 * h ** (5.0 / 3.0))))
        dt = T / steps
        Qe, _ = O.rk3(spec, Q, dt, steps)
        exact = 1.0 + 0.2 * np.sin(2 * math.pi * (X - u0 * T + Y - v0 * T))
        errs.append(np.max(np.abs(Qe[0] - exact)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 4.4), (errs, slopes)


def test_rk3_amplification_polynomial_via_sponge():
    # A 2x2 grid whose cells all lie on the outer ring has a uniform sponge rate sigma, and a
    # uniform state keeps zero convective and viscous terms, so each cell obeys
    # dq/dt = -sigma (q - q_inf).  One SSP-RK3 step multiplies q - q_inf by the third-order
    # Taylor polynomial R(z) = 1 + z + z^2/2 + z^3/6, z = -sigma dt.
    sigma = 3.0
    spec = W.GridSpec(dim=2, n=(2, 2, 1), lo=(0, 0, 0), hi=(1, 1, 1), Re=10.0,
                      qinf=W.freestream(2, 1.4), sponge_cells=4, sponge_sigma=sigma)
    base = np.array(spec.qinf[:4])
    dq = np.array([0.01, 0.02, -0.015, 0.03])
    Q = np.empty(spec.shape())
    for c in range(4):
        Q[c] = base[c] + dq[c]
    for dt in (0.05, 0.1, 0.2):
        Q1, _ = O.rk3(spec, Q, dt, 1)
        z = -sigma * dt
        R = 1 + z + z * z / 2 + z ** 3 / 6
        for c in range(4):
            assert np.allclose(Q1[c] - base[c], R * dq[c], rtol=1e-12, atol=1e-16)
    # and the error against exp(z) is third order
    errs = []
    for dt in (0.1, 0.05, 0.025):
        Q1, _ = O.rk3(spec, Q, dt, int(round(0.4 / dt)))
        errs.append(abs((Q1[0, 0, 0, 0] - base[0]) - dq[0] * math.exp(-sigma * 0.4)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - 3.0) < 0.25), slopes


def test_probe_exact_for_linear_pressure():
    spec = W.GridSpec(dim=2, n=(20, 18, 1), lo=(-1, -1, 0), hi=(1, 1, 1), qinf=W.freestream(2, 1.4))
    X, Y, _ = W.mesh(spec)
    p = 1.0 / 1.4 + 0.01 * X - 0.02 * Y
    Q = W.conservative(spec, np.ones(X.shape), [np.zeros(X.shape)] * 2, p)
    xp = np.array([[0.1, -0.33, 0.5], [0.2, 0.4, -0.45]])
    got = O.probe(spec, Q, xp)
    assert np.allclose(got, 0.01 * xp[0] - 0.02 * xp[1], atol=1e-15)


def test_penalty_force_law_and_spreading_in_rhs():
    # Eq. 7: F = alpha xi + beta (U_ib - U); the momentum source integrates to -sum F dS and the
    # energy source is f.u.  In a fluid at rest with uniform u = 0 the slip is -U.
    spec = W.GridSpec(dim=2, n=(20, 20, 1), lo=(-1, -1, 0), hi=(1, 1, 1),
                      qinf=W.freestream(2, 1.4), alpha_pen=7.0, beta_pen=3.0)
    Q = np.empty(spec.shape())
    for c in range(4):
        Q[c] = spec.qinf[c]
    X = np.array([[0.05, -0.2], [0.1, 0.3]])
    U = np.array([[0.5, 0.0], [0.0, -0.25]])
    xi = np.array([[0.01, 0.02], [0.03, 0.04]])
    dS = np.array([0.1, 0.2])
    L, F, rate, _ = O.rhs(spec, Q, X, U, dS, xi, return_markers=True)
    assert np.allclose(rate, -U, atol=1e-15)
    assert np.allclose(F, 7.0 * xi + 3.0 * (-U), atol=1e-14)
    h2 = np.prod(spec.h)
    assert np.allclose(L[1].sum() * h2, -(F[0] * dS).sum(), atol=1e-14)
    assert np.allclose(L[2].sum() * h2, -(F[1] * dS).sum(), atol=1e-14)
    assert np.all(L[0] == 0.0)
    assert np.all(L[3] == 0.0)  # u = 0 everywhere: the source does no work


def test_teno5_keeps_all_stencils_when_tau_is_small_against_the_smoothest():
    # premise of the kernels' shortcut: tau5 <= 4 (min beta + eps) implies every gamma_k is in
    # [1, 5^6], chi_k >= 1/(3 5^6) > C_T, so TENO5 returns the optimal linear combination
    rng = np.random.default_rng(9)
    hits = 0
    for _ in range(20000):
        v = np.cumsum(rng.standard_normal(5) * rng.choice([1e-6, 1e-3, 1.0, 10.0]))
        v += rng.standard_normal(5) * rng.choice([0.0, 1e-8, 1e-3])
        a, b, c, d, e = v
        b0 = 13 / 12 * (a - 2 * b + c) ** 2 + 0.25 * (a - 4 * b + 3 * c) ** 2
        b1 = 13 / 12 * (b - 2 * c + d) ** 2 + 0.25 * (b - d) ** 2
        b2 = 13 / 12 * (c - 2 * d + e) ** 2 + 0.25 * (3 * c - 4 * d + e) ** 2
        if abs(b0 - b2) <= 4.0 * (min(b0, b1, b2) + 1e-40):
            hits += 1
            lin = (2 * a - 13 * b + 47 * c + 27 * d - 3 * e) / 60
            assert abs(O.teno5(v) - lin) <= 1e-13 * (np.max(np.abs(v)) + 1e-300)
    assert hits > 1000
