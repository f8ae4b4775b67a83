"""Seeded synthetic inputs shared by the CUDA path, its tests, the bench and the oracle.

This module holds only problem set-up: grid descriptions, initial fields, Lagrangian marker
and probe point sets, and random perturbations.  It contains none of the method's arithmetic
(no fluxes, reconstructions, delta kernels or time stepping), so that neither side of a parity
test can lean on the other through it.

Set-ups follow arXiv:1905.00182:
  * Sec. 3.1 (acoustic pulse scattered by a cylinder): rho = 1, u = 0,
    p = 1/gamma + eps exp(-ln2 ((x-4)^2 + y^2) / 0.04), eps = 1e-3, cylinder D = 1 at the origin;
  * Sec. 3.3 (rotating cylinder in a stream): Mach 0.2, Re 150, markers move with Omega x X;
  * Sec. 3.6 (sphere scattering): rigid sphere of radius 0.5 at the origin; here an initial
    Gaussian pulse centred at (2, 0, 0) replaces the periodic source.
The sphere surface uses golden-spiral (Fibonacci) points with equal areas instead of the
paper's triangulation; circle markers get a seeded phase offset.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

WENO5JS = 0
TENO5 = 1
MLP_TENO5 = 2

FP64 = 0
FP32_PERTURB = 1

BC_ZERO_GRAD = 0
BC_FREESTREAM = 1
BC_PERIODIC = 2
BC_CHARACTERISTIC = 3


@dataclasses.dataclass
class GridSpec:
    dim: int
    n: tuple                       # interior cells (nx, ny, nz); nz = 1 in 2D
    lo: tuple                      # domain box
    hi: tuple
    gamma: float = 1.4
    Re: float = 0.0                # <= 0: inviscid
    qinf: tuple = (1.0, 0.0, 0.0, 0.0, 0.0)
    scheme: int = WENO5JS
    precision: int = FP64
    bc: tuple = ((0, 0), (0, 0), (0, 0))
    sponge_cells: int = 0
    sponge_sigma: float = 0.0
    alpha_pen: float = 0.0
    beta_pen: float = 0.0
    max_markers: int = 0
    # periodic Gaussian pressure source (Sec. 3.6, Eq. 16): amp exp(-b ln2 |x - xc|^2) cos(omega t)
    src_amp: float = 0.0
    src_b: float = 0.0
    src_omega: float = 0.0
    src_xc: tuple = (0.0, 0.0, 0.0)
    # characteristic-wise reconstruction (FP64 forms) instead of component-wise
    charwise: bool = False

    @property
    def nv(self) -> int:
        return self.dim + 2

    @property
    def h(self) -> tuple:
        return tuple((self.hi[a] - self.lo[a]) / self.n[a] for a in range(self.dim))

    @property
    def cells(self) -> int:
        return int(np.prod(self.n[: self.dim]))

    def shape(self) -> tuple:
        """Interior state shape [nv][nz][ny][nx]."""
        nx, ny, nz = self.n
        return (self.nv, nz, ny, nx)


@dataclasses.dataclass
class PlateSpec:
    """A flexible plate (Eq. 1) in absolute nodal coordinates: n_el equal elements, node j
    carrying [x, y, x_s, y_s]; markers at s_k = (k + 1/2) L / n_markers.  clamped = 1: node 0
    follows the clamp motion of Eq. 17, x0 + (A0/2) cos(2 pi f t) [cos beta, sin beta] with the
    chord direction theta0 + (alpha_m/2) sin(2 pi f t + phi); clamped = 0: a free plate."""
    n_el: int = 40
    n_markers: int = 800
    length: float = 1.0
    rho_s: float = 1.0
    K_S: float = 1.0
    K_B: float = 1.0
    clamped: int = 1
    x0: tuple = (0.0, 0.0)
    theta0: float = 0.0
    A0: float = 0.0
    freq: float = 0.0
    beta: float = 0.0
    alpha_m: float = 0.0
    phi: float = 0.0
    newton_max: int = 30
    newton_tol: float = 1e-10   # on the last increment; Newton's error after it is ~ its square

    @property
    def ndof(self) -> int:
        return 4 * (self.n_el + 1)


def plate_straight(ps: PlateSpec, origin=None, theta=None, omega: Optional[float] = None,
                   vel=(0.0, 0.0)):
    """Straight plate from `origin` (default: the clamp position at t = 0) along angle `theta`
    (default: the clamp's chord direction at t = 0), moving rigidly with translation `vel` and
    rotation rate `omega` about the origin (default for a clamped plate: the clamp's own rate
    at t = 0, so the plate starts in step with its clamp).  Returns e, v [4 (n_el + 1)]."""
    w = 2.0 * math.pi * ps.freq
    if origin is None:
        half = 0.5 * ps.A0
        origin = (ps.x0[0] + half * math.cos(ps.beta), ps.x0[1] + half * math.sin(ps.beta))
    if theta is None:
        theta = ps.theta0 + 0.5 * ps.alpha_m * math.sin(ps.phi)
    if omega is None:
        omega = 0.5 * ps.alpha_m * w * math.cos(ps.phi) if ps.clamped else 0.0
    s = np.arange(ps.n_el + 1) * (ps.length / ps.n_el)
    c, sn = math.cos(theta), math.sin(theta)
    e = np.zeros((ps.n_el + 1, 4))
    e[:, 0] = origin[0] + s * c
    e[:, 1] = origin[1] + s * sn
    e[:, 2] = c
    e[:, 3] = sn
    v = np.zeros((ps.n_el + 1, 4))
    v[:, 0] = vel[0] - omega * s * sn
    v[:, 1] = vel[1] + omega * s * c
    v[:, 2] = -omega * sn
    v[:, 3] = omega * c
    return e.ravel(), v.ravel()


def splitmix64(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the splitmix64 generator (Steele, Lea & Flood 2014)."""
    out = np.empty(count, dtype=np.float64)
    mask = (1 << 64) - 1
    x = seed & mask
    for i in range(count):
        x = (x + 0x9E3779B97F4A7C15) & mask
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        z = z ^ (z >> 31)
        out[i] = (z >> 11) * (1.0 / 9007199254740992.0)
    return out


def freestream(dim: int, gamma: float, rho: float = 1.0, vel=(0.0, 0.0, 0.0), p: Optional[float] = None):
    """Conservative free-stream vector (padded to 5 entries) from rho, velocity and pressure."""
    if p is None:
        p = 1.0 / gamma
    m = [rho * vel[a] for a in range(dim)]
    ke = 0.5 * rho * sum(vel[a] ** 2 for a in range(dim))
    q = [rho] + m + [p / (gamma - 1.0) + ke]
    return tuple(q + [0.0] * (5 - len(q)))


def node_coords(spec: GridSpec):
    """Cell-centred node coordinates x_i = lo + (i + 1/2) h per active direction."""
    return [spec.lo[a] + (np.arange(spec.n[a]) + 0.5) * spec.h[a] for a in range(spec.dim)]


def mesh(spec: GridSpec):
    """Coordinate arrays broadcast to the interior [nz][ny][nx] shape."""
    xs = node_coords(spec)
    if spec.dim == 2:
        Y, X = np.meshgrid(xs[1], xs[0], indexing="ij")
        return X[None], Y[None], None
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return X, Y, Z


def conservative(spec: GridSpec, rho, vel, p) -> np.ndarray:
    """Pack primitive fields into the conservative state [rho, rho u, ..., E]."""
    shape = spec.shape()
    Q = np.empty(shape, dtype=np.float64)
    Q[0] = rho
    ke = np.zeros(shape[1:])
    for a in range(spec.dim):
        Q[1 + a] = rho * vel[a]
        ke = ke + 0.5 * rho * vel[a] * vel[a]
    Q[spec.nv - 1] = p / (spec.gamma - 1.0) + ke
    return Q


def gaussian_pulse_state(spec: GridSpec, center, amp: float = 1e-3, halfwidth: float = 0.2,
                         rho0: float = 1.0, p0: Optional[float] = None, vel0=(0.0, 0.0, 0.0)):
    """Initial pressure pulse p = p0 + amp exp(-ln2 |x - c|^2 / halfwidth^2), uniform rho, u."""
    if p0 is None:
        p0 = 1.0 / spec.gamma
    X, Y, Z = mesh(spec)
    r2 = (X - center[0]) ** 2 + (Y - center[1]) ** 2
    if spec.dim == 3:
        r2 = r2 + (Z - center[2]) ** 2
    p = p0 + amp * np.exp(-math.log(2.0) * r2 / halfwidth ** 2)
    rho = np.full(p.shape, rho0)
    vel = [np.full(p.shape, vel0[a]) for a in range(spec.dim)]
    return conservative(spec, rho, vel, p)


def random_smooth_state(spec: GridSpec, seed: int, amp: float = 1e-3, modes: int = 3,
                        vel0=(0.0, 0.0, 0.0), step: float = 0.0, periodic: bool = False):
    """Background (rho = 1, p = 1/gamma, u = vel0) plus seeded random Fourier modes of
    amplitude `amp` in every primitive, optionally a planar density step of relative size `step`
    at x = mid-domain (a contact discontinuity, to exercise the non-linear weights)."""
    rnd = splitmix64(seed, 8 * modes * (spec.dim + 2))
    X, Y, Z = mesh(spec)
    coords = [X, Y, Z][: spec.dim]
    L = [spec.hi[a] - spec.lo[a] for a in range(spec.dim)]
    fields = []
    it = 0
    for v in range(spec.dim + 2):
        f = np.zeros(X.shape)
        for _ in range(modes):
            ph = 0.0
            arg = np.zeros(X.shape)
            for a in range(spec.dim):
                kmax = 3
                kk = int(rnd[it] * kmax) + 1 if periodic else rnd[it] * kmax + 0.5
                it += 1
                arg = arg + 2.0 * math.pi * kk * (coords[a] - spec.lo[a]) / L[a]
            ph = 2.0 * math.pi * rnd[it]
            it += 1
            f = f + amp * np.sin(arg + ph)
        fields.append(f)
    rho = 1.0 + fields[0]
    if step != 0.0:
        xm = 0.5 * (spec.lo[0] + spec.hi[0])
        rho = rho * np.where(X > xm, 1.0 + step, 1.0)
    vel = [vel0[a] + fields[1 + a] for a in range(spec.dim)]
    p = 1.0 / spec.gamma + fields[spec.dim + 1]
    return conservative(spec, rho, vel, p)


def circle_markers(n: int, radius: float = 0.5, center=(0.0, 0.0), seed: int = 0,
                   omega: float = 0.0):
    """n equally spaced markers on a circle, theta_k = 2 pi (k + phi)/n with a seeded phase phi;
    velocity Omega z x X (zero for a fixed body); arc-length weights dS = 2 pi R / n.
    Returns X [2][n], U [2][n], dS [n]."""
    phi = splitmix64(seed, 1)[0]
    th = 2.0 * math.pi * (np.arange(n) + phi) / n
    X = np.stack([center[0] + radius * np.cos(th), center[1] + radius * np.sin(th)])
    U = np.stack([-omega * (X[1] - center[1]), omega * (X[0] - center[0])])
    dS = np.full(n, 2.0 * math.pi * radius / n)
    return X, U, dS


def fibonacci_sphere(n: int, radius: float = 0.5, center=(0.0, 0.0, 0.0)):
    """n golden-spiral points on a sphere with equal area weights 4 pi R^2 / n.
    Returns X [3][n], U [3][n] (zero), dS [n]."""
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ga = math.pi * (3.0 - math.sqrt(5.0))
    th = ga * k
    X = np.stack([center[0] + radius * r * np.cos(th), center[1] + radius * r * np.sin(th),
                  center[2] + radius * z])
    U = np.zeros_like(X)
    dS = np.full(n, 4.0 * math.pi * radius * radius / n)
    return X, U, dS


def ring_probes(n: int, radius: float, center=(0.0, 0.0)):
    th = 2.0 * math.pi * np.arange(n) / n
    return np.stack([center[0] + radius * np.cos(th), center[1] + radius * np.sin(th)])


def doppler_ring_probes(n: int, radius: float, mach: float, center=(0.0, 0.0)):
    """Probes at r = radius (1 - M cos theta), theta = 2 pi k / n: the ring of Sec. 3.3, drawn
    in by the convective Doppler factor downstream (theta = 0) of a stream along +x."""
    th = 2.0 * math.pi * np.arange(n) / n
    r = radius * (1.0 - mach * np.cos(th))
    return np.stack([center[0] + r * np.cos(th), center[1] + r * np.sin(th)])


def penalty_defaults(h: float, dt: float, kappa: float = 0.5, rho: float = 1.0):
    """Penalty constants of Eq. 7 (the paper gives none): a dense marker sheet feeds back a slip
    fraction of about dt * beta * (3/8) / (rho h) per stage, so beta = kappa rho h / ((3/8) dt)
    removes a fraction kappa of the slip per stage; alpha = k beta^2 / 4 with k = 3/(8 rho h)
    makes the spring-dashpot slip dynamics critically damped."""
    beta = kappa * rho * h / (0.375 * dt)
    k = 0.375 / (rho * h)
    alpha = k * beta * beta / 4.0
    return alpha, beta


# --------------------------------------------------------------------------------------------
# The five workloads (synthetic, seeded).
# --------------------------------------------------------------------------------------------

def cylinder_pulse_2d(n: int = 256, markers: int = 160, Re: float = 1e4, scheme: int = WENO5JS,
                      precision: int = FP64):
    """Acoustic pulse scattered by a rigid cylinder (Sec. 3.1): [-10,10]^2, D = 1, pulse at (4,0)
    with amplitude 1e-3 and half-width 0.2, gamma 1.4, zero-gradient boundaries."""
    g = 1.4
    spec = GridSpec(dim=2, n=(n, n, 1), lo=(-10.0, -10.0, 0.0), hi=(10.0, 10.0, 1.0), gamma=g,
                    Re=Re, qinf=freestream(2, g), scheme=scheme, precision=precision,
                    max_markers=markers)
    h = spec.h[0]
    dt = 0.5 / (2.0 / h)  # CFL 0.5 with alpha_x = alpha_y = c = 1 at rest (fixed from the start)
    spec.alpha_pen, spec.beta_pen = penalty_defaults(h, dt)
    Q = gaussian_pulse_state(spec, (4.0, 0.0))
    X, U, dS = circle_markers(markers, 0.5, seed=0)
    probes = np.array([[2.0, 2.0], [0.0, 2.0]])
    return dict(spec=spec, Q=Q, X=X, U=U, dS=dS, dt=dt, steps=100, probes=probes)


def rotating_cylinder_2d(n: int = 2048, markers: int = 1024, scheme: int = WENO5JS,
                         precision: int = FP64):
    """Rotating cylinder in a uniform stream (Sec. 3.3): Mach 0.2, Re = rho U D / mu = 150,
    [-40,40]^2, 20-cell sponge, surface speed 0.5 U, 360 probes on a ring r = 30.  Units:
    rho = 1, c = 1, D = 1, so the solver's Reynolds number (rho c D / mu) is 150 / 0.2."""
    g = 1.4
    U0 = 0.2
    spec = GridSpec(dim=2, n=(n, n, 1), lo=(-40.0, -40.0, 0.0), hi=(40.0, 40.0, 1.0), gamma=g,
                    Re=150.0 / U0, qinf=freestream(2, g, vel=(U0, 0.0, 0.0)), scheme=scheme,
                    precision=precision, bc=((1, 1), (1, 1), (0, 0)), sponge_cells=20,
                    max_markers=markers)
    h = spec.h[0]
    dt = 0.5 / ((1.0 + U0) / h + 1.0 / h)
    spec.alpha_pen, spec.beta_pen = penalty_defaults(h, dt)
    spec.sponge_sigma = 0.5 * (1.0 + U0) / h
    Q = random_smooth_state(spec, seed=3, amp=0.0, modes=1, vel0=(U0, 0.0, 0.0))
    omega = 0.5 * U0 / 0.5
    X, U, dS = circle_markers(markers, 0.5, seed=0, omega=omega)
    probes = ring_probes(360, 30.0)
    return dict(spec=spec, Q=Q, X=X, U=U, dS=dS, dt=dt, steps=20000, probes=probes)


def stationary_cylinder_2d(n: int = 1024, L: float = 20.0, scheme: int = TENO5,
                           precision: int = FP32_PERTURB):
    """Flow past a stationary cylinder (Sec. 3.2): Re = rho U0 D / mu = 150, M = U0 / c = 0.2,
    D = 1 at the origin, uniform grid on [-L, L]^2 (D/h = n / 2L), free-stream ghosts and a
    20-cell sponge, markers every quarter cell.  The paper starts the asymmetric vortex street
    with an initial velocity perturbation in the near wake: here a transverse velocity bump of
    0.1 U0 exp(-((x - 1.5)^2 + y^2) / 0.5)."""
    g = 1.4
    U0 = 0.2
    h = 2.0 * L / n
    markers = 4 * int(math.pi / h)
    spec = GridSpec(dim=2, n=(n, n, 1), lo=(-L, -L, 0.0), hi=(L, L, 1.0), gamma=g,
                    Re=150.0 / U0, qinf=freestream(2, g, vel=(U0, 0.0, 0.0)), scheme=scheme,
                    precision=precision, bc=((1, 1), (1, 1), (0, 0)), sponge_cells=20,
                    max_markers=markers)
    dt = 0.5 / ((1.0 + U0) / h + 1.0 / h)
    spec.alpha_pen, spec.beta_pen = penalty_defaults(h, dt)
    spec.sponge_sigma = 0.5 * (1.0 + U0) / h
    X, Y, _ = mesh(spec)
    v = 0.1 * U0 * np.exp(-((X - 1.5) ** 2 + Y ** 2) / 0.5)
    Q = conservative(spec, np.ones_like(X), [np.full(X.shape, U0), v], np.full(X.shape, 1.0 / g))
    Xm, Um, dS = circle_markers(markers, 0.5, seed=0)
    return dict(spec=spec, Q=Q, X=Xm, U=Um, dS=dS, dt=dt, U0=U0)


def _sphere_setup(n, markers, Re, scheme, precision, probes, L):
    g = 1.4
    spec = GridSpec(dim=3, n=(n, n, n), lo=(-L, -L, -L), hi=(L, L, L), gamma=g, Re=Re,
                    qinf=freestream(3, g), scheme=scheme, precision=precision,
                    max_markers=markers)
    h = spec.h[0]
    dt = 0.5 / (3.0 / h)
    spec.alpha_pen, spec.beta_pen = penalty_defaults(h, dt)
    X, U, dS = fibonacci_sphere(markers, 0.5)
    pr, _, _ = fibonacci_sphere(probes, 6.0 * L / 8.0)
    return spec, dt, X, U, dS, pr


def sphere_pulse_3d(n: int = 512, markers: int = 20000, Re: float = 1e4, scheme: int = TENO5,
                    precision: int = FP64, probes: int = 1000, L: float = 8.0, state: bool = True):
    """Acoustic pulse scattered by a rigid sphere (Sec. 3.6 analogue): [-L,L]^3 (h = 2L/n), sphere
    D = 1 at the origin with Fibonacci markers, Gaussian pulse (1e-3, half-width 0.2) at (2,0,0),
    TENO5, zero-gradient boundaries, probes on a Fibonacci sphere r = 6 (scaled with L).
    state=False skips building the host state (Q = None)."""
    spec, dt, X, U, dS, pr = _sphere_setup(n, markers, Re, scheme, precision, probes, L)
    Q = gaussian_pulse_state(spec, (2.0, 0.0, 0.0)) if state else None
    return dict(spec=spec, Q=Q, X=X, U=U, dS=dS, dt=dt, steps=2000, probes=pr)


def flapping_plate_2d(n=(4096, 2048), n_el: int = 40, markers: int = 800,
                      scheme: int = TENO5, precision: int = FP32_PERTURB):
    """Flexible plate flapping in a uniform stream (Sec. 4.1 set-up, Eq. 17-18): chord L = 1,
    40 elements, thickness ratio 0.01, mass ratio m* = rho_s/(rho_f L) = 1, bending stiffness
    K_B/(rho_f U^2 L^3) = 0.5, clamped leading edge heaving with amplitude A0/2 = 0.5 across the
    stream (beta = 90 deg) and pitching with amplitude alpha_m/2 = 30 deg, Mach number
    M = pi U/(2c) = 0.1 with U = 2 f A0, free stream U0 = 0.4 U (U_r of Sec. 4.1),
    Re = rho_f U L / mu = 200; uniform grid on [-20,20]x[-10,10] with free-stream ghosts and a
    20-cell sponge; 800 markers; 360 probes on a ring r = 8 around the mean clamp position.
    Units: rho_f = 1, c = 1, L = 1 (the solver's Re is then rho_f c L / mu)."""
    g = 1.4
    M = 0.1
    U = 2.0 * M / math.pi            # M = pi U / (2 c)
    A0 = 1.0
    f = U / (2.0 * A0)               # U = 2 f A0
    U0 = 0.4 * U
    Re_flow = 200.0
    K_B = 0.5 * U * U                # K_B / (rho_f U^2 L^3) = 0.5
    K_S = 12.0 * K_B / (0.01 ** 2)   # plate of thickness ratio 0.01: E A / E I = 12 / t^2
    spec = GridSpec(dim=2, n=(n[0], n[1], 1), lo=(-20.0, -10.0, 0.0), hi=(20.0, 10.0, 1.0),
                    gamma=g, Re=Re_flow / U, qinf=freestream(2, g, vel=(U0, 0.0, 0.0)),
                    scheme=scheme, precision=precision, bc=((1, 1), (1, 1), (0, 0)),
                    sponge_cells=20, max_markers=markers)
    h = min(spec.h[0], spec.h[1])
    dt = 0.5 / ((1.0 + U0) / spec.h[0] + 1.0 / spec.h[1])
    spec.alpha_pen, spec.beta_pen = penalty_defaults(h, dt)
    spec.sponge_sigma = 0.5 * (1.0 + U0) / h
    ps = PlateSpec(n_el=n_el, n_markers=markers, length=1.0, rho_s=1.0, K_S=K_S, K_B=K_B,
                   clamped=1, x0=(-0.5, 0.0), theta0=0.0, A0=A0, freq=f,
                   beta=0.5 * math.pi, alpha_m=math.radians(60.0), phi=0.0)
    e, v = plate_straight(ps)
    Q = random_smooth_state(spec, seed=3, amp=0.0, modes=1, vel0=(U0, 0.0, 0.0))
    probes = ring_probes(360, 8.0, center=(-0.5, 0.0))
    return dict(spec=spec, plate=ps, Q=Q, e=e, v=v, dt=dt, probes=probes, U_ref=U)


def sphere_source_3d(n: int = 512, markers: int = 20000, Re: float = 1e4, scheme: int = TENO5,
                     precision: int = FP64, probes: int = 1000, L: float = 8.0):
    """Sound of a periodic Gaussian source scattered by a rigid sphere (Sec. 3.6): the sphere
    workload at rest with the source of Eq. 16 instead of the initial pulse.  The paper's values
    in units of the radius R = 0.5 and of R/c: A = 0.01, B = 16, omega = 2 pi, centre (2R, 0, 0)
    -- here amp = -0.01, b = 16 / R^2, omega = 2 pi / R, xc = (1, 0, 0)."""
    spec, dt, X, U, dS, pr = _sphere_setup(n, markers, Re, scheme, precision, probes, L)
    R = 0.5
    spec.src_amp, spec.src_b, spec.src_omega = -0.01, 16.0 / (R * R), 2.0 * math.pi / R
    spec.src_xc = (2.0 * R, 0.0, 0.0)
    # the fluid starts at rest (rho = 1, u = 0, p = 1/gamma): rest_state(spec)
    return dict(spec=spec, Q=None, X=X, U=U, dS=dS, dt=dt, steps=2000, probes=pr)


def stretched_axis(n: int, h0: float, h1: float, n_inner: int, n_trans: int,
                   center: float = 0.0):
    """One direction of the paper's non-uniform mesh (Sec. 2; Sec. 3.2): spacing h0 over the
    n_inner central cells, a sinusoidal transition to h1 over n_trans cells on each side,
    h1 beyond.  Mapping x(xi) of a computational coordinate xi with unit spacing per cell,
    dx/dxi = h0 + (h1 - h0)(1 - cos(pi s))/2 on the transition (s from 0 to 1).
    Returns (lo, hi, nodes, metric): the box and the node coordinates and dx/dxi at the nodes
    i = -4 .. n+3 (n + 8 entries, node i at index i + 4)."""
    a, t = 0.5 * n_inner, float(n_trans)

    def X(z):  # x - center at distance z >= 0 from the middle, in cells
        if z <= a:
            return h0 * z
        if z <= a + t:
            d = z - a
            return h0 * a + h0 * d + 0.5 * (h1 - h0) * (d - t / math.pi * math.sin(math.pi * d / t))
        return h0 * a + h0 * t + 0.5 * (h1 - h0) * t + h1 * (z - a - t)

    def H(z):
        if z <= a:
            return h0
        if z <= a + t:
            return h0 + 0.5 * (h1 - h0) * (1.0 - math.cos(math.pi * (z - a) / t))
        return h1

    xi = np.arange(-4, n + 4) + 0.5 - 0.5 * n
    nodes = np.array([center + math.copysign(X(abs(z)), z) for z in xi])
    metric = np.array([H(abs(z)) for z in xi])
    return center - X(0.5 * n), center + X(0.5 * n), nodes, metric


def rest_state(spec: GridSpec) -> np.ndarray:
    """Uniform free-stream state of the grid (host)."""
    Q = np.empty(spec.shape())
    for c in range(spec.nv):
        Q[c] = spec.qinf[c]
    return Q


def gaussian_pulse_state_torch(spec: GridSpec, center, amp: float = 1e-3, halfwidth: float = 0.2,
                               device="cuda", rho0: float = 1.0, p0: Optional[float] = None):
    """gaussian_pulse_state generated directly in device memory (same field, fluid at rest),
    for grids too large to build on the host first."""
    import torch
    if p0 is None:
        p0 = 1.0 / spec.gamma
    f64 = torch.float64
    xs = [spec.lo[a] + (torch.arange(spec.n[a], dtype=f64, device=device) + 0.5) * spec.h[a]
          for a in range(spec.dim)]
    Q = torch.zeros(spec.shape(), dtype=f64, device=device)
    Q[0] = rho0
    if spec.dim == 2:
        r2 = (xs[0][None, :] - center[0]) ** 2 + (xs[1][:, None] - center[1]) ** 2
        p = p0 + amp * torch.exp(-math.log(2.0) * r2 / halfwidth ** 2)
        Q[spec.nv - 1, 0] = p / (spec.gamma - 1.0)
        return Q
    for k in range(spec.n[2]):  # plane by plane keeps the temporaries small
        r2 = ((xs[0][None, :] - center[0]) ** 2 + (xs[1][:, None] - center[1]) ** 2
              + (xs[2][k] - center[2]) ** 2)
        p = p0 + amp * torch.exp(-math.log(2.0) * r2 / halfwidth ** 2)
        Q[spec.nv - 1, k] = p / (spec.gamma - 1.0)
    return Q


MLP_SIZES = [(32, 5), (32,), (32, 32), (32,), (32, 32), (32,), (3, 32), (3,)]
MLP_NPARAM = sum(int(np.prod(s)) for s in MLP_SIZES)


def mlp_init_params(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters of the learned-weight network, one flat float32 vector
    [W1 (32x5), b1, W2, b2, W3, b3, W4 (3x32), b4]: scaled normal weights, zero biases except
    b4 = log(0.1, 0.6, 0.3), so the untrained network starts near the linear weights."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in MLP_SIZES:
        if len(s) == 2:
            parts.append(rng.standard_normal(s) * math.sqrt(1.0 / s[1]))
        else:
            parts.append(np.zeros(s))
    parts[6] = parts[6] * 0.1
    parts[7] = np.log(np.array([0.1, 0.6, 0.3]))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def stress_state_torch(spec: GridSpec, seed: int = 1, amp: float = 1e-3, step: float = 0.1,
                       device="cuda"):
    """The rest state plus seeded smooth random modes of amplitude `amp` in every primitive and a
    planar density step of relative size `step` at mid-x (a contact discontinuity), generated in
    device memory: every cell carries a perturbation, so the non-linear weights (and the learned
    form's network) are exercised everywhere instead of only around a pulse."""
    import torch
    f64 = torch.float64
    rnd = splitmix64(seed, 8 * (spec.dim + 2) * 2)
    xs = [(torch.arange(spec.n[a], dtype=f64, device=device) + 0.5) / spec.n[a]
          for a in range(spec.dim)]
    Q = torch.zeros(spec.shape(), dtype=f64, device=device)
    it = 0
    prim = []
    for v in range(spec.dim + 2):
        kk = [int(rnd[it + a] * 3) + 1 for a in range(spec.dim)]
        ph = 2.0 * math.pi * rnd[it + spec.dim]
        it += spec.dim + 1
        prim.append((kk, ph))
    for k in range(spec.n[2]):
        def field(kk, ph):
            arg = 2.0 * math.pi * (kk[0] * xs[0][None, :] + kk[1] * xs[1][:, None])
            if spec.dim == 3:
                arg = arg + 2.0 * math.pi * kk[2] * xs[2][k]
            return amp * torch.sin(arg + ph)
        rho = 1.0 + field(*prim[0])
        rho = rho * torch.where(xs[0][None, :] > 0.5, 1.0 + step, 1.0)
        vel = [field(*prim[1 + a]) for a in range(spec.dim)]
        p = 1.0 / spec.gamma + field(*prim[spec.dim + 1])
        Q[0, k] = rho
        ke = torch.zeros_like(rho)
        for a in range(spec.dim):
            Q[1 + a, k] = rho * vel[a]
            ke = ke + 0.5 * rho * vel[a] * vel[a]
        Q[spec.nv - 1, k] = p / (spec.gamma - 1.0) + ke
    return Q
