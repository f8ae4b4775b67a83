"""Seeded parity cases shared by the GPU tests (inputs only; no arithmetic of the method)."""
import math

import numpy as np

from paper_1905_00182_gb300 import workloads as W


def case_2d_weno(n=(37, 29)):
    """2D, WENO5-JS, viscous, zero-gradient walls, pulse + random modes + contact step,
    a cylinder of 24 markers with a non-zero penalty integral.  Ragged sizes."""
    g = 1.4
    spec = W.GridSpec(dim=2, n=(n[0], n[1], 1), lo=(-1.2, -1.0, 0.0), hi=(1.3, 1.1, 1.0), gamma=g,
                      Re=500.0, qinf=W.freestream(2, g), scheme=W.WENO5JS, max_markers=24)
    h = spec.h[0]
    spec.alpha_pen, spec.beta_pen = W.penalty_defaults(h, 0.25 * h)
    Q = W.random_smooth_state(spec, seed=11, amp=2e-3, step=0.05)
    Q = Q + (W.gaussian_pulse_state(spec, (0.6, 0.1)) - W.gaussian_pulse_state(spec, (0.6, 0.1), amp=0.0))
    X, U, dS = W.circle_markers(24, 0.3, center=(-0.1, 0.05), seed=5, omega=0.4)
    xi = 1e-3 * np.stack([np.sin(np.arange(24)), np.cos(np.arange(24))])
    return dict(spec=spec, Q=Q, X=X, U=U, dS=dS, xi=xi, dt=0.25 * h)


def case_2d_teno_stream(n=(40, 33)):
    """2D, TENO5, stream at Mach 0.3, periodic in x, free-stream ghosts in y, sponge."""
    g = 1.4
    spec = W.GridSpec(dim=2, n=(n[0], n[1], 1), lo=(0.0, -1.0, 0.0), hi=(2.0, 1.0, 1.0), gamma=g,
                      Re=200.0, qinf=W.freestream(2, g, vel=(0.3, 0.0, 0.0)), scheme=W.TENO5,
                      bc=((2, 2), (1, 1), (0, 0)), sponge_cells=5, sponge_sigma=3.0,
                      max_markers=16)
    h = spec.h[0]
    spec.alpha_pen, spec.beta_pen = W.penalty_defaults(h, 0.2 * h)
    Q = W.random_smooth_state(spec, seed=12, amp=1e-2, vel0=(0.3, 0.0, 0.0), step=0.1,
                              periodic=True)
    X, U, dS = W.circle_markers(16, 0.25, center=(1.0, 0.0), seed=6)
    xi = np.zeros((2, 16))
    return dict(spec=spec, Q=Q, X=X, U=U, dS=dS, xi=xi, dt=0.2 * h)


def case_3d_teno(n=(21, 18, 17)):
    """3D, TENO5, viscous, zero-gradient walls, pulse + modes, 60 sphere markers."""
    g = 1.4
    spec = W.GridSpec(dim=3, n=n, lo=(-1.0, -0.9, -0.85), hi=(1.1, 0.9, 0.85), gamma=g, Re=300.0,
                      qinf=W.freestream(3, g), scheme=W.TENO5, max_markers=60)
    h = spec.h[0]
    spec.alpha_pen, spec.beta_pen = W.penalty_defaults(h, 0.15 * h)
    Q = W.random_smooth_state(spec, seed=13, amp=2e-3, step=0.05)
    X, U, dS = W.fibonacci_sphere(60, 0.35)
    U = 0.05 * np.stack([np.ones(60), -np.ones(60), np.zeros(60)])
    xi = 1e-3 * np.stack([np.sin(np.arange(60)), np.cos(np.arange(60)), np.sin(2 * np.arange(60))])
    return dict(spec=spec, Q=Q, X=X, U=U, dS=dS, xi=xi, dt=0.15 * h)


def case_3d_weno_periodic(n=(16, 12, 20)):
    """3D, WENO5-JS, inviscid, periodic box, moving stream, no markers, free-stream ghosts off."""
    g = 1.4
    spec = W.GridSpec(dim=3, n=n, lo=(0.0, 0.0, 0.0), hi=(1.0, 0.75, 1.25), gamma=g, Re=0.0,
                      qinf=W.freestream(3, g, vel=(0.2, -0.1, 0.15)), scheme=W.WENO5JS,
                      bc=((2, 2), (2, 2), (2, 2)))
    Q = W.random_smooth_state(spec, seed=14, amp=5e-2, vel0=(0.2, -0.1, 0.15), periodic=True)
    return dict(spec=spec, Q=Q, X=None, U=None, dS=None, xi=None, dt=0.1 * spec.h[0])


def case_3d_teno_x36():
    """3D TENO5 with an x extent that is a multiple of 4 (the FP32 y/z passes then stage their
    tiles with tensor copies): one full and one 4-line tile in x, ragged 15-cell segments in y
    and z."""
    return case_3d_teno(n=(36, 19, 17))


def cylinder_scattering(ppd, t_end=8.0, sample=0.1, precision=W.FP64):
    """Sec. 3.1's pulse scattered by a rigid cylinder (D = 1 at the origin, pulse at (4, 0)) on
    the window [-6, 8] x [-6, 6], from which no boundary reflection reaches the probes (2, 0)
    and (2, 2) before t = 8; D/h = ppd, WENO5-JS, Re 1e4, markers at most h/2 apart (at least
    the 160 of the 256^2 set-up), dt = sample / m with CFL <= 0.5."""
    h = 1.0 / ppd
    nx, ny = int(round(14.0 * ppd)), int(round(12.0 * ppd))
    lo = (-6.0, -0.5 * ny * h, 0.0)
    spec = W.GridSpec(dim=2, n=(nx, ny, 1), lo=lo, hi=(lo[0] + nx * h, 0.5 * ny * h, 1.0),
                      gamma=1.4, Re=1e4, qinf=W.freestream(2, 1.4), scheme=W.WENO5JS,
                      precision=precision)
    m = int(math.ceil(4.0 * sample * ppd))
    dt = sample / m
    markers = max(160, int(math.ceil(2.0 * math.pi * 0.5 / (0.5 * h))))
    spec.max_markers = markers
    spec.alpha_pen, spec.beta_pen = W.penalty_defaults(h, dt)
    X, U, dS = W.circle_markers(markers, 0.5, seed=0)
    return dict(spec=spec, Q=W.gaussian_pulse_state(spec, (4.0, 0.0)), X=X, U=U, dS=dS, dt=dt,
                every=m, samples=int(round(t_end / sample)), sample=sample,
                probes=np.array([[2.0, 2.0], [0.0, 2.0]]))


ALL = {
    "2d_weno": case_2d_weno,
    "2d_teno_stream": case_2d_teno_stream,
    "3d_teno": case_3d_teno,
    "3d_teno_x36": case_3d_teno_x36,
    "3d_weno_periodic": case_3d_weno_periodic,
}
