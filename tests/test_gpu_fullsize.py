"""Parity at the full benchmark size: the 512^3 sphere-pulse workload (TENO5, 20000 markers,
Re 1e4) in the launch configuration bench.py times.

The oracle cannot evaluate 1.3e8 cells in a test, but the right-hand side of a cell depends only
on the cells within 4 of it, on the markers within 2 cells of it, and on the split speeds (a
maximum over the whole domain).  So the test computes the split speeds of the full state with
the oracle, then for sampled cells evaluates the oracle on a crop around each (real boundary
rules where the crop touches the domain boundary, the markers that reach the cell, the global
split speeds) and compares the crop's centre with the GPU value: bit for bit for strict FP64,
within the rounding bounds of the other parity tests for fast FP64 and for the FP32 form.
h = 1/32 is a power of two, so crop coordinates and spacings are exact.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00182_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = float(np.finfo(np.float64).eps)
EPS32 = float(np.finfo(np.float32).eps)
N = 512


def _setup():
    L = 8.0
    spec = W.GridSpec(dim=3, n=(N, N, N), lo=(-L, -L, -L), hi=(L, L, L), gamma=1.4, Re=1e4,
                      qinf=W.freestream(3, 1.4), scheme=W.TENO5, max_markers=20000)
    h = spec.h[0]
    dt = 0.5 / (3.0 / h)
    spec.alpha_pen, spec.beta_pen = W.penalty_defaults(h, dt)
    X, U, dS = W.fibonacci_sphere(20000, 0.5)
    return spec, X, U, dS


def _samples(spec, X, rng):
    h = spec.h[0]
    cells = []
    # bulk cells across the pulse (x near 2) and the quiescent region
    for _ in range(120):
        c = rng.integers(6, N - 6, 3)
        if rng.random() < 0.6:
            c[0] = int((2.0 - spec.lo[0]) / h) + rng.integers(-10, 10)
            c[1] = N // 2 + rng.integers(-10, 10)
            c[2] = N // 2 + rng.integers(-10, 10)
        cells.append(c)
    # cells next to markers (the IB source)
    for k in rng.choice(X.shape[1], 40, replace=False):
        c = np.floor((X[:, k] - np.array(spec.lo)) / h - 0.5).astype(int) + rng.integers(-1, 2, 3)
        cells.append(c)
    # cells at the domain boundary (zero-gradient ghosts)
    for _ in range(24):
        c = rng.integers(0, N, 3)
        a = rng.integers(0, 3)
        c[a] = rng.choice([0, 1, 2, N - 3, N - 2, N - 1])
        cells.append(c)
    return np.array(cells)  # (i, j, k) = (x, y, z)


def _crop_oracle(spec, Qh, X, U, dS, alpha, c):
    """oracle right-hand side at cell c from a crop of the full state"""
    h = spec.h[0]
    lo_i = np.maximum(c - 6, 0)
    hi_i = np.minimum(c + 7, N)
    sub = Qh[:, lo_i[2]:hi_i[2], lo_i[1]:hi_i[1], lo_i[0]:hi_i[0]]
    n = tuple(int(x) for x in (hi_i - lo_i))
    bc = tuple((0, 0) for _ in range(3))  # the workload's walls are zero-gradient too
    cs = dataclasses.replace(spec, n=n, lo=tuple(spec.lo[a] + lo_i[a] * h for a in range(3)),
                             hi=tuple(spec.lo[a] + hi_i[a] * h for a in range(3)), bc=bc)
    # markers within two cells of the centre reach it
    centre = np.array(spec.lo) + (c + 0.5) * h
    near = np.all(np.abs(X - centre[:, None]) < 2.0 * h, axis=0)
    if near.any():
        Lc = O.rhs_given_alpha(cs, np.ascontiguousarray(sub), alpha, X[:, near], U[:, near],
                               dS[near])
    else:
        Lc = O.rhs_given_alpha(cs, np.ascontiguousarray(sub), alpha)
    o = c - lo_i
    return Lc[:, o[2], o[1], o[0]]


def _gpu_rhs_at(ib, spec, Qd, X, U, dS, cells, strict, precision):
    g = ib.Grid(dataclasses.replace(spec, precision=precision), strict=strict)
    g.set_state(Qd)
    g.set_markers(X, U, dS)
    L = g.rhs()
    alpha = np.array(g.max_wavespeed())
    assert g.status() == 0
    idx = torch.from_numpy((cells[:, 2] * N + cells[:, 1]) * N + cells[:, 0]).cuda()
    vals = L.reshape(spec.nv, -1)[:, idx].cpu().numpy().T
    g.close()
    del g, L
    torch.cuda.empty_cache()
    return vals, alpha


def test_full_size_sampled_parity():
    from paper_1905_00182_gb300 import ibfsa as ib
    ib.lib()
    spec, X, U, dS = _setup()
    Qd = W.gaussian_pulse_state_torch(spec, (2.0, 0.0, 0.0))
    Qh = Qd.cpu().numpy()
    alpha = O.wavespeeds(spec, Qh)
    rng = np.random.default_rng(2024)
    cells = _samples(spec, X, rng)
    want = np.array([_crop_oracle(spec, Qh, X, U, dS, alpha, c) for c in cells])

    strict, a_strict = _gpu_rhs_at(ib, spec, Qd, X, U, dS, cells, True, W.FP64)
    np.testing.assert_array_equal(a_strict, alpha[:3])
    np.testing.assert_array_equal(strict, want)

    # per-component split-flux scale of this state (rest state with a 1e-3 pulse)
    p_scale = 1.0 / 1.4 + 1e-3
    flux_scale = np.array([1.2 * 1.0, p_scale + 1.2 * 1e-3, p_scale + 1.2 * 1e-3,
                           p_scale + 1.2 * 1e-3, 1.2 * (1.0 / 0.4 / 1.4 + 1e-2)]) / spec.h[0]
    fast, _ = _gpu_rhs_at(ib, spec, Qd, X, U, dS, cells, False, W.FP64)
    assert np.all(np.abs(fast - want) <= 64 * EPS * flux_scale), np.max(np.abs(fast - want) / flux_scale)

    # FP32 form: the perturbation of this state is at most the pulse (1e-3 in p, 2.5e-3 in E)
    pert_scale = 1.2 * np.array([1e-3, 1e-3, 1e-3, 1e-3, 3e-3]) / spec.h[0]
    f32, _ = _gpu_rhs_at(ib, spec, Qd, X, U, dS, cells, False, W.FP32_PERTURB)
    err = np.abs(f32 - want)
    assert np.all(err <= 256 * EPS32 * pert_scale), np.max(err / pert_scale)
