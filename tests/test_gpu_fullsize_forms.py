"""Parity at the full benchmark size for the two further FP32 forms bench.py times on the 512^3
sphere workload (TENO5, 20000 markers, Re 1e4): the characteristic-wise reconstruction on the
pulse, and the learned weights on the stress state (where the network supplies nearly every
reconstruction).

As in the full-size test of the component-wise forms, the oracle evaluates crops around sampled
cells with the split speeds of the full state (the right-hand side of a cell depends only on the
cells within 4 of it, the markers within 2 cells, and the global split speeds):

* characteristic-wise FP32: every sampled value within 256 eps32 of the perturbation-flux scale
  of the oracle's characteristic-wise option (the bound of the component-wise FP32 form);
* learned weights: over the sampled values, the network's increment over TENO5,
  D = L(learned) - L(TENO5), agrees with the oracle's within 2^-4 of its RMS per component (the
  bound of the element-wise learned parity test) plus twice the FP32 rounding of a TENO5
  right-hand side there (RMS of the FP32 TENO5 form against the oracle at the same cells; D
  takes the difference of two FP32 right-hand sides).  At 512^3 the stress state's modes span
  hundreds of cells and the network's increment is only about ten times that rounding, where on
  the small grids of the element-wise test it is a hundred times; the whole right-hand side
  stays within the FP32 bound plus the network term.
"""
import dataclasses
import os

import numpy as np
import pytest

from oracle import mlp_oracle as M
from oracle import oracle as O
from paper_1905_00182_gb300 import workloads as W
from tests.test_gpu_fullsize import N, _samples, _setup

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EPS32 = float(np.finfo(np.float32).eps)


def _crop(spec, Qh, X, U, dS, alpha, c, **kw):
    """oracle right-hand side at cell c from a crop of the full state"""
    h = spec.h[0]
    lo_i = np.maximum(c - 6, 0)
    hi_i = np.minimum(c + 7, N)
    sub = Qh[:, lo_i[2]:hi_i[2], lo_i[1]:hi_i[1], lo_i[0]:hi_i[0]]
    n = tuple(int(x) for x in (hi_i - lo_i))
    cs = dataclasses.replace(spec, n=n, lo=tuple(spec.lo[a] + lo_i[a] * h for a in range(3)),
                             hi=tuple(spec.lo[a] + hi_i[a] * h for a in range(3)),
                             bc=((0, 0), (0, 0), (0, 0)))
    centre = np.array(spec.lo) + (c + 0.5) * h
    near = np.all(np.abs(X - centre[:, None]) < 2.0 * h, axis=0)
    if near.any():
        Lc = O.rhs_given_alpha(cs, np.ascontiguousarray(sub), alpha, X[:, near], U[:, near],
                               dS[near], **kw)
    else:
        Lc = O.rhs_given_alpha(cs, np.ascontiguousarray(sub), alpha, **kw)
    o = c - lo_i
    return Lc[:, o[2], o[1], o[0]]


def _gpu_at(ib, spec, Qd, X, U, dS, cells, net=None):
    g = ib.Grid(spec)
    if net is not None:
        ib.ibfsa_set_mlp(g.h, net.ptr)
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


def test_full_size_charwise_fp32_sampled():
    from paper_1905_00182_gb300 import ibfsa as ib
    ib.lib()
    spec, X, U, dS = _setup()
    Qd = W.gaussian_pulse_state_torch(spec, (2.0, 0.0, 0.0))
    Qh = Qd.cpu().numpy()
    alpha = O.wavespeeds(spec, Qh)
    cells = _samples(spec, X, np.random.default_rng(2025))
    want = np.array([_crop(spec, Qh, X, U, dS, alpha, c, charwise=True) for c in cells])
    got, a_gpu = _gpu_at(ib, dataclasses.replace(spec, precision=W.FP32_PERTURB, charwise=True),
                         Qd, X, U, dS, cells)
    np.testing.assert_allclose(a_gpu, alpha[:3], rtol=4e-6)
    pert_scale = 1.2 * np.array([1e-3, 1e-3, 1e-3, 1e-3, 3e-3]) / spec.h[0]
    err = np.abs(got - want)
    print("charwise FP32 at 512^3: max err / scale", np.max(err / pert_scale, axis=0) / EPS32,
          "eps32")
    assert np.all(err <= 256 * EPS32 * pert_scale), np.max(err / pert_scale)
    # On this smooth state TENO5 keeps every stencil, and the linear weights commute with the
    # projection on the characteristic fields: the two options agree to rounding here.  The
    # test on the stress state's contact below is the one that tells them apart.


def test_full_size_charwise_fp32_at_the_contact():
    """the characteristic-wise FP32 form at 512^3 on the stress state, sampled on both sides of
    its contact (where TENO5 cuts stencils and the option changes the result)"""
    from paper_1905_00182_gb300 import ibfsa as ib
    from tests.test_gpu_fp32 import _perturbation_scale
    ib.lib()
    spec, X, U, dS = _setup()
    Qd = W.stress_state_torch(spec)
    Qh = Qd.cpu().numpy()
    alpha = O.wavespeeds(spec, Qh)
    cells = _contact_samples(spec, np.random.default_rng(2027))
    want = np.array([_crop(spec, Qh, X, U, dS, alpha, c, charwise=True) for c in cells])
    comp = np.array([_crop(spec, Qh, X, U, dS, alpha, c) for c in cells])
    got, _ = _gpu_at(ib, dataclasses.replace(spec, precision=W.FP32_PERTURB, charwise=True),
                     Qd, X, U, dS, cells)
    sc = _perturbation_scale(spec, Qh[:, ::2, ::2, ::2])
    err = np.abs(got - want)
    print("charwise FP32 at the contact: max err / scale", np.max(err / sc, axis=0) / EPS32,
          "eps32; charwise - componentwise", np.max(np.abs(comp - want) / sc, axis=0) / EPS32)
    assert np.all(err <= 256 * EPS32 * sc), np.max(err / sc)
    assert np.max(np.abs(comp - want) / sc) > 1e3 * EPS32


def _contact_samples(spec, rng):
    """cells on both sides of the stress state's contact (mid-x), where TENO5 cuts stencils"""
    cells = []
    for _ in range(30):
        c = rng.integers(6, N - 6, 3)
        c[0] = N // 2 + rng.integers(-4, 4)
        cells.append(c)
    return np.array(cells)


def test_full_size_learned_stress_sampled():
    from paper_1905_00182_gb300 import ibfsa as ib
    ib.lib()
    spec, X, U, dS = _setup()
    spec = dataclasses.replace(spec, precision=W.FP32_PERTURB)
    Qd = W.stress_state_torch(spec)
    Qh = Qd.cpu().numpy()
    alpha = O.wavespeeds(spec, Qh)
    rng = np.random.default_rng(2026)
    cells = np.concatenate([_samples(spec, X, rng), _contact_samples(spec, rng)])
    params = np.load(os.path.join(ROOT, "paper_1905_00182_gb300", "mlp_weights.npz"))["params"]
    net = ib.MLP(params)
    L_ml, _ = _gpu_at(ib, dataclasses.replace(spec, scheme=W.MLP_TENO5), Qd, X, U, dS, cells, net)
    L_te, _ = _gpu_at(ib, spec, Qd, X, U, dS, cells)
    mlp = O.Learned(M.bf16(np.asarray(params, dtype=np.float32).astype(np.float64)),
                    round_act=True, floor=1e-9)
    mspec = dataclasses.replace(spec, scheme=W.MLP_TENO5)
    Lo_ml = np.array([_crop(mspec, Qh, X, U, dS, alpha, c, mlp=mlp) for c in cells])
    Lo_te = np.array([_crop(spec, Qh, X, U, dS, alpha, c) for c in cells])
    # perturbation-flux scale of the stress state (its modes are smooth: every second cell of
    # each direction gives the maximum to well within the bound's slack)
    from tests.test_gpu_fp32 import _perturbation_scale
    pert_scale = _perturbation_scale(spec, Qh[:, ::2, ::2, ::2])
    for c in range(spec.nv):
        D, Do = L_ml[:, c] - L_te[:, c], Lo_ml[:, c] - Lo_te[:, c]
        rms_do = np.sqrt(np.mean(Do ** 2))
        rms_dd = np.sqrt(np.mean((D - Do) ** 2))
        rms_err = np.sqrt(np.mean((L_ml[:, c] - Lo_ml[:, c]) ** 2))
        rms_te = np.sqrt(np.mean((L_te[:, c] - Lo_te[:, c]) ** 2))
        print(f"learned at 512^3, comp {c}: RMS D_oracle {rms_do:.3e}, RMS(D_gpu - D_oracle) "
              f"{rms_dd:.3e} ({rms_dd / rms_do:.4f}); FP32 TENO5 rounding {rms_te:.3e}; "
              f"RMS |L_gpu - L_oracle| {rms_err:.3e}")
        assert rms_te <= 64 * EPS32 * pert_scale[c], c
        assert rms_do > 4.0 * rms_te, c  # the network's increment stands out of the rounding
        assert rms_dd <= 2.0 ** -4 * rms_do + 2.0 * rms_te, (c, rms_dd / rms_do)
        assert rms_err <= 64 * EPS32 * pert_scale[c] + 2.0 ** -4 * rms_do, c
