"""GPU parity on the non-uniform (stretched) mesh of Sec. 2 -- a uniform box around the body,
a sinusoidal transition (Sec. 3.2) to a coarser spacing outside -- set through ibfsa_set_mesh,
against the oracle's stretched grid (node coordinates and dx/dxi per direction; differences
in xi divided by dx/dxi at the node; markers and probes in the uniform box, their delta taken
with its spacing).

* strict FP64: bit for bit (right-hand side, marker forces, three SSP-RK3 steps with xi, probes;
  2D and 3D, both schemes, viscous, sponge, pressure source, a uniform direction beside
  stretched ones, the characteristic-wise option);
* fast FP64: within 64 eps of the split-flux scale over the smallest spacing (the bound of the
  uniform-grid parity tests);
* FP32 perturbation form: RMS within 64 eps32 of the perturbation-flux scale, 99.9 % quantile
  within 256 eps32 (the FP32 bounds of the uniform grid);
* a uniform mapping given explicitly gives what the uniform grid gives, bit for bit;
* a free stream gives exactly zero; a marker whose support reaches the transition is reported.
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00182_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = float(np.finfo(np.float64).eps)
EPS32 = float(np.finfo(np.float32).eps)
G = 1.4


def _ib():
    from paper_1905_00182_gb300 import ibfsa
    ibfsa.lib()
    return ibfsa


def case_2d(scheme=W.TENO5):
    """2D, both directions stretched (h0 = 0.04 in the box, 0.1 / 0.09 outside), viscous,
    zero-gradient and free-stream walls, 4-cell sponge, pressure source, contact step, a
    cylinder of 20 markers in the uniform box.  Ragged sizes."""
    ax = [W.stretched_axis(45, 0.04, 0.10, 21, 8, center=0.0),
          W.stretched_axis(38, 0.04, 0.09, 21, 6, center=0.05)]
    spec = W.GridSpec(dim=2, n=(45, 38, 1), lo=(ax[0][0], ax[1][0], 0.0),
                      hi=(ax[0][1], ax[1][1], 1.0), gamma=G, Re=300.0, qinf=W.freestream(2, G),
                      scheme=scheme, bc=((0, 1), (1, 0), (0, 0)), sponge_cells=4,
                      sponge_sigma=2.0, max_markers=20)
    spec.src_amp, spec.src_b, spec.src_omega, spec.src_xc = 1e-3, 30.0, 4.0, (0.1, 0.0, 0.0)
    h0 = 0.04
    spec.alpha_pen, spec.beta_pen = W.penalty_defaults(h0, 0.2 * h0)
    Q = W.random_smooth_state(spec, seed=21, amp=2e-3, step=0.05)
    X, U, dS = W.circle_markers(20, 0.2, center=(0.02, 0.04), seed=3, omega=0.3)
    xi = 1e-3 * np.stack([np.sin(np.arange(20)), np.cos(np.arange(20))])
    return dict(spec=spec, Q=Q, X=X, U=U, dS=dS, xi=xi, dt=0.2 * h0,
                mesh=[(ax[0][2], ax[0][3]), (ax[1][2], ax[1][3])], t=0.3)


def case_3d(scheme=W.WENO5JS):
    """3D, x and z stretched, y uniform (h = 0.05), viscous, zero-gradient walls, a sphere of
    40 markers in the uniform box."""
    ax = [W.stretched_axis(30, 0.05, 0.11, 16, 5, center=0.0), None,
          W.stretched_axis(22, 0.05, 0.08, 16, 2, center=-0.02)]
    spec = W.GridSpec(dim=3, n=(30, 26, 22), lo=(ax[0][0], -0.65, ax[2][0]),
                      hi=(ax[0][1], 0.65, ax[2][1]), gamma=G, Re=250.0,
                      qinf=W.freestream(3, G, vel=(0.1, 0.0, -0.05)), scheme=scheme,
                      max_markers=40)
    h0 = 0.05
    spec.alpha_pen, spec.beta_pen = W.penalty_defaults(h0, 0.15 * h0)
    Q = W.random_smooth_state(spec, seed=22, amp=2e-3, vel0=(0.1, 0.0, -0.05), step=0.05)
    X, U, dS = W.fibonacci_sphere(40, 0.17, center=(0.0, 0.02, -0.01))
    xi = 1e-3 * np.stack([np.sin(np.arange(40)), np.cos(np.arange(40)), np.sin(2 * np.arange(40))])
    return dict(spec=spec, Q=Q, X=X, U=U, dS=dS, xi=xi, dt=0.15 * h0,
                mesh=[(ax[0][2], ax[0][3]), None, (ax[2][2], ax[2][3])], t=0.0)


CASES = {"2d_teno": lambda: case_2d(W.TENO5), "2d_weno": lambda: case_2d(W.WENO5JS),
         "3d_weno": lambda: case_3d(W.WENO5JS), "3d_teno": lambda: case_3d(W.TENO5)}


def _grid(case, strict, precision=W.FP64, charwise=False, probes=0, markers=True):
    ib = _ib()
    spec = dataclasses.replace(case["spec"], precision=precision, charwise=charwise)
    g = ib.Grid(spec, strict=strict, max_probes=probes)
    for a, m in enumerate(case["mesh"]):
        if m is not None:
            g.set_mesh(a, *m)
    g.set_state(case["Q"])
    g.set_time(case["t"])
    if markers and case["X"] is not None:
        g.set_markers(case["X"], case["U"], case["dS"])
        xi = torch.from_numpy(np.ascontiguousarray(case["xi"])).cuda()
        ib.ibfsa_set_penalty_integral(g.h, xi.data_ptr())
        torch.cuda.synchronize()
    return g


def _oracle_rhs(case, charwise=False, markers=True):
    m = markers and case["X"] is not None
    return O.rhs(case["spec"], case["Q"], case["X"] if m else None, case["U"] if m else None,
                 case["dS"] if m else None, case["xi"] if m else None, return_markers=True,
                 t=case["t"], charwise=charwise, stretch=case["mesh"])


def _min_spacing(case):
    spec = case["spec"]
    return min(float(np.min(m[1])) if m is not None else spec.h[a]
               for a, m in enumerate(case["mesh"][:spec.dim]))


def _flux_scale(case, perturbation=False):
    """max over cells and directions of |F_d| + alpha |q| per component over the smallest
    spacing: of the full fluxes, or (perturbation) of F' and q' = Q - q_inf"""
    spec, Q = case["spec"], case["Q"]
    nv, dim = spec.nv, spec.dim
    u = [Q[1 + a] / Q[0] for a in range(dim)]
    p = (G - 1.0) * (Q[nv - 1] - 0.5 * sum(Q[1 + a] * u[a] for a in range(dim)))
    alpha = max(np.max(np.abs(u[a]) + np.sqrt(G * p / Q[0])) for a in range(dim))
    qinf = np.array(spec.qinf[:nv])
    uinf = [qinf[1 + a] / qinf[0] for a in range(dim)]
    pinf = (G - 1.0) * (qinf[nv - 1] - 0.5 * sum(qinf[1 + a] * uinf[a] for a in range(dim)))
    sc = np.zeros(nv)
    for c in range(nv):
        m = 0.0
        for a in range(dim):
            def F(Qc, ua, pp):
                if c == 0:
                    return Qc[1 + a]
                if c == nv - 1:
                    return (Qc[nv - 1] + pp) * ua
                return Qc[c] * ua + (pp if c - 1 == a else 0.0)
            if perturbation:
                Fv = F(Q, u[a], p) - F(qinf, uinf[a], pinf)
                qv = Q[c] - qinf[c]
            else:
                Fv, qv = F(Q, u[a], p), Q[c]
            m = max(m, np.max(np.abs(Fv) + alpha * np.abs(qv)))
        sc[c] = m / _min_spacing(case)
    return sc


@pytest.mark.parametrize("name", list(CASES))
def test_stretched_rhs_strict_bitwise(name):
    case = CASES[name]()
    g = _grid(case, strict=True)
    L = g.rhs().cpu().numpy()
    F = g.marker_forces().cpu().numpy()
    assert g.status() == 0
    Lo, Fo, _, _ = _oracle_rhs(case)
    np.testing.assert_array_equal(L, Lo)
    np.testing.assert_array_equal(F, Fo)


def test_stretched_rhs_strict_bitwise_charwise():
    case = case_2d(W.TENO5)
    g = _grid(case, strict=True, charwise=True)
    L = g.rhs().cpu().numpy()
    assert g.status() == 0
    Lo, _, _, _ = _oracle_rhs(case, charwise=True)
    np.testing.assert_array_equal(L, Lo)


@pytest.mark.parametrize("name", list(CASES))
def test_stretched_rhs_fast_within_roundings(name):
    case = CASES[name]()
    g = _grid(case, strict=False)
    L = g.rhs().cpu().numpy()
    assert g.status() == 0
    Lo, Fo, _, _ = _oracle_rhs(case)
    sc = _flux_scale(case)
    for c in range(case["spec"].nv):
        err = np.max(np.abs(L[c] - Lo[c]))
        assert err <= 64 * EPS * sc[c], (c, err, sc[c])
    F = g.marker_forces().cpu().numpy()
    assert np.max(np.abs(F - Fo)) <= 1e-12 * np.max(np.abs(Fo))


@pytest.mark.parametrize("name", list(CASES))
def test_stretched_rhs_fp32_within_fp32_roundings(name):
    case = CASES[name]()
    g = _grid(case, strict=False, precision=W.FP32_PERTURB)
    L = g.rhs().cpu().numpy()
    assert g.status() == 0
    Lo, _, _, _ = _oracle_rhs(case)
    sc = _flux_scale(case, perturbation=True)
    for c in range(case["spec"].nv):
        err = np.abs(L[c] - Lo[c])
        rms = float(np.sqrt(np.mean(err ** 2)))
        assert rms <= 64 * EPS32 * sc[c], (c, rms, sc[c])
        assert np.quantile(err, 0.999) <= 256 * EPS32 * sc[c], c


@pytest.mark.parametrize("name", ["2d_teno", "3d_weno"])
def test_stretched_rk3_strict_bitwise(name):
    case = CASES[name]()
    steps = 3
    g = _grid(case, strict=True)
    g.rk3_step(case["dt"], steps)
    Q = g.get_state().cpu().numpy()
    xi = g.penalty_integral().cpu().numpy()
    assert g.status() == 0
    Qo, xio = O.rk3(case["spec"], case["Q"], case["dt"], steps, case["X"], case["U"],
                    case["dS"], case["xi"], t=case["t"], stretch=case["mesh"])
    np.testing.assert_array_equal(Q, Qo)
    np.testing.assert_array_equal(xi, xio)


def test_stretched_fp32_steps_track_the_oracle():
    case = case_2d(W.TENO5)
    steps = 10
    g = _grid(case, strict=False, precision=W.FP32_PERTURB)
    g.rk3_step(case["dt"], steps)
    Q = g.get_state().cpu().numpy()
    assert g.status() == 0
    Qo, _ = O.rk3(case["spec"], case["Q"], case["dt"], steps, case["X"], case["U"], case["dS"],
                  case["xi"], t=case["t"], stretch=case["mesh"])
    qinf = np.array(case["spec"].qinf[:4])
    for c in range(4):
        pert = np.linalg.norm(Qo[c] - qinf[c])
        assert np.linalg.norm(Q[c] - Qo[c]) <= 1e-4 * pert, c


def test_stretched_probes_strict_bitwise():
    case = case_2d(W.TENO5)
    xp = np.array([[0.0, 0.15, -0.3, 0.3], [0.05, -0.2, 0.1, 0.3]])
    g = _grid(case, strict=True, probes=xp.shape[1])
    got = g.probe(xp).cpu().numpy()
    assert g.status() == 0
    np.testing.assert_array_equal(got, O.probe(case["spec"], case["Q"], xp, stretch=case["mesh"]))


@pytest.mark.parametrize("strict,precision", [(True, W.FP64), (False, W.FP64),
                                              (False, W.FP32_PERTURB)])
def test_marker_reaching_the_transition_is_reported(strict, precision):
    case = case_2d(W.TENO5)
    g = _grid(case, strict=strict, precision=precision)
    X = case["X"].copy()
    X[0, 0] = 0.5  # the box ends at 0.42: the support reaches the transition
    g.set_markers(X, case["U"], case["dS"])
    g.rhs()
    assert g.status() & 1


@pytest.mark.parametrize("strict,precision", [(True, W.FP64), (False, W.FP64),
                                              (False, W.FP32_PERTURB)])
def test_stretched_free_stream_gives_zero(strict, precision):
    case = case_3d(W.TENO5)
    spec = case["spec"]
    case["Q"] = W.rest_state(spec)
    g = _grid(case, strict=strict, precision=precision, markers=False)
    assert torch.all(g.rhs() == 0.0)


def test_explicit_uniform_mesh_is_the_uniform_grid():
    spec = W.GridSpec(dim=2, n=(23, 19, 1), lo=(-1.0, -0.7, 0.0), hi=(1.3, 1.1, 1.0), gamma=G,
                      Re=300.0, qinf=W.freestream(2, G), scheme=W.TENO5,
                      bc=((0, 1), (1, 1), (0, 0)))
    Q = W.random_smooth_state(spec, seed=4, amp=3e-3, step=0.05)
    ib = _ib()
    out = []
    for explicit in (False, True):
        g = ib.Grid(spec, strict=True)
        if explicit:
            for a in range(2):
                h = (spec.hi[a] - spec.lo[a]) / spec.n[a]
                i = np.arange(-4, spec.n[a] + 4)
                g.set_mesh(a, np.array([spec.lo[a] + (float(k) + 0.5) * h for k in i]),
                           np.full(i.size, h))
        g.set_state(Q)
        out.append(g.rhs().cpu().numpy())
    np.testing.assert_array_equal(out[0], out[1])


def test_set_mesh_rejects_bad_arrays():
    ib = _ib()
    spec = W.GridSpec(dim=2, n=(10, 8, 1), lo=(0, 0, 0), hi=(1, 1, 1), qinf=W.freestream(2, G),
                      bc=((0, 0), (2, 2), (0, 0)))
    g = ib.Grid(spec)
    x = np.linspace(-0.35, 1.35, 18)
    with pytest.raises(ib.IbfsaError):
        g.set_mesh(0, x[::-1], np.full(18, 0.1))     # decreasing nodes
    with pytest.raises(ib.IbfsaError):
        g.set_mesh(0, x, np.full(18, -0.1))          # negative metric
    with pytest.raises(ib.IbfsaError):
        g.set_mesh(1, np.linspace(0, 1, 16), np.full(16, 0.1))  # periodic direction
    g.set_mesh(0, x, np.full(18, 0.1))
    g.set_mesh(0)  # uniform again
