"""GPU parity of the characteristic-wise reconstruction option (charwise = 1: the split fluxes
of each stencil projected on the Euler eigenvectors at the Roe average of the face's two cells)
against the oracle's option of the same name, on the seeded cases of the component-wise parity
tests (2D/3D, WENO5-JS/TENO5, ragged sizes, viscous, markers, sponge, periodic / free-stream /
zero-gradient walls).  Strict arithmetic: bit for bit; fast arithmetic: 99 % of the cells
within a rounding bound of the split-flux scale (the projections add a few roundings of O(1)
eigenvector entries), the rest within 1 % of the largest right-hand side; the FP32 perturbation
form within the FP32 bounds of the component-wise tests times (1 + c)."""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from tests import cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


def _case(name):
    c = cases.ALL[name]()
    c["spec"] = dataclasses.replace(c["spec"], charwise=True)
    return c


def _grid(case, strict):
    from paper_1905_00182_gb300 import ibfsa as ib
    ib.lib()
    g = ib.Grid(case["spec"], strict=strict)
    g.set_state(case["Q"])
    if case["X"] is not None:
        g.set_markers(case["X"], case["U"], case["dS"])
        if case["xi"] is not None:
            xi = torch.from_numpy(np.ascontiguousarray(case["xi"])).cuda()
            ib.ibfsa_set_penalty_integral(g.h, xi.data_ptr())
            torch.cuda.synchronize()
    return g


@pytest.mark.parametrize("name", list(cases.ALL))
def test_charwise_rhs_strict_bitwise(name):
    case = _case(name)
    g = _grid(case, strict=True)
    L = g.rhs().cpu().numpy()
    assert g.status() == 0
    Lo = O.rhs(case["spec"], case["Q"], case["X"], case["U"], case["dS"], case["xi"])
    np.testing.assert_array_equal(L, Lo)
    # and it is a different discretisation from the component-wise one
    Lc = O.rhs(dataclasses.replace(case["spec"], charwise=False), case["Q"], case["X"],
               case["U"], case["dS"], case["xi"])
    assert np.max(np.abs(Lc - Lo)) > 0.0


@pytest.mark.parametrize("name", ["2d_weno", "3d_teno"])
def test_charwise_rk3_strict_bitwise(name):
    case = _case(name)
    g = _grid(case, strict=True)
    g.rk3_step(case["dt"], 2)
    Q = g.get_state().cpu().numpy()
    assert g.status() == 0
    Qo, _ = O.rk3(case["spec"], case["Q"], case["dt"], 2, case["X"], case["U"], case["dS"],
                  case["xi"])
    np.testing.assert_array_equal(Q, Qo)


@pytest.mark.parametrize("name", list(cases.ALL))
def test_charwise_rhs_fast_within_rounding_bound(name):
    case = _case(name)
    g = _grid(case, strict=False)
    L = g.rhs().cpu().numpy()
    assert g.status() == 0
    Lo = O.rhs(case["spec"], case["Q"], case["X"], case["U"], case["dS"], case["xi"])
    spec, Q = case["spec"], case["Q"]
    # split-flux scale / h per component, as in the component-wise parity tests
    rho = Q[0]
    u = [Q[1 + a] / rho for a in range(spec.dim)]
    p = (spec.gamma - 1.0) * (Q[-1] - 0.5 * sum(Q[1 + a] * u[a] for a in range(spec.dim)))
    c = np.sqrt(spec.gamma * p / rho)
    alpha = max(np.max(np.abs(u[a]) + c) for a in range(spec.dim))
    scale = ((np.max(np.abs(Q)) * (1.0 + alpha) + np.max(np.abs(p))) * (1.0 + np.max(c))
             / min(spec.h))
    err = np.abs(L - Lo)
    # rounding of the projections and reconstructions everywhere; a TENO cut-off that the
    # fused arithmetic decides differently right at its threshold may move a few faces further
    assert np.quantile(err, 0.99) <= 2.0 ** 14 * EPS * scale, (np.quantile(err, 0.99), scale)
    assert err.max() <= 1e-2 * np.max(np.abs(Lo)), err.max()


# ---- the option in the FP32 perturbation form -------------------------------------------------
# The split-flux perturbations are projected on eigenvectors built in FP32 from the Roe average
# of the face's full primitive state: per right-hand side a few FP32 roundings of the
# perturbation fluxes, each projection adding roundings of O(1) eigenvector entries (at most
# (1 + c) times the component-wise bound, c the largest sound speed).

def _perturbation_scale(spec, Q):
    from tests.test_gpu_fp32 import _perturbation_scale as ps
    return ps(spec, Q)


@pytest.mark.parametrize("name", list(cases.ALL))
def test_charwise_rhs_fp32_within_fp32_roundings(name):
    from paper_1905_00182_gb300 import workloads as W
    case = _case(name)
    spec32 = dataclasses.replace(case["spec"], precision=W.FP32_PERTURB)
    g = _grid(dict(case, spec=spec32), strict=False)
    L = g.rhs().cpu().numpy()
    assert g.status() == 0
    Lo = O.rhs(case["spec"], case["Q"], case["X"], case["U"], case["dS"], case["xi"])
    Lc = O.rhs(dataclasses.replace(case["spec"], charwise=False), case["Q"], case["X"],
               case["U"], case["dS"], case["xi"])
    spec, Q = case["spec"], case["Q"]
    rho = Q[0]
    u = [Q[1 + a] / rho for a in range(spec.dim)]
    p = (spec.gamma - 1.0) * (Q[-1] - 0.5 * sum(Q[1 + a] * u[a] for a in range(spec.dim)))
    amp = 1.0 + float(np.max(np.sqrt(spec.gamma * p / rho)))
    sc = _perturbation_scale(spec, Q) * amp
    for c in range(spec.nv):
        err = np.abs(L[c] - Lo[c])
        rms = float(np.sqrt(np.mean(err ** 2)))
        print(f"{name} comp {c}: RMS {rms:.3e} (bound {64 * EPS32 * sc[c]:.3e}), 99.9 % "
              f"{np.quantile(err, 0.999):.3e}, charwise - componentwise RMS "
              f"{np.sqrt(np.mean((Lo[c] - Lc[c]) ** 2)):.3e}")
        assert rms <= 64 * EPS32 * sc[c], (c, rms, sc[c])
        assert np.quantile(err, 0.999) <= 256 * EPS32 * sc[c], c


def test_charwise_fp32_steps_track_the_oracle():
    from paper_1905_00182_gb300 import workloads as W
    case = _case("2d_teno_stream")
    spec32 = dataclasses.replace(case["spec"], precision=W.FP32_PERTURB)
    g = _grid(dict(case, spec=spec32), strict=False)
    g.rk3_step(case["dt"], 10)
    Q = g.get_state().cpu().numpy()
    assert g.status() == 0
    Qo, _ = O.rk3(case["spec"], case["Q"], case["dt"], 10, case["X"], case["U"], case["dS"],
                  case["xi"])
    qinf = np.array(case["spec"].qinf[:4])
    for c in range(4):
        pert = np.linalg.norm(Qo[c] - qinf[c])
        assert np.linalg.norm(Q[c] - Qo[c]) <= 1e-4 * pert, c


EPS32 = float(np.finfo(np.float32).eps)
