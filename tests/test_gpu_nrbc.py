"""GPU parity of the characteristic non-reflecting faces (IBFSA_BC_CHARACTERISTIC; Sec. 2,
after Thompson) against the oracle's boundary rule 3, and the condition at work on the GPU.

* strict FP64: bit for bit (right-hand side with markers, viscosity, sponge and source; three
  SSP-RK3 steps; 2D and 3D, both schemes, corner cells where two characteristic faces meet, a
  stretched direction, the characteristic-wise reconstruction);
* fast FP64 within 64 eps of the split-flux scale; FP32 form within the FP32 bounds of the
  uniform-grid tests (RMS 64 eps32, 99.9 % quantile 256 eps32 of the perturbation-flux scale);
* a free stream gives exactly zero in all forms;
* a planar acoustic pulse leaves a box through characteristic faces with a reflection far below
  that of zero-gradient ghosts (FP32 form, against a box three times larger).
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00182_gb300 import workloads as W
from tests import cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = float(np.finfo(np.float64).eps)
EPS32 = float(np.finfo(np.float32).eps)
CH = W.BC_CHARACTERISTIC


def _ib():
    from paper_1905_00182_gb300 import ibfsa
    ibfsa.lib()
    return ibfsa


def _case(name):
    if name == "2d_weno":
        c = cases.case_2d_weno()
        c["spec"] = dataclasses.replace(c["spec"], bc=((CH, CH), (CH, 1), (0, 0)),
                                        sponge_cells=3, sponge_sigma=1.5)
    elif name == "2d_teno":
        c = cases.case_2d_weno()
        c["spec"] = dataclasses.replace(c["spec"], scheme=W.TENO5, bc=((0, CH), (CH, CH), (0, 0)))
    elif name == "3d_teno":
        c = cases.case_3d_teno()
        c["spec"] = dataclasses.replace(c["spec"], bc=((CH, CH), (0, CH), (CH, 1)))
    else:  # 3D WENO, a stream through the box, no markers
        c = cases.case_3d_weno_periodic()
        q = W.freestream(3, 1.4, vel=(0.2, -0.1, 0.15))
        c["spec"] = dataclasses.replace(c["spec"], bc=((CH, CH), (CH, CH), (2, 2)), qinf=q)
    return c


NAMES = ["2d_weno", "2d_teno", "3d_teno", "3d_weno_stream"]


def _grid(case, strict, precision=W.FP64, charwise=False, mesh=None):
    ib = _ib()
    spec = dataclasses.replace(case["spec"], precision=precision, charwise=charwise)
    g = ib.Grid(spec, strict=strict)
    if mesh is not None:
        for a, m in enumerate(mesh):
            if m is not None:
                g.set_mesh(a, *m)
    g.set_state(case["Q"])
    if case["X"] is not None:
        g.set_markers(case["X"], case["U"], case["dS"])
        xi = torch.from_numpy(np.ascontiguousarray(case["xi"])).cuda()
        ib.ibfsa_set_penalty_integral(g.h, xi.data_ptr())
        torch.cuda.synchronize()
    return g


def _scale(spec, Q, perturbation=False):
    from tests.test_gpu_fp32 import _perturbation_scale
    from tests.test_gpu_parity import _flux_scale
    return _perturbation_scale(spec, Q) if perturbation else _flux_scale(spec, Q)


@pytest.mark.parametrize("name", NAMES)
def test_characteristic_rhs_strict_bitwise(name):
    case = _case(name)
    g = _grid(case, strict=True)
    L = g.rhs().cpu().numpy()
    assert g.status() == 0
    Lo = O.rhs(case["spec"], case["Q"], case["X"], case["U"], case["dS"], case["xi"])
    np.testing.assert_array_equal(L, Lo)


def test_characteristic_rhs_strict_bitwise_charwise_and_stretched():
    case = _case("2d_teno")
    spec = case["spec"]
    ax = W.stretched_axis(spec.n[0], 0.06, 0.1, 21, 6, center=0.05)
    mesh = [(ax[2], ax[3]), None]
    case["spec"] = dataclasses.replace(spec, lo=(ax[0], spec.lo[1], 0.0), hi=(ax[1], spec.hi[1], 1.0))
    case["X"] = None
    for charwise in (False, True):
        g = _grid(case, strict=True, charwise=charwise, mesh=mesh)
        L = g.rhs().cpu().numpy()
        assert g.status() == 0
        Lo = O.rhs(case["spec"], case["Q"], charwise=charwise, stretch=mesh)
        np.testing.assert_array_equal(L, Lo)


@pytest.mark.parametrize("name", ["2d_weno", "3d_teno"])
def test_characteristic_rk3_strict_bitwise(name):
    case = _case(name)
    g = _grid(case, strict=True)
    g.rk3_step(case["dt"], 3)
    Q = g.get_state().cpu().numpy()
    assert g.status() == 0
    Qo, _ = O.rk3(case["spec"], case["Q"], case["dt"], 3, case["X"], case["U"], case["dS"],
                  case["xi"])
    np.testing.assert_array_equal(Q, Qo)


@pytest.mark.parametrize("name", NAMES)
def test_characteristic_rhs_fast_and_fp32(name):
    case = _case(name)
    Lo = O.rhs(case["spec"], case["Q"], case["X"], case["U"], case["dS"], case["xi"])
    g = _grid(case, strict=False)
    L = g.rhs().cpu().numpy()
    sc = _scale(case["spec"], case["Q"])
    for c in range(case["spec"].nv):
        assert np.max(np.abs(L[c] - Lo[c])) <= 64 * EPS * sc[c], c
    g = _grid(case, strict=False, precision=W.FP32_PERTURB)
    L = g.rhs().cpu().numpy()
    assert g.status() == 0
    sc = _scale(case["spec"], case["Q"], perturbation=True)
    for c in range(case["spec"].nv):
        err = np.abs(L[c] - Lo[c])
        assert np.sqrt(np.mean(err ** 2)) <= 64 * EPS32 * sc[c], c
        assert np.quantile(err, 0.999) <= 256 * EPS32 * sc[c], c


@pytest.mark.parametrize("strict,precision", [(True, W.FP64), (False, W.FP64),
                                              (False, W.FP32_PERTURB)])
def test_characteristic_free_stream_gives_zero(strict, precision):
    case = _case("3d_weno_stream")
    case["Q"] = W.rest_state(case["spec"])
    g = _grid(case, strict=strict, precision=precision)
    assert torch.all(g.rhs() == 0.0)


def _pulse_run(L, n, bc, mach, T):
    spec = W.GridSpec(dim=2, n=(n, 8, 1), lo=(-L, 0.0, 0.0), hi=(L, 8 * 2 * L / n, 1.0),
                      gamma=1.4, Re=0.0, qinf=W.freestream(2, 1.4, vel=(mach, 0.0, 0.0)),
                      scheme=W.TENO5, precision=W.FP32_PERTURB, bc=((bc, bc), (2, 2), (0, 0)))
    X, _, _ = W.mesh(spec)
    dp = 1e-3 * np.exp(-math.log(2.0) * (X / 0.25) ** 2)
    Q = W.conservative(spec, 1.0 + dp, [mach + dp, np.zeros(X.shape)], 1.0 / 1.4 + dp)
    g = _ib().Grid(spec)
    g.set_state(Q)
    h = 2 * L / n
    steps = int(math.ceil(T / (0.2 * h / (1.0 + mach))))
    g.rk3_step(T / steps, steps)
    Qe = g.get_state().cpu().numpy()
    assert g.status() == 0
    ke = (Qe[1] ** 2 + Qe[2] ** 2) / Qe[0]
    return (0.4 * (Qe[3] - 0.5 * ke) - 1.0 / 1.4)[0]


@pytest.mark.parametrize("mach", [0.0, 0.2])
def test_characteristic_faces_let_a_pulse_out_on_the_gpu(mach):
    n, L = 80, 1.0
    T = 1.5 / (1.0 + mach)
    ref = _pulse_run(3 * L, 3 * n, 0, mach, T)[:, n:2 * n]
    e_zg = np.abs(_pulse_run(L, n, 0, mach, T) - ref).max()
    e_ch = np.abs(_pulse_run(L, n, CH, mach, T) - ref).max()
    print(f"M {mach}: reflected max |dp| zero-gradient {e_zg:.3e}, characteristic {e_ch:.3e}")
    assert e_ch < 0.2 * e_zg and e_ch < 5e-6
