"""Body force and power from the Lagrangian penalty forces (Eq. 7): against the oracle's marker
forces, and against the momentum source the spreading of Eq. 9 puts into the fluid (the force
the body exerts on the fluid is the opposite of the force on the body)."""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00182_gb300 import workloads as W
from tests import cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ib():
    from paper_1905_00182_gb300 import ibfsa
    ibfsa.lib()
    return ibfsa


@pytest.mark.parametrize("name", ["2d_weno", "3d_teno"])
def test_body_force_matches_oracle_marker_forces(name):
    ib = _ib()
    case = cases.ALL[name]()
    g = ib.Grid(case["spec"], strict=True)
    g.set_state(case["Q"])
    g.set_markers(case["X"], case["U"], case["dS"])
    xi = torch.from_numpy(np.ascontiguousarray(case["xi"])).cuda()
    ib.ibfsa_set_penalty_integral(g.h, xi.data_ptr())
    g.rhs()
    force, power = ib.ibfsa_body_force(g.h)
    _, F, _, _ = O.rhs(case["spec"], case["Q"], case["X"], case["U"], case["dS"], case["xi"],
                       return_markers=True)
    want = (F * case["dS"][None, :]).sum(1)
    want_p = np.sum(F * case["U"] * case["dS"][None, :])
    dim = case["spec"].dim
    np.testing.assert_allclose(force[:dim], want, rtol=1e-13, atol=1e-16)
    assert power == pytest.approx(want_p, rel=1e-13, abs=1e-16)


def test_momentum_given_to_the_fluid_is_minus_the_body_force():
    # fluid at rest, uniform: the convective and viscous terms vanish, so L = S and
    # sum_j L_m,j h^2 = -sum_k F_k dS_k (partition of unity of the four-point kernel)
    ib = _ib()
    w = W.cylinder_pulse_2d(n=128, markers=200)
    spec = w["spec"]
    Q = np.empty(spec.shape())
    for c in range(spec.nv):
        Q[c] = spec.qinf[c]
    X, U, dS = W.circle_markers(200, 0.5, omega=0.3)
    for prec in (W.FP64, W.FP32_PERTURB):
        g = ib.Grid(dataclasses.replace(spec, precision=prec))
        g.set_state(Q)
        g.set_markers(X, U, dS)
        L = g.rhs().cpu().numpy()
        force, power = ib.ibfsa_body_force(g.h)
        h2 = np.prod(spec.h)
        tol = 1e-12 if prec == W.FP64 else 1e-6
        for a in range(2):
            assert abs(L[1 + a].sum() * h2 + force[a]) <= tol * np.sum(np.abs(L[1 + a])) * h2
        assert power < 0.0  # the resting fluid holds the spinning wall back
