"""Edge cases on the GPU: degenerate grid sizes (1 to 4 cells in a direction, narrower than one
stencil), all boundary rules on tiny grids, a NaN planted in the state on the host (reported
through the device status word, never a trap), and argument errors on a live grid."""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00182_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ib():
    from paper_1905_00182_gb300 import ibfsa
    ibfsa.lib()
    return ibfsa


EDGE_GRIDS = [
    (2, (1, 7, 1), ((0, 0), (0, 0), (0, 0)), W.TENO5),
    (2, (3, 5, 1), ((0, 1), (1, 0), (0, 0)), W.WENO5JS),
    (2, (4, 4, 1), ((2, 2), (2, 2), (0, 0)), W.TENO5),
    (3, (2, 3, 4), ((0, 0), (1, 1), (2, 2)), W.TENO5),
    (3, (1, 1, 1), ((0, 0), (0, 0), (0, 0)), W.WENO5JS),
]


@pytest.mark.parametrize("dim,n,bc,scheme", EDGE_GRIDS)
def test_tiny_grids_strict_bitwise(dim, n, bc, scheme):
    spec = W.GridSpec(dim=dim, n=n, lo=(0, 0, 0), hi=(1.0, 0.8, 0.6), Re=40.0,
                      qinf=W.freestream(dim, 1.4, vel=(0.1, -0.05, 0.02)), scheme=scheme, bc=bc)
    Q = W.random_smooth_state(spec, seed=21, amp=3e-2, vel0=(0.1, -0.05, 0.02))
    ib = _ib()
    g = ib.Grid(spec, strict=True)
    g.set_state(Q)
    L = g.rhs().cpu().numpy()
    np.testing.assert_array_equal(L, O.rhs(spec, Q))
    dt = 0.05 * min(spec.h)
    g.rk3_step(dt, 2)
    Qo, _ = O.rk3(spec, Q, dt, 2)
    np.testing.assert_array_equal(g.get_state().cpu().numpy(), Qo)
    assert g.status() == 0
    # the other forms run on them too
    for prec in (W.FP64, W.FP32_PERTURB):
        gf = ib.Grid(dataclasses.replace(spec, precision=prec))
        gf.set_state(Q)
        gf.rk3_step(dt, 2)
        assert np.all(np.isfinite(gf.get_state().cpu().numpy()))
        assert gf.status() == 0


@pytest.mark.parametrize("prec", [W.FP64, W.FP32_PERTURB])
def test_nan_in_state_is_reported_not_trapped(prec):
    ib = _ib()
    w = W.cylinder_pulse_2d(n=64, markers=40)
    Q = w["Q"].copy()
    Q[0, 0, 30, 30] = np.nan
    g = ib.Grid(dataclasses.replace(w["spec"], precision=prec))
    g.set_state(Q)
    g.rk3_step(w["dt"], 1)
    assert g.status() & ib.IBFSA_STATUS_NONFINITE
    # the context stays usable: a clean state steps without errors afterwards
    g.set_state(w["Q"])
    g.rk3_step(w["dt"], 1)
    assert g.status() == 0


def test_argument_errors_on_a_live_grid():
    ib = _ib()
    w = W.cylinder_pulse_2d(n=64, markers=40)
    g = ib.Grid(w["spec"], max_probes=2)
    g.set_state(w["Q"])
    X = np.zeros((2, 41))
    with pytest.raises(ib.IbfsaError) as e:
        g.set_markers(X, X, np.zeros(41))      # more markers than the grid was made for
    assert e.value.code == ib.IBFSA_ERR_ARG
    with pytest.raises(ib.IbfsaError):
        g.probe(np.zeros((2, 3)))              # more probes than capacity
    with pytest.raises(ib.IbfsaError):
        g.rk3_step(-1.0, 1)
    g.set_markers(np.zeros((2, 0)), np.zeros((2, 0)), np.zeros(0))  # zero markers is valid
    g.rk3_step(w["dt"], 1)
    assert g.status() == 0
