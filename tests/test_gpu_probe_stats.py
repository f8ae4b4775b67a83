"""GPU probe statistics (Sec. 3.2: dp~ = dp - its time mean; the RMS of dp~ of Sec. 3.3 and 4)
against the oracle's two-pass definition applied to the oracle's own probe histories, the edge
cases of the accumulator, and the full-size rotating cylinder on the Doppler ring of Sec. 3.3.

The GPU folds samples one by one (Welford), the oracle sums two passes: the two differ by
rounding only, bounded by T eps max|dp| for the mean and by that plus 1e-9 of the RMS for the
RMS over T samples."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00182_gb300 import workloads as W
from tests import cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


def _ib():
    from paper_1905_00182_gb300 import ibfsa
    ibfsa.lib()
    return ibfsa


def _close(gm, gr, want_m, want_r, hist):
    T, big = hist.shape[0], np.abs(hist).max()
    assert np.all(np.abs(gm - want_m) <= T * EPS * big), np.abs(gm - want_m).max()
    assert np.all(np.abs(gr - want_r) <= 1e-9 * want_r + T * EPS * big), np.abs(gr - want_r).max()


def test_probe_stats_match_the_oracle_on_its_own_histories():
    ib = _ib()
    c = cases.case_2d_weno()
    xp = np.array([[0.5, -0.6, 0.9, -0.9, 0.2], [0.5, -0.4, -0.7, 0.8, 0.0]])
    T = 25
    g = ib.Grid(c["spec"], strict=True, max_probes=8)
    g.set_state(c["Q"])
    g.set_markers(c["X"], c["U"], c["dS"])
    xi_d = torch.from_numpy(np.ascontiguousarray(c["xi"])).to(g.device)
    ib.ibfsa_set_penalty_integral(g.h, xi_d.data_ptr())
    acc = torch.zeros(3 * xp.shape[1], dtype=torch.float64, device=g.device)
    gpu_hist = []
    Q, xi, orc_hist = c["Q"], c["xi"], []
    for _ in range(T):
        g.rk3_step(c["dt"], 1)
        gpu_hist.append(g.probe_accumulate(xp, acc).cpu().numpy())
        Q, xi = O.rk3(c["spec"], Q, c["dt"], 1, c["X"], c["U"], c["dS"], xi)
        orc_hist.append(O.probe(c["spec"], Q, xp))
    assert g.status() == 0
    gpu_hist, orc_hist = np.array(gpu_hist), np.array(orc_hist)
    # the strict form samples exactly the oracle's probe values
    assert np.array_equal(gpu_hist, orc_hist)
    # the samples folded are the ones ibfsa_probe returns
    assert np.array_equal(g.probe(xp).cpu().numpy(), gpu_hist[-1])
    mean, rms = (t.cpu().numpy() for t in g.probe_stats(acc))
    want_m, want_r = O.probe_stats(orc_hist)
    assert np.all(want_r > 0)
    _close(mean, rms, want_m, want_r, orc_hist)
    assert np.array_equal(acc[:xp.shape[1]].cpu().numpy(), np.full(xp.shape[1], float(T)))


def test_probe_stats_edge_cases():
    ib = _ib()
    c = cases.case_2d_weno()
    g = ib.Grid(c["spec"], strict=True, max_probes=4)
    g.set_state(c["Q"])
    xp = np.array([[0.1, 0.3], [0.2, -0.1]])
    acc = torch.zeros(6, dtype=torch.float64, device=g.device)
    mean, rms = g.probe_stats(acc)                    # no samples yet: 0 and 0
    assert not mean.any() and not rms.any()
    once = g.probe_accumulate(xp, acc).cpu().numpy()  # one sample: mean = sample, RMS = 0
    mean, rms = g.probe_stats(acc)
    assert np.array_equal(mean.cpu().numpy(), once) and not rms.any()
    ib.ibfsa_probe_accumulate(g.h, 0, 0, 0, 0)       # zero probes: nothing to do
    ib.ibfsa_probe_stats(g.h, 0, 0, 0, 0)
    host = np.zeros(6)
    with pytest.raises(ib.IbfsaError):                # host accumulator rejected before any launch
        ib.ibfsa_probe_accumulate(g.h, 2, torch.as_tensor(xp, device=g.device).data_ptr(), 0,
                                  host.ctypes.data)
    with pytest.raises(ib.IbfsaError):                # more probes than the grid holds
        g.probe_accumulate(np.zeros((2, 5)), torch.zeros(15, dtype=torch.float64, device=g.device))
    assert g.status() == 0


def test_rotating_cylinder_doppler_ring_full_size():
    """2048^2 rotating cylinder (FP32 form), 360 probes on the Doppler ring r = 2 (1 - 0.2 cos
    theta), sampled every 10 steps over 600 steps (t c / D = 5.3: the start-up sound has
    crossed the ring): the accumulated statistics against the oracle's definition applied to
    the sampled history."""
    ib = _ib()
    w = W.rotating_cylinder_2d(precision=W.FP32_PERTURB)
    xp = W.doppler_ring_probes(360, 2.0, 0.2)
    g = ib.Grid(w["spec"], max_probes=360)
    g.set_state(w["Q"])
    g.set_markers(w["X"], w["U"], w["dS"])
    acc = torch.zeros(3 * 360, dtype=torch.float64, device=g.device)
    hist = []
    for _ in range(60):
        g.rk3_step(w["dt"], 10)
        hist.append(g.probe_accumulate(xp, acc).cpu().numpy())
    assert g.status() == 0
    hist = np.array(hist)
    mean, rms = (t.cpu().numpy() for t in g.probe_stats(acc))
    want_m, want_r = O.probe_stats(hist)
    assert np.all(want_r > 0)
    _close(mean, rms, want_m, want_r, hist)
