"""Sec. 3.1's pulse scattered by a rigid cylinder, against the exact linear-acoustics solution
(tests/acoustic_scattering.py), on the GPU at D/h = 12.8, 25 and 50.  The FP64 runs take the
bit-reproducible arithmetic (equal to the oracle's, which the parity tests show bit for bit),
so this is the oracle's convergence study at sizes the CPU does not reach in a test; the FP32
perturbation form must match the FP64 error.  Probes at (2, 0) and (2, 2), on the source's side,
and at (-2, 0) and (-3, 0) behind the cylinder, where only the diffracted wave arrives and the
diffuse interface limits the error to first order in h."""
import dataclasses

import numpy as np
import pytest

from paper_1905_00182_gb300 import workloads as W
from tests import cases
from tests.acoustic_scattering import scattered_pulse

torch = pytest.importorskip("torch")
pytest.importorskip("scipy.special")
pytestmark = pytest.mark.gpu


def _history(ib, case, strict):
    g = ib.Grid(case["spec"], strict=strict, max_probes=case["probes"].shape[1])
    g.set_state(case["Q"])
    g.set_markers(case["X"], case["U"], case["dS"])
    out = []
    for _ in range(case["samples"]):
        g.rk3_step(case["dt"], case["every"])
        out.append(g.probe(case["probes"]).cpu().numpy())
    assert g.status() == 0
    return np.array(out)


def test_cylinder_scattering_converges_to_linear_acoustics():
    from paper_1905_00182_gb300 import ibfsa as ib
    ib.lib()
    base = cases.cylinder_scattering(12.8)
    front = base["probes"]
    # behind the cylinder, on the source's axis (the wave diffracted round the body)
    shadow = np.array([[-2.0, -3.0], [0.0, 0.0]])
    probes = np.concatenate([front, shadow], axis=1)
    nf = front.shape[1]
    t = base["sample"] * np.arange(1, base["samples"] + 1)
    want = scattered_pulse(probes, t, nk=2500)

    def err(got, sl):
        return float(np.sqrt(np.sum((got[:, sl] - want[:, sl]) ** 2) / np.sum(want[:, sl] ** 2)))

    hist = {ppd: _history(ib, dict(cases.cylinder_scattering(ppd), probes=probes), True)
            for ppd in (12.8, 25, 50)}
    e = {ppd: err(h, slice(0, nf)) for ppd, h in hist.items()}
    es = {ppd: err(h, slice(nf, None)) for ppd, h in hist.items()}
    c25 = cases.cylinder_scattering(25)
    h32 = _history(ib, dict(c25, probes=probes,
                            spec=dataclasses.replace(c25["spec"], precision=W.FP32_PERTURB)),
                   False)
    e32 = err(h32, slice(0, nf))
    print("relative RMS of the probe histories vs exact: " +
          ", ".join(f"D/h {k}: {v:.4f}" for k, v in e.items()) +
          f"; FP32 form at D/h 25: {e32:.4f}; behind the cylinder: " +
          ", ".join(f"D/h {k}: {v:.4f}" for k, v in es.items()))
    assert e[12.8] > e[25] > e[50], e
    assert e[25] <= 0.15, e
    assert abs(e32 - e[25]) <= 0.01, (e32, e[25])
    # the diffracted wave converges too, at first order (the diffuse interface)
    assert es[12.8] > es[25] > es[50], es
    assert es[50] <= 0.3, es
