"""Host-side checks of the C ABI that need no GPU: the library builds for sm_103a, loads, exports
every symbol include/ibfsa.h declares, and rejects bad descriptors before touching a device."""
import os
import re

import pytest

from paper_1905_00182_gb300 import build as B
from paper_1905_00182_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ib():
    B.build()
    from paper_1905_00182_gb300 import ibfsa
    ibfsa.lib()
    return ibfsa


def _declared():
    with open(os.path.join(ROOT, "include", "ibfsa.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"\b(ibfsa_\w+)\s*\(", src)))


def test_header_and_binding_agree(ib):
    assert _declared() == sorted(ib.EXPORTS)


def test_every_declared_symbol_exported(ib):
    L = ib.lib()
    for name in _declared():
        assert hasattr(L, name), name


def _good():
    return W.GridSpec(dim=3, n=(16, 12, 8), lo=(0, 0, 0), hi=(1, 1, 1), Re=10.0,
                      qinf=W.freestream(3, 1.4), max_markers=10)


def test_workspace_bytes_counts_buffers(ib):
    spec = _good()
    nbytes = ib.ibfsa_workspace_bytes(ib.desc_from_spec(spec))
    N = 16 * 12 * 8
    NP = 24 * 20 * 16
    NB = 20 * 16 * 12
    expect = 8 * (4 * 5 * N + 5 * NP + 4 * NP + 12 * NB)
    assert expect <= nbytes <= expect + 64 * 1024
    # strict arithmetic adds the marker-order spreading buffer
    assert ib.ibfsa_workspace_bytes(ib.desc_from_spec(spec, strict=True)) >= nbytes + 8 * 3 * N


@pytest.mark.parametrize("field,value,code", [
    ("dim", 4, -1), ("n", (0, 12, 8), -1), ("hi", (0.0, 1.0, 1.0), -1),
    ("bc", ((2, 0), (0, 0), (0, 0)), -1), ("bc", ((2, 2), (0, 0), (0, 0)), None),
    ("n", (3, 12, 8), None), ("gamma", 1.0, -1), ("scheme", 7, -5), ("precision", 9, -5),
    ("charwise", True, None), ("charwise", 2, -1),
    ("bc", ((3, 3), (3, 1), (0, 3)), None), ("bc", ((4, 0), (0, 0), (0, 0)), -1),
])
def test_descriptor_validation(ib, field, value, code):
    spec = _good()
    setattr(spec, field, value)
    if field == "n" and value[0] == 3:
        spec.bc = ((2, 2), (0, 0), (0, 0))  # periodic with n < 4 ghosts
        code = -1
    if code is None:
        assert ib.ibfsa_workspace_bytes(ib.desc_from_spec(spec)) > 0
        return
    with pytest.raises(ib.IbfsaError) as e:
        ib.ibfsa_workspace_bytes(ib.desc_from_spec(spec))
    assert e.value.code == code
    assert ib.lib().ibfsa_last_error()


def test_characteristic_face_needs_five_cells(ib):
    spec = _good()
    spec.n = (16, 12, 4)
    spec.bc = ((0, 0), (0, 0), (0, 3))
    with pytest.raises(ib.IbfsaError) as e:
        ib.ibfsa_workspace_bytes(ib.desc_from_spec(spec))
    assert e.value.code == ib.IBFSA_ERR_ARG
    spec.n = (16, 12, 5)
    assert ib.ibfsa_workspace_bytes(ib.desc_from_spec(spec)) > 0


def test_charwise_in_every_form_but_the_learned_one(ib):
    spec = _good()
    spec.charwise = True
    spec.precision = W.FP32_PERTURB
    assert ib.ibfsa_workspace_bytes(ib.desc_from_spec(spec)) > 0
    spec.scheme = W.MLP_TENO5
    with pytest.raises(ib.IbfsaError) as e:
        ib.ibfsa_workspace_bytes(ib.desc_from_spec(spec))
    assert e.value.code == ib.IBFSA_ERR_UNSUPPORTED


def test_plate_workspace_counts_buffers(ib):
    ps = W.PlateSpec(n_el=40, n_markers=800)
    nbytes = ib.ibfsa_plate_workspace_bytes(ib.plate_desc_from_spec(ps))
    # e, v, Fbar, X, U, dS, marker shape values, force result, step velocities; marker elements
    # and first marker per element
    expect = 8 * (2 * 164 + 4 * 2 * 800 + 800 + 4 * 800 + 3) + 4 * (800 + 41)
    assert expect <= nbytes <= expect + 13 * 256


@pytest.mark.parametrize("field,value", [
    ("n_el", 0), ("n_el", 129), ("n_markers", 0), ("length", 0.0), ("rho_s", -1.0),
    ("K_S", -1.0), ("clamped", 3), ("newton_max", 0), ("newton_tol", 0.0),
])
def test_plate_descriptor_validation(ib, field, value):
    ps = W.PlateSpec()
    setattr(ps, field, value)
    d = ib.plate_desc_from_spec(ps)
    if field == "clamped":
        d.clamp = value
    with pytest.raises(ib.IbfsaError) as e:
        ib.ibfsa_plate_workspace_bytes(d)
    assert e.value.code == -1
    assert ib.ibfsa_plate_workspace_bytes(ib.plate_desc_from_spec(W.PlateSpec())) > 0
