"""ibfsa_rhs_noalloc: the right-hand side for callers that cannot allocate device memory.

Such callers (plug-ins whose host application owns the device-memory budget, loops that must
not pay cudaMalloc's implicit synchronisation, front ends that only pass pointers) get the same
result as ibfsa_rhs without a grid object or workspace; the scratch lives in a static device
array inside the library.  The GPU test calls the entry point through the C ABI three times in a
row: strict arithmetic on one grid, fast arithmetic on another (so it runs on scratch the first
call left behind), then strict arithmetic on the first grid again, on scratch the fast call left
behind (the strict form's force field must be cleared by the call itself); each result is
checked against the grid entry point ibfsa_rhs.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1905_00182_gb300 import workloads as W
from tests import cases

EPS = np.finfo(np.float64).eps


def _ib():
    from paper_1905_00182_gb300 import build as B
    try:
        B.nvcc()
    except RuntimeError as e:  # no CUDA toolchain on this machine: nothing to build or load
        pytest.skip(str(e))
    B.build()  # a compile error fails the test
    from paper_1905_00182_gb300 import ibfsa
    try:
        ibfsa.lib()
    except OSError as e:  # the CUDA runtime library cannot be loaded here
        pytest.skip(f"libibfsa cannot be loaded: {e}")
    return ibfsa


def _flux_scale(spec, Q):
    nv, dim = spec.nv, spec.dim
    u = [Q[1 + a] / Q[0] for a in range(dim)]
    p = (spec.gamma - 1.0) * (Q[nv - 1] - 0.5 * sum(Q[1 + a] * u[a] for a in range(dim)))
    alpha = max(np.max(np.abs(u[a]) + np.sqrt(spec.gamma * p / Q[0])) for a in range(dim))
    return np.array([(np.max(np.abs(Q[c])) * (alpha + 2.0) + np.max(np.abs(p))) / min(spec.h)
                     for c in range(nv)])


def _noalloc_rhs(ib, torch, case, strict):
    spec = case["spec"]
    desc = ib.desc_from_spec(spec, strict=strict)
    dev = torch.device("cuda")
    Q = torch.from_numpy(np.ascontiguousarray(case["Q"])).to(dev)
    L = torch.full(spec.shape(), float("nan"), dtype=torch.float64, device=dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    nm = 0 if case["X"] is None else case["X"].shape[1]
    if nm:
        X = torch.from_numpy(np.ascontiguousarray(case["X"])).to(dev)
        U = torch.from_numpy(np.ascontiguousarray(case["U"])).to(dev)
        dS = torch.from_numpy(np.ascontiguousarray(case["dS"])).to(dev)
        xi = torch.from_numpy(np.ascontiguousarray(case["xi"])).to(dev)
        F = torch.full((spec.dim, nm), float("nan"), dtype=torch.float64, device=dev)
        ptrs = (X.data_ptr(), U.data_ptr(), dS.data_ptr(), xi.data_ptr(), F.data_ptr())
    else:
        F = None
        ptrs = (0, 0, 0, 0, 0)
    stream = torch.cuda.current_stream()
    ib.ibfsa_rhs_noalloc(desc, Q.data_ptr(), nm, ptrs[0], ptrs[1], ptrs[2], ptrs[3],
                         L.data_ptr(), ptrs[4], status.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return L.cpu().numpy(), (None if F is None else F.cpu().numpy()), int(status.item())


def _grid_rhs(ib, case, strict):
    import torch
    g = ib.Grid(case["spec"], strict=strict)
    g.set_state(case["Q"])
    F = None
    if case["X"] is not None:
        g.set_markers(case["X"], case["U"], case["dS"])
        xi = torch.from_numpy(np.ascontiguousarray(case["xi"])).cuda()
        ib.ibfsa_set_penalty_integral(g.h, xi.data_ptr())
    L = g.rhs().cpu().numpy()
    if case["X"] is not None:
        F = g.marker_forces().cpu().numpy()
    g.close()
    return L, F


@pytest.mark.gpu
def test_noalloc_rhs_matches_grid_rhs_on_calls_in_a_row():
    torch = pytest.importorskip("torch")
    ib = _ib()
    first = cases.case_2d_weno()      # strict arithmetic: must agree bit for bit
    second = cases.case_3d_teno()     # fast arithmetic, different grid and marker count

    L1, F1, st1 = _noalloc_rhs(ib, torch, first, strict=True)
    L2, F2, st2 = _noalloc_rhs(ib, torch, second, strict=False)
    L3, F3, st3 = _noalloc_rhs(ib, torch, first, strict=True)   # on the fast call's leftovers

    R1, G1 = _grid_rhs(ib, first, strict=True)
    np.testing.assert_array_equal(L1, R1)
    np.testing.assert_array_equal(F1, G1)
    assert st1 == 0

    R2, G2 = _grid_rhs(ib, second, strict=False)
    sc = _flux_scale(second["spec"], second["Q"])
    for c in range(second["spec"].nv):
        # atomics may sum the spreading contributions in another order: a few roundings of the
        # split-flux scale, the tolerance of the other fast-arithmetic parity tests
        assert np.max(np.abs(L2[c] - R2[c])) <= 64 * EPS * sc[c], c
    np.testing.assert_array_equal(F2, G2)
    assert st2 == 0

    np.testing.assert_array_equal(L3, R1)
    np.testing.assert_array_equal(F3, G1)
    assert st3 == 0


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    ib = _ib()
    spec = W.GridSpec(dim=3, n=(96, 96, 96), lo=(0, 0, 0), hi=(1, 1, 1), Re=100.0,
                      qinf=W.freestream(3, 1.4))
    desc = ib.desc_from_spec(spec)
    with pytest.raises(ib.IbfsaError) as e:
        ib.ibfsa_rhs_noalloc(desc, 1 << 20, 0, 0, 0, 0, 0, 1 << 21)
    assert e.value.code == ib.IBFSA_ERR_WORKSPACE
    assert b"static scratch" in ib.lib().ibfsa_last_error()
