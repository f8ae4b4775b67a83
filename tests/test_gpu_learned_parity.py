"""The learned-weight form (IBFSA_MLP_TENO5) element by element against the oracle's learned
scheme, on the stress state (smooth random modes in every primitive plus a 10 % contact step),
where the network supplies the weights of nearly every reconstruction: 2D with the generic and
with the tensor-copy tiles in y, 3D, and 2D on a stretched x direction with characteristic
non-reflecting faces.

The GPU evaluates the same definition as the oracle -- TENO5's cut-off as the guard, the
normalised stencil, the network on bfloat16 parameters and bfloat16 activations, the delta-form
face value -- but in the FP32 perturbation form with FP32 accumulation and the hardware tanh
approximation inside gelu (relative error about 2^-11).  So the comparison has two parts:

* the whole right-hand side: within the FP32 form's own bound (RMS 64 eps32 of the
  perturbation-flux scale, as the TENO5 FP32 parity tests) plus the network term below;
* the network's increment over TENO5, D = L(learned) - L(TENO5), on each side: the GPU's D
  (its learned minus its TENO5 FP32 right-hand side, same split fluxes) against the oracle's.
  The tanh approximation moves a bfloat16 activation by one unit in the last place (2^-8
  relative) in about one activation out of sixteen, which moves the logits by a few 1e-3 and
  the weights' deviation from the linear ones by about a percent: the bound is
  RMS(D_gpu - D_oracle) <= 2^-4 RMS(D_oracle) per component, with the network used in more
  than 90 % of the reconstructions on both sides and the two shares of use within 0.5 %.
"""
import dataclasses
import os

import numpy as np
import pytest

from oracle import mlp_oracle as M
from oracle import oracle as O
from paper_1905_00182_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EPS32 = float(np.finfo(np.float32).eps)


def _ib():
    from paper_1905_00182_gb300 import ibfsa
    ibfsa.lib()
    return ibfsa


def _params():
    return np.load(os.path.join(ROOT, "paper_1905_00182_gb300", "mlp_weights.npz"))["params"]


def _perturbation_scale(spec, Q):
    from tests.test_gpu_fp32 import _perturbation_scale as ps
    return ps(spec, Q)


def _spec(dim, n):
    bc = ((0, 0), (2, 2), (2, 2) if dim == 3 else (0, 0))  # the contact is normal to x
    return W.GridSpec(dim=dim, n=n, lo=(0, 0, 0), hi=(1, 1, 1), Re=0.0,
                      qinf=W.freestream(dim, 1.4), scheme=W.MLP_TENO5,
                      precision=W.FP32_PERTURB, bc=bc)


def _gpu_rhs(ib, spec, Q, net=None, mesh=None):
    g = ib.Grid(spec)
    for a, m in enumerate(mesh or []):
        if m is not None:
            g.set_mesh(a, *m)
    if net is not None:
        ib.ibfsa_set_mlp(g.h, net.ptr)
        ib.ibfsa_mlp_stats(g.h)
    g.set_state(Q)
    L = g.rhs().cpu().numpy()
    counts = ib.ibfsa_mlp_stats(g.h) if net is not None else None
    assert g.status() == 0
    g.close()
    return L, counts


# (dim, n, variant): the x extent 90 takes the generic tiles in y, 92 and 36 the tensor-copy
# tiles; "stretched+char" stretches x (the contact inside the uniform part) and puts the
# characteristic non-reflecting rule on both x faces and the high-y face (zero-gradient low y)
CASES = [(2, (90, 70, 1), None), (2, (92, 70, 1), None), (3, (36, 30, 28), None),
         (2, (92, 70, 1), "stretched+char")]


@pytest.mark.parametrize("dim,n,variant", CASES)
def test_learned_rhs_matches_the_oracle_on_the_stress_state(dim, n, variant):
    ib = _ib()
    spec = _spec(dim, n)
    mesh = None
    if variant == "stretched+char":
        ax = W.stretched_axis(n[0], 1.0 / n[0], 1.6 / n[0], 40, 8, center=0.5)
        mesh = [(ax[2], ax[3]), None]
        CH = W.BC_CHARACTERISTIC
        spec = dataclasses.replace(spec, lo=(ax[0], 0.0, 0.0), hi=(ax[1], 1.0, 1.0),
                                   bc=((CH, CH), (0, CH), (0, 0)))
    Q = W.stress_state_torch(spec, device="cpu").numpy()
    params = _params()
    net = ib.MLP(params)
    L_ml, (used, seen) = _gpu_rhs(ib, spec, Q, net, mesh)
    L_te, _ = _gpu_rhs(ib, dataclasses.replace(spec, scheme=W.TENO5), Q, None, mesh)

    mlp = O.Learned(M.bf16(np.asarray(params, dtype=np.float32).astype(np.float64)),
                    round_act=True, floor=1e-9)
    Lo_ml = O.rhs(spec, Q, mlp=mlp, stretch=mesh)
    o_used, o_seen = O.mlp_counts()
    Lo_te = O.rhs(spec, Q, stretch=mesh)

    # the GPU evaluates the faces on its tiles' edges once for each tile (its counts include
    # them); the oracle counts each face once: compare the shares
    assert seen >= o_seen
    assert used > 0.9 * seen and o_used > 0.9 * o_seen
    assert abs(used / seen - o_used / o_seen) <= 0.005, (used, seen, o_used, o_seen)

    sc = _perturbation_scale(spec, Q)
    for c in range(spec.nv):
        D, Do = L_ml[c] - L_te[c], Lo_ml[c] - Lo_te[c]
        rms_do = np.sqrt(np.mean(Do ** 2))
        rms_dd = np.sqrt(np.mean((D - Do) ** 2))
        err = np.abs(L_ml[c] - Lo_ml[c])
        rms_err = np.sqrt(np.mean(err ** 2))
        print(f"dim {dim} comp {c}: network use {used}/{seen} (oracle {o_used}); "
              f"RMS D_oracle {rms_do:.3e}, RMS(D_gpu - D_oracle) {rms_dd:.3e} "
              f"({rms_dd / rms_do:.4f}); RMS |L_gpu - L_oracle| {rms_err:.3e} "
              f"vs 64 eps32 scale {64 * EPS32 * sc[c]:.3e}")
        assert rms_dd <= 2.0 ** -4 * rms_do, (c, rms_dd / rms_do)
        assert rms_err <= 64 * EPS32 * sc[c] + 2.0 ** -4 * rms_do, c
        # and the network's increment is not lost in the FP32 noise: the comparison discriminates
        assert rms_do > 8 * np.sqrt(np.mean((L_te[c] - Lo_te[c]) ** 2)), c
