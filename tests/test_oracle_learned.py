"""Pins of the oracle's learned reconstruction weights (the learned-weight variant of the
fifth-order reconstruction of Sec. 2, text after Eq. 5): TENO5's cut-off decides where the data
is smooth; there the network's softmax weights combine the three third-order candidates of the
normalised stencil, and the face value is taken in delta form v_2 + amp sum_k w_k qhat_k.

What fixes the result independently of the oracle's own code:
* the network in C agrees with the numpy network of oracle/mlp_oracle.py (itself pinned by
  finite differences, gelu symmetry, bfloat16 rounding and softmax convexity), with and without
  the bfloat16 rounding of activations;
* any convex combination of the candidates is exact on cell averages of a quadratic, so the
  learned face value is too, for ANY parameters (a wrong candidate, a lost amplitude or a lost
  v_2 breaks it);
* a network whose output layer is zero with biases ln(1/10), ln(6/10), ln(3/10) gives the
  optimal linear weights, so the learned form reproduces TENO5 wherever TENO5 keeps all three
  stencils (a permuted or mis-ordered weight breaks it), on single stencils and on whole
  right-hand sides;
* the guard: where TENO5 cuts a stencil, or the stencil is flat, the result is TENO5's, bit for
  bit; a free stream gives a right-hand side of exactly zero.
"""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import mlp_oracle as M  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_1905_00182_gb300 import workloads as W  # noqa: E402


def _params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for s in M.SIZES:
        fan_in = s[1] if len(s) == 2 else 8
        parts.append(rng.normal(0.0, scale / math.sqrt(fan_in), size=s))
    return M.pack(parts)


def _linear_weight_params():
    """zero output layer, biases ln(d_k): softmax gives the optimal weights 0.1, 0.6, 0.3"""
    parts = [np.zeros(s) for s in M.SIZES]
    parts[7] = np.log(np.array([0.1, 0.6, 0.3]))
    rng = np.random.default_rng(5)
    for i in range(6):  # hidden layers arbitrary: the output layer ignores them
        parts[i] = rng.normal(0.0, 0.5, size=M.SIZES[i])
    return M.pack(parts)


@pytest.mark.parametrize("round_act", [False, True])
def test_c_network_matches_the_numpy_network(round_act):
    rng = np.random.default_rng(1)
    x = rng.uniform(-1.0, 1.0, size=(200, 5))
    x[:, 2] = 0.0
    for seed in (2, 3):
        th = _params(seed, scale=1.5)
        if round_act:
            th = M.bf16(th)
        want, _ = M.forward(th, x, round_activations=round_act)
        got = O.mlp_weights(th, x, round_act=round_act)
        assert np.max(np.abs(got - want)) <= 1e-12
        assert np.allclose(got.sum(axis=1), 1.0, atol=1e-15)


def test_learned_face_is_exact_on_quadratics_for_any_parameters():
    rng = np.random.default_rng(7)
    t = np.arange(-2, 3, dtype=np.float64)  # cells [t - 1/2, t + 1/2]; the face at t = 1/2
    n_used = 0
    for seed in range(6):
        mlp = O.Learned(M.bf16(_params(100 + seed, scale=3.0)), round_act=True, floor=0.0)
        for _ in range(40):
            a, b, c = rng.normal(size=3)
            c *= 0.1  # gentle curvature: TENO5 keeps all stencils and the network runs
            v = a + b * t + c * (t * t + 1.0 / 12.0)   # cell averages of a + b x + c x^2
            face, used = O.learned_recon(mlp, v[None, :])
            want = a + 0.5 * b + 0.25 * c
            assert abs(face[0] - want) <= 1e-13 * (abs(a) + abs(b) + abs(c)), (seed, a, b, c)
            n_used += int(used[0])
    assert n_used > 200  # the network supplied the weights in (nearly) every case


def test_linear_weight_network_reproduces_teno5_where_it_keeps_all_stencils():
    mlp = O.Learned(_linear_weight_params(), round_act=True, floor=0.0)
    rng = np.random.default_rng(11)
    v = np.cumsum(rng.normal(size=(300, 5)) * 0.1, axis=1) + rng.normal(size=(300, 1))
    face, used = O.learned_recon(mlp, v)
    teno = np.array([O.teno5(row) for row in v])
    scale = np.max(np.abs(v - v[:, 2:3]), axis=1)
    assert np.all(np.abs(face - teno) <= 1e-14 * (scale + np.abs(v[:, 2])))
    assert used.sum() > 100


def test_guard_falls_back_to_teno5_bit_for_bit():
    mlp = O.Learned(M.bf16(_params(9, scale=2.0)), round_act=True, floor=1e-9)
    cases = [
        [0.0, 0.0, 0.0, 1.0, 1.0],          # a jump: TENO5 cuts the downwind stencils
        [1.0, 1.0, 1.0, 0.0, 0.0],
        [0.0, 0.0, 1.0, 1.0, 1.0],
        [2.5, 2.5, 2.5, 2.5, 2.5],          # flat: amplitude 0
        [1.0, 1.0 + 1e-12, 1.0, 1.0, 1.0 - 3e-13],   # amplitude below the floor
    ]
    for v in cases:
        face, used = O.learned_recon(mlp, np.array([v]))
        assert not used[0], v
        assert face[0] == O.teno5(v), v
    # a smooth stencil above the floor does use the network
    face, used = O.learned_recon(mlp, np.array([[0.0, 0.1, 0.2, 0.3, 0.4]]))
    assert used[0]


def _smooth_spec(dim, n):
    return W.GridSpec(dim=dim, n=(n, n, n if dim == 3 else 1), lo=(0, 0, 0), hi=(1, 1, 1),
                      Re=0.0, qinf=W.freestream(dim, 1.4, vel=(0.2, -0.1, 0.05)),
                      scheme=W.TENO5, bc=((2, 2), (2, 2), (2, 2) if dim == 3 else (0, 0)))


@pytest.mark.parametrize("dim,n", [(2, 32), (3, 12)])
def test_free_stream_gives_exactly_zero(dim, n):
    spec = _smooth_spec(dim, n)
    Q = W.rest_state(spec)
    mlp = O.Learned(M.bf16(_params(4)), round_act=True)
    L = O.rhs(spec, Q, mlp=mlp)
    assert np.all(L == 0.0)


@pytest.mark.parametrize("dim,n", [(2, 40), (3, 14)])
def test_linear_weight_network_rhs_equals_teno5_rhs(dim, n):
    spec = _smooth_spec(dim, n)
    Q = W.random_smooth_state(spec, seed=3, amp=1e-2, vel0=(0.2, -0.1, 0.05), periodic=True)
    L_teno = O.rhs(spec, Q)
    mlp = O.Learned(_linear_weight_params(), round_act=True, floor=1e-9)
    L_ml = O.rhs(spec, Q, mlp=mlp)
    used, seen = O.mlp_counts()
    assert seen == 2 * spec.nv * sum(
        (spec.n[a] + 1) * spec.cells // spec.n[a] for a in range(dim))
    assert used > 0.9 * seen
    for c in range(spec.nv):
        scale = np.max(np.abs(Q[c])) * 3.0 / min(spec.h[:dim])
        assert np.max(np.abs(L_ml[c] - L_teno[c])) <= 64 * np.finfo(float).eps * scale, c


def test_learned_rhs_differs_from_teno5_with_a_trained_network():
    """the committed trained weights do change the right-hand side where they are used, and
    leave it TENO5's where they are not (the contact step)"""
    p = np.load(os.path.join(ROOT, "paper_1905_00182_gb300", "mlp_weights.npz"))["params"]
    mlp = O.Learned(M.bf16(np.asarray(p, dtype=np.float64)), round_act=True)
    spec = W.GridSpec(dim=2, n=(48, 48, 1), lo=(0, 0, 0), hi=(1, 1, 1), Re=0.0,
                      qinf=W.freestream(2, 1.4), scheme=W.TENO5, precision=W.FP32_PERTURB,
                      bc=((2, 2), (2, 2), (0, 0)))
    Q = W.stress_state_torch(spec, device="cpu").numpy()
    L_teno = O.rhs(spec, Q)
    L_ml = O.rhs(spec, Q, mlp=mlp)
    used, seen = O.mlp_counts()
    assert 0.8 * seen < used < seen
    d = L_ml - L_teno
    # away from the contact (x in [0.42, 0.58]) and the walls the modes are resolved by 16 or
    # more cells per wavelength, where the trained weights stay close to the linear ones: the
    # network moves the right-hand side there by a few 1e-4 of itself
    keep = np.ones(48, dtype=bool)
    keep[20:28] = False
    keep[:4] = False
    keep[-4:] = False
    for c in range(spec.nv):
        rel = np.linalg.norm(d[c][..., keep]) / np.linalg.norm(L_teno[c][..., keep])
        assert 1e-4 < rel < 1e-2, (c, rel)
