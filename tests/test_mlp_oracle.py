"""Pins of the FP64 oracle of the learned reconstruction weights."""

import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_1905_00182_gb300 import workloads as W


def _stencils(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 5)) * 0.3 + np.cumsum(rng.standard_normal((n, 5)), axis=1)
    return v


def test_parameter_count_and_layout():
    assert M.NPARAM == 2403 == W.MLP_NPARAM
    theta = np.arange(M.NPARAM, dtype=np.float64)
    parts = M.unpack(theta)
    assert [p.shape for p in parts] == [tuple(s) for s in M.SIZES]
    np.testing.assert_array_equal(M.pack(parts), theta)


def test_gelu_identities():
    x = np.linspace(-6, 6, 1001)
    np.testing.assert_allclose(M.gelu(x) - M.gelu(-x), x, atol=1e-14)  # x Phi(x) symmetry
    assert M.gelu(np.array([0.0]))[0] == 0.0
    h = 1e-6
    np.testing.assert_allclose(M.gelu_grad(x), (M.gelu(x + h) - M.gelu(x - h)) / (2 * h),
                               rtol=1e-7, atol=1e-9)


def test_bf16_rounding():
    cases = {1.0: 1.0, 1.0 + 2 ** -8: 1.0, 1.0 + 3 * 2 ** -8: 1.0 + 2 ** -6,
             1.0 + 2 ** -7: 1.0 + 2 ** -7, -2.5: -2.5, 1.0 + 2 ** -9: 1.0}
    for x, want in cases.items():
        assert M.bf16(np.array([x]))[0] == want, x


def test_softmax_weights_are_convex():
    theta = W.mlp_init_params(3).astype(np.float64)
    x, _ = M.normalise(_stencils(200, 1))
    om, _ = M.forward(theta, x)
    assert np.all(om > 0)
    np.testing.assert_allclose(om.sum(1), 1.0, atol=1e-15)


def test_linear_data_reconstructed_exactly_by_any_parameters():
    # linear stencils: all three candidates equal the exact face value, so any convex weights do
    theta = W.mlp_init_params(4).astype(np.float64) * 3.0
    v = np.array([[1, 2, 3, 4, 5], [3, 1, -1, -3, -5], [0.5, 0.75, 1.0, 1.25, 1.5]], float)
    x, amp = M.normalise(v)
    fn, _ = M.face_normalised(theta, x)
    face = v[:, 2] + amp * fn
    np.testing.assert_allclose(face, (v[:, 2] + v[:, 3]) / 2, atol=1e-14)


def test_untrained_network_starts_near_linear_weights():
    theta = W.mlp_init_params(0).astype(np.float64)
    x, _ = M.normalise(_stencils(500, 2))
    om, _ = M.forward(theta, x)
    assert np.max(np.abs(om - np.array([0.1, 0.6, 0.3]))) < 0.1


@pytest.mark.parametrize("round_act", [False, True])
def test_gradient_matches_central_differences(round_act):
    rng = np.random.default_rng(5)
    theta = W.mlp_init_params(1).astype(np.float64) + 0.05 * rng.standard_normal(M.NPARAM)
    x, _ = M.normalise(_stencils(64, 6))
    t = rng.standard_normal(64) * 0.3
    loss, g = M.loss_and_grad(theta, x, t, round_act)
    idx = rng.choice(M.NPARAM, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(M.NPARAM)
        e[i] = h
        if round_act:
            # activations are rounded to bfloat16: the loss is piecewise smooth, so compare
            # the analytic gradient of the rounded network with its own definition instead
            continue
        lp, _ = M.loss_and_grad(theta + e, x, t)
        lm, _ = M.loss_and_grad(theta - e, x, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])
    assert np.isfinite(loss) and np.all(np.isfinite(g))
