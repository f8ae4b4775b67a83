"""Tensor-core MLP kernels of the learned reconstruction weights against the FP64 oracle.

Forward: weights and face values against the oracle evaluated with the same bfloat16-rounded
parameters and bfloat16-rounded activations (the GPU's operand rounding), and against the
unrounded FP64 network.  Backward: the gradient of the batch loss per parameter tensor, relative
L2 error <= 2e-2 and cosine >= 0.999 against the oracle's FP64 gradient.  Training: Adam on the
GPU lowers the loss on smooth synthetic stencils with exact targets.
"""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_1905_00182_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ib():
    from paper_1905_00182_gb300 import ibfsa
    ibfsa.lib()
    return ibfsa


def smooth_stencils(n, seed, kmax=1.2):
    """Stencils of f(x) = A sin(k x + phi) + B sin(k2 x + phi2) + C at unit spacing, and the
    exact face value of the flux-reconstruction target: the function h whose cell averages are
    f, at x = 1/2 -- for a mode of wavenumber k, h = f (k/2)/sin(k/2)."""
    rng = np.random.default_rng(seed)
    k1 = rng.uniform(0.05, kmax, n)
    k2 = rng.uniform(0.05, kmax, n)
    A = rng.uniform(0.2, 1.0, n)
    B = rng.uniform(0.0, 0.5, n)
    C = rng.uniform(-1, 1, n)
    p1 = rng.uniform(0, 2 * math.pi, n)
    p2 = rng.uniform(0, 2 * math.pi, n)
    j = np.arange(-2, 3)[None, :]
    S = (A[:, None] * np.sin(k1[:, None] * j + p1[:, None]) +
         B[:, None] * np.sin(k2[:, None] * j + p2[:, None]) + C[:, None])
    g1 = (k1 / 2) / np.sin(k1 / 2)
    g2 = (k2 / 2) / np.sin(k2 / 2)
    T = A * g1 * np.sin(k1 * 0.5 + p1) + B * g2 * np.sin(k2 * 0.5 + p2) + C
    return S.astype(np.float32), T.astype(np.float32)


def _theta(seed):
    th = W.mlp_init_params(seed).astype(np.float64)
    th += 0.2 * np.random.default_rng(seed + 100).standard_normal(th.size)
    return th


def test_forward_matches_oracle():
    ib = _ib()
    th = _theta(1)
    S, T = smooth_stencils(4099, 2)  # ragged: not a multiple of the 16-row tile
    net = ib.MLP(th.astype(np.float32))
    face, omega, _ = net.eval(torch.from_numpy(S).cuda())
    face, omega = face.cpu().numpy(), omega.cpu().numpy()
    thb = M.bf16(th.astype(np.float32))
    x, amp = M.normalise(S.astype(np.float64))
    fn_r, om_r = M.face_normalised(thb, x, round_activations=True)
    fn_f, om_f = M.face_normalised(thb, x, round_activations=False)
    assert np.max(np.abs(omega - om_r)) <= 8e-3, np.max(np.abs(omega - om_r))
    assert np.sqrt(np.mean((omega - om_r) ** 2)) <= 1e-3
    assert np.max(np.abs(omega - om_f)) <= 2e-2
    want = S[:, 2].astype(np.float64) + amp * fn_r
    assert np.max(np.abs(face - want) / (amp + 1e-30)) <= 1e-2


def test_gradient_matches_oracle():
    ib = _ib()
    th = _theta(3)
    S, T = smooth_stencils(2048, 4)
    net = ib.MLP(th.astype(np.float32))
    loss, g = net.gradient(torch.from_numpy(S).cuda(), torch.from_numpy(T).cuda())
    thb = M.bf16(th.astype(np.float32))
    x, amp = M.normalise(S.astype(np.float64))
    tn = (T.astype(np.float64) - S[:, 2]) / amp
    lo, go = M.loss_and_grad(thb, x, tn, round_activations=True)
    assert abs(loss - lo) <= 2e-2 * lo, (loss, lo)
    parts_g, parts_o = M.unpack(g.astype(np.float64)), M.unpack(go)
    for k, (a, b) in enumerate(zip(parts_g, parts_o)):
        a, b = a.ravel(), b.ravel()
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        assert rel <= 2e-2 and cos >= 0.999, (k, rel, cos)


def test_adam_training_lowers_the_loss():
    ib = _ib()
    S, T = smooth_stencils(1 << 16, 5, kmax=1.6)
    Sd, Td = torch.from_numpy(S).cuda(), torch.from_numpy(T).cuda()
    net = ib.MLP(W.mlp_init_params(0))
    _, _, l0 = net.eval(Sd, Td)
    for _ in range(300):
        net.train_step(Sd, Td, 2e-3)
    _, _, l1 = net.eval(Sd, Td)
    assert l1 < 0.5 * l0, (l0, l1)
