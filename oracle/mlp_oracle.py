"""FP64 oracle of the learned reconstruction weights (the workload's learned-weight variant of the
fifth-order reconstruction of Sec. 2, text after Eq. 5).

TEST INFRASTRUCTURE ONLY (tests, smoke, bench baseline); shares no code with the CUDA kernels.

The network maps the normalised five-point stencil of one split-flux component to the three
non-linear weights of the third-order candidates:

  v = (f_{i-2}, ..., f_{i+2}),  amp = max_j |v_j - v_2|,  x = (v - v_2) / amp
  h1 = gelu(W1 x + b1), h2 = gelu(W2 h1 + b2), h3 = gelu(W3 h2 + b3)     (32 units each)
  omega = softmax(W4 h3 + b4)                                              (3 weights)
  face  = v_2 + amp * sum_k omega_k qhat_k,  qhat = candidates of x (which have x_2 = 0)

gelu is the tanh form 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).  Parameters are one flat
vector [W1 (32x5), b1, W2 (32x32), b2, W3 (32x32), b3, W4 (3x32), b4] of 2403 numbers, rows =
output units.  The loss of a batch is mean_b (sum_k omega_k qhat_k - that_b)^2 with the target in
the same normalised units, that = (t - v_2) / amp.  Everything here is float64; `bf16` rounds a
float64 array to the nearest bfloat16 (ties to even) for emulating the GPU's operand rounding.
"""
from __future__ import annotations

import math

import numpy as np

SIZES = [(32, 5), (32,), (32, 32), (32,), (32, 32), (32,), (3, 32), (3,)]
NPARAM = sum(int(np.prod(s)) for s in SIZES)
GELU_K = math.sqrt(2.0 / math.pi)
GELU_C = 0.044715


def unpack(theta):
    out, o = [], 0
    for s in SIZES:
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def bf16(x):
    """Round float64 values to the nearest bfloat16 (round to nearest, ties to even)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_K * (z + GELU_C * z ** 3)))


def gelu_grad(z):
    t = np.tanh(GELU_K * (z + GELU_C * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_K * (1.0 + 3.0 * GELU_C * z * z)


def normalise(v):
    """x = (v - v_2) / amp, amp = max_j |v_j - v_2| (rows of v are stencils)."""
    v = np.asarray(v, dtype=np.float64)
    d = v - v[:, 2:3]
    amp = np.max(np.abs(d), axis=1)
    return d / amp[:, None], amp


def candidates(x):
    """third-order candidate values at the face from the normalised stencil"""
    a, b, c, d, e = (x[:, j] for j in range(5))
    return np.stack([(2 * a - 7 * b + 11 * c) / 6.0, (-b + 5 * c + 2 * d) / 6.0,
                     (2 * c + 5 * d - e) / 6.0], axis=1)


def forward(theta, x, round_activations=False):
    """x: normalised stencils [B, 5].  Returns (omega [B, 3], cache)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta)
    r = bf16 if round_activations else (lambda a: a)
    a0 = r(x)
    z1 = a0 @ W1.T + b1
    h1 = gelu(z1)
    z2 = r(h1) @ W2.T + b2
    h2 = gelu(z2)
    z3 = r(h2) @ W3.T + b3
    h3 = gelu(z3)
    z4 = r(h3) @ W4.T + b4
    z4 = z4 - z4.max(axis=1, keepdims=True)
    e = np.exp(z4)
    om = e / e.sum(axis=1, keepdims=True)
    return om, (a0, z1, r(h1), z2, r(h2), z3, r(h3), om)


def face_normalised(theta, x, round_activations=False):
    om, _ = forward(theta, x, round_activations)
    return np.sum(om * candidates(x), axis=1), om


def loss_and_grad(theta, x, target_n, round_activations=False):
    """mean squared error of the normalised face value and its gradient w.r.t. theta"""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta)
    om, (a0, z1, h1, z2, h2, z3, h3, _) = forward(theta, x, round_activations)
    q = candidates(x)
    fn = np.sum(om * q, axis=1)
    B = x.shape[0]
    res = fn - target_n
    loss = np.mean(res * res)
    dfn = 2.0 * res / B
    dom = dfn[:, None] * q
    dz4 = om * (dom - np.sum(om * dom, axis=1, keepdims=True))
    gW4 = dz4.T @ h3
    gb4 = dz4.sum(0)
    dz3 = (dz4 @ W4) * gelu_grad(z3)
    gW3 = dz3.T @ h2
    gb3 = dz3.sum(0)
    dz2 = (dz3 @ W3) * gelu_grad(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * gelu_grad(z1)
    gW1 = dz1.T @ a0
    gb1 = dz1.sum(0)
    return loss, pack([gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4])
