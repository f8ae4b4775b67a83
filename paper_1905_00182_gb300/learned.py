"""Training of the learned reconstruction weights on stencils the solver itself generates.

Data: the FP32 perturbation form runs the 2D acoustic-pulse / cylinder workload, the
rotating-cylinder workload and the flexible flapping plate (coupled to its FP64 plate; the last
two at reduced resolution) and, at several times, ibfsa_mlp_sample draws
random faces, directions, components and split-flux signs where the learned form would use the
network (TENO5 keeps all three stencils, amplitude above the floor).  The target of each stencil
is the face value of the ninth-order upwind-biased reconstruction of the same split flux along
the same line (9 cells, exact for polynomials of degree 8): four orders above what five points
allow, with the same upwind bias (a central target would teach the network to remove the
scheme's dissipation, which made under-resolved runs unstable).  10 % of the stencils are held out.  Training: Adam on the tensor-core kernels of
libibfsa (ibfsa_mlp_train_step), mini-batches drawn on the GPU.  Everything runs on the GPU;
this module only sequences the calls.
"""
from __future__ import annotations

import dataclasses
import os

import numpy as np

from . import ibfsa as ib
from . import workloads as W

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mlp_weights.npz")


def _sample_run(spec, Q, X, U, dS, dt, steps, every, per_snapshot, seed, out_S, out_T, fill):
    import torch
    g = ib.Grid(dataclasses.replace(spec, precision=W.FP32_PERTURB, scheme=W.TENO5))
    g.set_state(Q)
    if X is not None:
        g.set_markers(X, U, dS)
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    cap = out_S.shape[0]
    for s in range(0, steps + 1, every):
        if fill >= cap:
            break
        if s > 0:
            g.rk3_step(dt, every)
        n_max = min(per_snapshot, cap - fill)
        ib.ibfsa_mlp_sample(g.h, n_max, seed * 1000003 + s, 8, out_S[fill:].data_ptr(),
                            out_T[fill:].data_ptr(), count.data_ptr())
        fill += min(int(count.item()), n_max)
    g.close()
    return fill


def _sample_fsi_run(w, steps, every, per_snapshot, seed, out_S, out_T, fill):
    import torch
    g = ib.Grid(dataclasses.replace(w["spec"], precision=W.FP32_PERTURB, scheme=W.TENO5))
    g.set_state(w["Q"])
    P = ib.Plate(w["plate"])
    P.set_state(w["e"], w["v"], 0.0)
    X, U, dS = P.markers()
    g.set_markers(X, U, dS)
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    cap = out_S.shape[0]
    for s in range(0, steps + 1, every):
        if fill >= cap:
            break
        if s > 0:
            ib.fsi_step(g, P, w["dt"], every)
        n_max = min(per_snapshot, cap - fill)
        ib.ibfsa_mlp_sample(g.h, n_max, seed * 1000003 + s, 8, out_S[fill:].data_ptr(),
                            out_T[fill:].data_ptr(), count.data_ptr())
        fill += min(int(count.item()), n_max)
    g.close()
    P.close()
    return fill


def generate_dataset(n_total: int, seed: int = 0):
    """n_total stencils [n, 5] and targets [n] (float32, on the GPU) from solver runs."""
    import torch
    S = torch.empty((n_total, 5), dtype=torch.float32, device="cuda")
    T = torch.empty(n_total, dtype=torch.float32, device="cuda")
    fill = 0
    half = n_total // 2
    # acoustic pulse scattered by a cylinder, two resolutions
    for n, frac in ((256, 0.5), (384, 0.5)):
        w = W.cylinder_pulse_2d(n=n, markers=160)
        target = fill + int(half * frac)
        fill = _sample_run(w["spec"], w["Q"], w["X"], w["U"], w["dS"], w["dt"], 400, 20,
                           max(1, (target - fill) // 20), seed + n, S[:target], T[:target], fill)
    # flexible plate flapping in a stream (1024 x 512 on the 4096 x 2048 workload's domain)
    w = W.flapping_plate_2d(n=(1024, 512))
    target = fill + (n_total - fill) // 2
    fill = _sample_fsi_run(w, 600, 30, max(1, (target - fill) // 20), seed + 11, S[:target],
                           T[:target], fill)
    # rotating cylinder in a Mach 0.2 stream (512^2 on [-40,40]^2 is too coarse for the body;
    # a [-10,10]^2 window keeps the wake and the spinning surface)
    w = W.rotating_cylinder_2d(n=512, markers=256)
    spec = dataclasses.replace(w["spec"], lo=(-10.0, -10.0, 0.0), hi=(10.0, 10.0, 1.0))
    h = spec.h[0]
    dt = 0.5 / ((1.0 + 0.2) / h + 1.0 / h)
    spec.alpha_pen, spec.beta_pen = W.penalty_defaults(h, dt)
    spec.sponge_sigma = 0.5 * 1.2 / h
    fill = _sample_run(spec, w["Q"], w["X"], w["U"], w["dS"], dt, 600, 30,
                       max(1, (n_total - fill) // 20), seed + 7, S, T, fill)
    return S[:fill], T[:fill]


def split(S, T, held_out=0.1, seed=0):
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    perm = torch.randperm(S.shape[0], device="cuda", generator=gen)
    n_test = int(S.shape[0] * held_out)
    te, tr = perm[:n_test], perm[n_test:]
    return (S[tr], T[tr]), (S[te], T[te])


def linear_loss(S, T):
    """held-out loss (same normalised units as the network's) of the optimal linear weights
    (0.1, 0.6, 0.3) -- what TENO5 uses wherever the network would be used"""
    import torch
    S64, T64 = S.double(), T.double()
    d = S64 - S64[:, 2:3]
    amp = d.abs().max(dim=1).values
    x = d / amp[:, None]
    q0 = (2 * x[:, 0] - 7 * x[:, 1] + 11 * x[:, 2]) / 6
    q1 = (-x[:, 1] + 5 * x[:, 2] + 2 * x[:, 3]) / 6
    q2 = (2 * x[:, 2] + 5 * x[:, 3] - x[:, 4]) / 6
    tn = (T64 - S64[:, 2]) / amp
    res = 0.1 * q0 + 0.6 * q1 + 0.3 * q2 - tn
    return float(torch.mean(res * res))


def train(S, T, steps=3000, batch=1 << 16, lr=2e-3, seed=0, log_every=0):
    import torch
    net = ib.MLP(W.mlp_init_params(seed))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    n = S.shape[0]
    for k in range(steps):
        idx = torch.randint(0, n, (batch,), device="cuda", generator=gen)
        lr_k = lr * (0.1 ** (k / steps))
        net.train_step(S[idx].contiguous(), T[idx].contiguous(), lr_k)
        if log_every and k % log_every == 0:
            print(k, net.params()[1], flush=True)
    return net


def main(n_total=1 << 23, steps=3000, out=WEIGHTS):
    (Str, Ttr), (Ste, Tte) = split(*generate_dataset(n_total))
    net = train(Str, Ttr, steps=steps)
    lin = linear_loss(Ste, Tte)
    mlp = net.eval(Ste, Tte)[2]
    params, _ = net.params()
    np.savez(out, params=params, heldout_mlp=mlp, heldout_linear=lin, n_train=Str.shape[0],
             n_test=Ste.shape[0], steps=steps)
    print(f"stencils: train {Str.shape[0]}, held out {Ste.shape[0]}; held-out loss "
          f"linear {lin:.4e}, network {mlp:.4e} (gain {lin / mlp:.2f}x)")
    return params


if __name__ == "__main__":
    main()
