#!/usr/bin/env python
"""Throughput of the IB-WENO/TENO stage right-hand side (arXiv:1905.00182, Sec. 2) on one GB300.

Workload: 3D acoustic pulse scattered by a rigid sphere, 512^3 cells on [-8,8]^3 (h = 1/32),
sphere D = 1 with 20000 Fibonacci markers, Gaussian pulse 1e-3 / half-width 0.2 at (2,0,0),
gamma 1.4, Re 1e4, TENO5, SSP-RK3 at CFL 0.5.  One step = one SSP-RK3 step = three stage
right-hand sides (convective + viscous + penalty IB) with their RK combinations.

Metric: cell-stage updates per second (cells x 3 / step time), device-timed with CUDA events on
the library's stream, inputs resident in HBM (each state copy is 5.4 GB > 129 MB L2, so no L2
flush is needed).  Printed as one JSON line with the roofline of the measured unit (one whole
stage: 106.7 algorithmic bytes per cell against the HBM peak, its operations against the ALU
peak), each kernel class's own roofline, an end-to-end figure through the C ABI with host
buffers, the FP64 CPU oracle timed on the host cores, and the SM clocks sampled during the
timed region.

  python bench.py [--gpus N --steps K --warmup W --n 512 --scheme teno5|weno5js --strict]
  python bench.py --impl reference ...   (the FP64 CPU oracle on a bounded sample)
For N > 1 (torchrun) every rank runs an independent replica of the workload (weak scaling).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1905_00182_gb300 import workloads as W  # noqa: E402

HBM_FALLBACK_GBS = 6800.0
SMS = 152
FP64_FLOP_PER_CLK_PER_SM = 4  # 2 DFMA per SM per clock by the unit count (the pipe-rate probe
                              # measures 1.7)
FP32_FLOP_PER_CLK_PER_SM = 256  # 128 FP32 FMA lanes per SM per clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--markers", type=int, default=20000)
    ap.add_argument("--scheme", default="teno5", choices=["teno5", "weno5js"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="fp32: perturbation form (FP64 RK state, markers, probes); fp64: plain")
    ap.add_argument("--strict", action="store_true", help="strict (bit-reproducible) FP64")
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip the FP64 comparison run of the fp32 form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--form", default="teno", choices=["teno", "learned"],
                    help="learned: the timed run uses the learned weights (FP32 form)")
    ap.add_argument("--state", default="pulse", choices=["pulse", "stress"],
                    help="initial state of the timed run")
    ap.add_argument("--workload", default="sphere", choices=["sphere", "fsi"],
                    help="sphere: the 512^3 headline; fsi: only the coupled flapping-plate step "
                         "(4096x2048), e.g. for profiling")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------
# workload
# ------------------------------------------------------------------------------------------
def workload_spec(n, markers, scheme):
    L = 8.0 * n / 512.0
    spec = W.GridSpec(dim=3, n=(n, n, n), lo=(-L, -L, -L), hi=(L, L, L), gamma=1.4, Re=1e4,
                      qinf=W.freestream(3, 1.4), scheme=scheme, max_markers=markers)
    h = spec.h[0]
    dt = 0.5 / (3.0 / h)  # CFL 0.5 with alpha = c = 1 in every direction at rest
    spec.alpha_pen, spec.beta_pen = W.penalty_defaults(h, dt)
    return spec, dt


def config_dict(args, n):
    if getattr(args, "precision", "fp64") == "fp32":
        form = "FP32 perturbation form (FP64 RK state, markers, probes)"
        prec = "fp32-perturbation"
    else:
        form = f"FP64 {'strict' if args.strict else 'fused-multiply-add'}"
        prec = "fp64-strict" if args.strict else "fp64"
    if getattr(args, "form", "teno") == "learned":
        form += ", learned reconstruction weights behind the TENO5 guard"
    state = getattr(args, "state", "pulse")
    what = ("3D acoustic pulse scattered by a rigid sphere" if state == "pulse" else
            "3D stress state (smooth random modes everywhere + 10 % contact step) around a rigid sphere")
    return {
        "workload": f"{what}, {n}^3 on [-8,8]^3, "
                    f"{args.scheme.upper()}, {args.markers} markers, Re 1e4, SSP-RK3, {form}",
        "grid": [n, n, n], "scheme": args.scheme, "markers": args.markers,
        "precision": prec,
        "step": "one SSP-RK3 step = 3 stage right-hand sides + RK combinations",
        "l2": "inputs larger than L2 (5.4 GB per state copy at 512^3), no flush",
    }


# ------------------------------------------------------------------------------------------
# algorithmic work per cell-stage (counted from the formulas; divisions and square roots count
# as one operation each) -- see the per-kernel breakdown in the design notes
# ------------------------------------------------------------------------------------------
def flops_per_cell(scheme, dim=3, viscous=True):
    """Operations per cell and stage of each kernel class (3D unless dim = 2)."""
    nv = dim + 2
    # one reconstruction: candidates 16, smoothness indicators 33, non-linear weights and the
    # weighted sum (TENO5 29, WENO5-JS 19)
    recon = 16 + 33 + (29 if scheme == "teno5" else 19)
    flux = dim + 3                       # physical flux of one direction
    split = 5 * nv                       # alpha q, F +- alpha q, halves
    faces = nv * (2 * recon + 1)         # two reconstructions and their sum per component
    diff = 3 * nv                        # difference, / h, accumulate
    conv = flux + split + faces + diff
    pad = dim + (2 * dim - 1) + 3 + 3 + dim
    visc_flux = (5 * dim * dim + (dim - 1) + dim * (3 * dim + 2)) if viscous else 0
    visc_div = ((dim + 1) * (5 * dim + (dim - 1) + 2)) if viscous else 0
    finish = 5 * nv
    per = {"pad": pad, "conv_x": conv, "conv_y": conv, "conv_z": conv if dim == 3 else 0,
           "visc_flux": visc_flux, "visc_div": visc_div, "finish": finish}
    per["total"] = sum(per.values())
    return per


def bytes_per_cell(precision, dim=3, viscous=True):
    """Algorithmic DRAM bytes per cell and stage of each kernel class (averaged over the three
    stages; padded arrays counted per interior cell with their ghost overhead at 512^3)."""
    nv = dim + 2
    pad_ratio = (520 / 512) ** 3
    if precision == "fp32":
        prim = 4 * (nv + dim + 1)                     # padded q' and primitive perturbations
        inc = 4 * nv * 2 / 3                          # stage increments read in stages 2 and 3
        # 3D with viscosity: the finish pass also forms the viscous fluxes from the padded
        # velocity perturbations (read once), so no viscous-flux arrays go to DRAM
        return {"pad": 4 * nv + inc + prim * pad_ratio,
                "conv_x": prim + 4 * nv, "conv_y": prim + 8 * nv, "conv_z": prim + 8 * nv,
                "finish": 4 * nv + (4 * dim if viscous else 0) + inc +
                          (4 * nv * 2 + (8 * nv * 2 + 4 * nv)) / 3}
    prim = 8 * (nv + dim + 1)
    return {"pad": 8 * nv + prim * pad_ratio, "conv_x": prim + 8 * nv, "conv_y": prim + 16 * nv,
            "conv_z": prim + 16 * nv,
            "visc_flux": (8 * dim + 8 * dim * (dim + 1)) if viscous else 0,
            "visc_div": (8 * dim * (dim + 1) + 16 * (dim + 1)) if viscous else 0,
            "finish": 8 * nv + (8 * nv * 3 + 8 * nv * 4 + 8 * nv * 4) / 3}


def bytes_per_cell_stage(dim=3):
    # fused minimum: stage 1 reads Qn and writes Q1; stages 2, 3 read Qn and Qs, write Qo
    nv = dim + 2
    return (2 * nv * 8 + 3 * nv * 8 + 3 * nv * 8) / 3.0


def stage_roofline(bpc, cells, stage_ms, hbm_peak, peak_kind, flops, peak_tf, traffic):
    """The roofline of the measured unit, one whole stage (every launch of a right-hand side
    with its RK combination and the IB): its algorithmic bytes (bpc per cell) over the mean
    stage time against the HBM peak, and, beside it, its algorithmic operations against the
    ALU peak.  traffic: DRAM bytes of one stage from ncu (sum over its kernels), or None."""
    achieved = bpc * cells / (stage_ms * 1e-3) / 1e9
    alu = flops * cells / (stage_ms * 1e-3) / 1e12
    return {"bound": "hbm", "kernel": "whole stage (all its launches)", "achieved": achieved,
            "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
            "peak_note": f"{peak_kind} copy bandwidth", "bytes_per_cell_stage": bpc,
            "stage_ms": stage_ms, "alu_achieved_tflops": alu, "alu_peak_tflops": peak_tf,
            "alu_frac": alu / peak_tf,
            "alu_note": "algorithmic operations of the method (TENO5's non-linear weights at "
                        "every face); the FP32 and fast FP64 forms take the linear weights "
                        "where TENO5 keeps every stencil, so this rate can exceed the pipe's",
            "traffic": traffic}


def stage_traffic(classes, precision):
    """DRAM bytes of one stage at the full size: the sum over the stage's kernel classes of the
    committed ncu bytes per launch (times launches per stage), or None when a class has no
    figure taken on the current kernel source."""
    total = 0.0
    for k, v in classes.items():
        if k == "probe":
            continue
        b = ncu_traffic(k, precision)
        if b is None:
            return None
        total += b
    return total


# ------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(gpu_index)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def wait_first(self, timeout=3.0):
        """Block until the sampler has produced its first row (so the timed region is covered)."""
        t0 = time.time()
        while self.proc is not None and not self.rows and time.time() - t0 < timeout:
            time.sleep(0.02)

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(self.rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": HBM_FALLBACK_GBS}, "fallback"


def ncu_traffic(kernel_class, precision):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    name = "stage_fp32.cu" if precision == "fp32" else "stage_fp64.cuh"
    src = os.path.join(ROOT, "paper_1905_00182_gb300", "csrc", name)
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    ent = rec.get(f"{precision}:{kernel_class}")
    if not ent or ent.get("source_sha") != sha:
        return None
    return ent.get("bytes_per_launch_full")


# ------------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, as it stands, on a bounded sample of the workload
# ------------------------------------------------------------------------------------------
def oracle_sample(n_sample, steps, scheme, markers):
    from oracle import oracle as O
    L = 8.0 * n_sample / 512.0
    spec, dt = workload_spec(n_sample, markers, W.TENO5 if scheme == "teno5" else W.WENO5JS)
    Q = W.gaussian_pulse_state(spec, (min(2.0, 0.6 * L), 0.0, 0.0))
    X, U, dS = W.fibonacci_sphere(markers, 0.5)
    t0 = time.perf_counter()
    O.rk3(spec, Q, dt, steps, X, U, dS)
    el = time.perf_counter() - t0
    return spec.cells * 3 * steps / el, el


def cpu_baseline(args):
    n_s = 96
    v, el = oracle_sample(n_s, 2, args.scheme, args.markers)
    return {"value": v, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"same set-up on a {n_s}^3 grid of the same spacing (h = 1/32, "
                      f"[-1.5,1.5]^3, pulse at (0.9,0,0)), 2 SSP-RK3 steps, single thread, "
                      f"{el:.1f} s"}


def _oracle_pool_init():
    from oracle import oracle as O
    O.build()


def _oracle_pool_task(job):
    return oracle_sample(*job)


def cpu_baseline_all_cores(args):
    """The same oracle sample run concurrently in one process per host core (spawned, so no
    GPU state is inherited): the oracle as it stands, each process single-threaded, the way the
    paper's CPU code spreads one problem over a node's cores."""
    import multiprocessing as mp
    P = os.cpu_count() or 1
    n_s, steps = 96, 2
    with mp.get_context("spawn").Pool(P, initializer=_oracle_pool_init) as pool:
        pool.map(_oracle_pool_task, [(48, 1, args.scheme, 64)] * P, chunksize=1)  # all started
        t0 = time.perf_counter()
        res = pool.map(_oracle_pool_task, [(n_s, steps, args.scheme, args.markers)] * P,
                       chunksize=1)
        wall = time.perf_counter() - t0
    cells = n_s ** 3
    value = P * cells * 3 * steps / wall
    return {"value": value, "unit": "cell-updates/s", "cores": P, "kind": "oracle",
            "sample": f"{P} concurrent single-threaded processes, each the single-thread "
                      f"sample ({n_s}^3, {steps} SSP-RK3 steps); {wall:.1f} s wall, slowest "
                      f"process {max(r[1] for r in res):.1f} s"}


def run_reference(args, rank):
    if rank != 0:
        return
    n_s = 64
    vals = []
    for i in range(args.warmup + args.steps):
        v, _ = oracle_sample(n_s, 1, args.scheme, args.markers)
        if i >= args.warmup:
            vals.append(v)
    value = len(vals) / sum(1.0 / v for v in vals)
    n = args.n
    out = {"metric": "stage-RHS cell-updates/s", "value": value, "unit": "cell-updates/s",
           "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": config_dict(args, n),
           "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": 1,
                            "kind": "oracle",
                            "sample": f"each step: one SSP-RK3 step of the set-up on a {n_s}^3 "
                                      f"grid of the same spacing, single thread"},
           "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------
def make_grid(ib, args, precision, strict=False, scheme=None, state="pulse", mlp=None,
              charwise=False):
    n = args.n
    if scheme is None:
        scheme = W.TENO5 if args.scheme == "teno5" else W.WENO5JS
    spec, dt = workload_spec(n, args.markers, scheme)
    spec.precision = precision
    spec.charwise = charwise
    X, U, dS = W.fibonacci_sphere(args.markers, 0.5)
    probes, _, _ = W.fibonacci_sphere(1000, 6.0 * n / 512.0)
    g = ib.Grid(spec, strict=strict, max_probes=probes.shape[1])
    if mlp is not None:
        ib.ibfsa_set_mlp(g.h, mlp.ptr)
    if state == "pulse":
        g.set_state(W.gaussian_pulse_state_torch(spec, (2.0 * n / 512.0, 0.0, 0.0)))
    else:
        g.set_state(W.stress_state_torch(spec))
    g.set_markers(X, U, dS)
    return g, spec, dt, (X, U, dS), probes


def learned_weights(ib):
    """the committed trained parameters of the learned weights"""
    path = os.path.join(ROOT, "paper_1905_00182_gb300", "mlp_weights.npz")
    params = np.load(path)["params"]
    return ib.MLP(params)


def timed_steps(ib, g, dt, steps, barrier, profile):
    """device time (ms) of `steps` SSP-RK3 steps on the grid's stream, and the per-kernel
    profile of those steps"""
    import torch
    if profile:
        ib.ibfsa_profile_read(g.h)
        ib.ibfsa_profile_enable(g.h, True)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(g.stream)
    for _ in range(steps):
        g.rk3_step(dt, 1)
    e1.record(g.stream)
    torch.cuda.synchronize()
    barrier()
    prof = None
    if profile:
        prof = ib.ibfsa_profile_read(g.h)
        ib.ibfsa_profile_enable(g.h, False)
    return e0.elapsed_time(e1), prof


def pressure(spec, Q):
    nv = spec.nv
    ke = sum(Q[1 + a] * Q[1 + a] for a in range(spec.dim)) / Q[0]
    return (spec.gamma - 1.0) * (Q[nv - 1] - 0.5 * ke)


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest value of x over all ranks (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ms_local, units_per_rank, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: the units all ranks processed over the
    slowest rank's time.  Returns (value per second, max ms)."""
    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    ms = max_over_ranks(ms_local, dist, device)
    return units_per_rank * world / (ms * 1e-3), ms


def fsi_form(ib, barrier, max_ranks, world, warmup=3, steps=10, steps64=2):
    """The coupled plate-fluid step on the flexible flapping plate workload (4096x2048, TENO5,
    40-element FP64 plate, 800 markers): FP32 perturbation form and FP64 form, device-timed
    with the per-class split (the plate class is the structure solve plus marker and force
    bookkeeping)."""
    import torch
    w = W.flapping_plate_2d()
    out = {"workload": "flexible plate flapping in a stream, 4096x2048 on [-20,20]x[-10,10], "
                       "TENO5, Re 200, Ma 0.1, 40-element FP64 ANCF plate, 800 markers, "
                       "one coupled step = one SSP-RK3 fluid step + one plate step"}
    for prec, k in ((W.FP32_PERTURB, steps), (W.FP64, steps64)):
        spec = W.GridSpec(**{**w["spec"].__dict__, "precision": prec})
        g = ib.Grid(spec)
        g.set_state(w["Q"])
        pl = ib.Plate(w["plate"])
        pl.set_state(w["e"], w["v"], 0.0)
        X, U, dS = pl.markers()
        g.set_markers(X, U, dS)
        ib.fsi_step(g, pl, w["dt"], warmup)
        torch.cuda.synchronize()
        ib.ibfsa_profile_enable(g.h, True)
        ib.ibfsa_profile_read(g.h)
        pl.status()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(g.stream)
        ib.fsi_step(g, pl, w["dt"], k)
        e1.record(g.stream)
        torch.cuda.synchronize()
        ms = max_ranks(e0.elapsed_time(e1)) / k
        prof = ib.ibfsa_profile_read(g.h)
        flags, iters = pl.status()
        force, power = pl.force()
        Ur = w["U_ref"]  # Eq. 19: 2 F / (rho U^2 L), -2 P / (rho U^3 L), rho = L = 1
        coeff = {"C_T": -2.0 * force[0] / Ur ** 2, "C_L": 2.0 * force[1] / Ur ** 2,
                 "C_p": -2.0 * power / Ur ** 3, "t": pl.get_state()[2]}
        key = "fp32" if prec == W.FP32_PERTURB else "fp64"
        out[key] = {"value": spec.cells * 3 * world / (ms * 1e-3), "unit": "cell-updates/s",
                    "ms_per_step": ms,
                    "plate_ms_per_step": prof["plate"]["ms"] / k,
                    "kernel_ms_per_step": {c: v["ms"] / k for c, v in prof.items() if v["timed"]},
                    "newton_max_iterations": iters, "plate_status": flags,
                    "grid_status": g.status(), "coefficients_last_step": coeff}
        g.close()
        pl.close()
        del g, pl
        torch.cuda.empty_cache()
    out["fp32_speedup_vs_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1905_00182_gb300 import ibfsa as ib

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_ranks(x):
        return max_over_ranks(x, dist, "cuda")

    fp32 = args.precision == "fp32"
    prec = W.FP32_PERTURB if fp32 else W.FP64
    net = learned_weights(ib) if (fp32 and args.form == "learned") else None
    g, spec, dt, (X, U, dS), probes = make_grid(ib, args, prec, strict=args.strict and not fp32,
                                                scheme=W.MLP_TENO5 if net is not None else None,
                                                state=args.state, mlp=net)
    for _ in range(args.warmup):
        g.rk3_step(dt, 1)
    torch.cuda.synchronize()
    clocks = Clocks(local_rank)
    clocks.wait_first()
    ms, prof = timed_steps(ib, g, dt, args.steps, barrier, profile=True)
    clk = clocks.stop()
    status = g.status()
    value, ms = job_throughput(ms, spec.cells * 3 * args.steps, dist, "cuda")
    # the FP32 and FP64 forms are compared after the same 8 steps from the initial state
    steps_done = 8
    p_head = None
    if fp32 and args.compare:
        gc, _, _, _, _ = make_grid(ib, args, prec)
        gc.rk3_step(dt, steps_done)
        p_head = pressure(spec, gc.get_state())
        gc.close()
        del gc
        torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers: markers in, one step, probes out
    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(np.ascontiguousarray(X)).pin_memory()
        Uh = torch.from_numpy(np.ascontiguousarray(U)).pin_memory()
        dSh = torch.from_numpy(np.ascontiguousarray(dS)).pin_memory()
        xph = torch.from_numpy(np.ascontiguousarray(probes)).pin_memory()
        outh = torch.empty(probes.shape[1], dtype=torch.float64).pin_memory()
        k_e2e = max(1, min(args.steps, 3))
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            ib.ibfsa_set_markers(g.h, X.shape[1], Xh.data_ptr(), Uh.data_ptr(), dSh.data_ptr(), 0)
            ib.ibfsa_rk3_step(g.h, dt, 1)
            ib.ibfsa_probe(g.h, probes.shape[1], xph.data_ptr(), outh.data_ptr())  # synchronises
        el = max_ranks(time.perf_counter() - t0)
        nm = X.shape[1]
        e2e = {"value": spec.cells * 3 * k_e2e * world / el, "unit": "cell-updates/s",
               "h2d_bytes_per_step": 8 * (2 * 3 * nm + nm + 3 * probes.shape[1]),
               "d2h_bytes_per_step": 8 * probes.shape[1], "steps": k_e2e}
    gpu_launches = sum(v["launches"] for v in prof.values())
    g.close()
    del g
    torch.cuda.empty_cache()

    # the plain FP64 form on the same workload: its throughput, and the pressure-field error
    # of the FP32 form after the same number of steps from the same initial state
    compare = None
    p64_keep = None
    if fp32 and args.compare:
        g64, _, _, _, _ = make_grid(ib, args, W.FP64)
        k64 = 2
        for _ in range(steps_done - k64):
            g64.rk3_step(dt, 1)
        ms64, prof64 = timed_steps(ib, g64, dt, k64, barrier, profile=True)
        ms64 = max_ranks(ms64)
        p64 = pressure(spec, g64.get_state())
        pinf = 1.0 / spec.gamma
        err = float(torch.linalg.vector_norm(p_head - p64) / torch.linalg.vector_norm(p64 - pinf))
        p64_keep = p64
        v64 = spec.cells * 3 * k64 * world / (ms64 * 1e-3)
        compare = {"fp64_value": v64, "fp64_ms_per_step": ms64 / k64,
                   "fp32_speedup_vs_fp64": value / v64,
                   "fp32_vs_fp64_pressure_rel_l2": err, "steps_compared": steps_done,
                   "fp64_kernel_ms_per_step": {k: v["ms"] / k64 for k, v in prof64.items()
                                               if v["timed"]}}
        g64.close()
        del g64, p_head
        torch.cuda.empty_cache()

    # the learned-weight form (TENO5 fallback) on the same workload, and on the stress state
    # (perturbations everywhere) next to the FP32 TENO5 form; fallback rate = share of
    # reconstructions that used TENO5's weights
    learned = None
    if fp32 and args.compare and args.scheme == "teno5":
        net = learned_weights(ib)
        k_l = 3
        warm_l = min(args.warmup, steps_done - k_l)
        out_l = {}
        # FP64 TENO5 on the stress state, the reference of both FP32 forms there
        g64s, _, _, _, _ = make_grid(ib, args, W.FP64, state="stress")
        g64s.rk3_step(dt, steps_done)
        p64s = pressure(spec, g64s.get_state())
        g64s.close()
        del g64s
        torch.cuda.empty_cache()

        def rel_to(p, p_ref):
            return float(torch.linalg.vector_norm(p - p_ref) /
                         torch.linalg.vector_norm(p_ref - 1.0 / spec.gamma))

        ref = {"pulse": p64_keep, "stress": p64s}
        for state in ("pulse", "stress"):
            gl, _, _, _, _ = make_grid(ib, args, W.FP32_PERTURB, scheme=W.MLP_TENO5,
                                       state=state, mlp=net)
            for _ in range(warm_l):
                gl.rk3_step(dt, 1)
            ib.ibfsa_mlp_stats(gl.h)
            msl, _ = timed_steps(ib, gl, dt, k_l, barrier, profile=False)
            used, seen = ib.ibfsa_mlp_stats(gl.h)
            out_l[state] = {"value": spec.cells * 3 * k_l * world / (max_ranks(msl) * 1e-3),
                            "ms_per_step": msl / k_l,
                            "fallback_rate": 1.0 - used / max(seen, 1)}
            gl.rk3_step(dt, steps_done - warm_l - k_l)
            p_l = pressure(spec, gl.get_state())
            if ref[state] is not None:
                e = rel_to(p_l, ref[state])
                out_l[state]["vs_fp64_pressure_rel_l2"] = e
                out_l[state]["within_1e-3_of_fp64"] = bool(e <= 1e-3)
            del p_l
            gl.close()
            del gl
            torch.cuda.empty_cache()
        gs, _, _, _, _ = make_grid(ib, args, W.FP32_PERTURB, state="stress")
        for _ in range(warm_l):
            gs.rk3_step(dt, 1)
        mss, _ = timed_steps(ib, gs, dt, k_l, barrier, profile=False)
        gs.rk3_step(dt, steps_done - warm_l - k_l)
        e_fp32_stress = rel_to(pressure(spec, gs.get_state()), p64s)
        gs.close()
        del gs, p64s
        torch.cuda.empty_cache()
        learned = {"pulse": out_l["pulse"], "stress": out_l["stress"],
                   "fp32_teno5_stress_value": spec.cells * 3 * k_l * world /
                   (max_ranks(mss) * 1e-3),
                   "fp32_teno5_stress_vs_fp64_pressure_rel_l2": e_fp32_stress,
                   "steps_compared": steps_done,
                   "weights": "paper_1905_00182_gb300/mlp_weights.npz"}

    # the characteristic-wise option in the FP32 perturbation form on the same workload
    charwise = None
    if fp32 and args.compare:
        gcw, _, _, _, _ = make_grid(ib, args, W.FP32_PERTURB, charwise=True)
        gcw.rk3_step(dt, 1)
        msc, _ = timed_steps(ib, gcw, dt, 2, barrier, profile=False)
        charwise = {"value": spec.cells * 3 * 2 * world / (max_ranks(msc) * 1e-3),
                    "ms_per_step": msc / 2, "steps": 2,
                    "vs_componentwise_fp32": (spec.cells * 3 * 2 / (msc * 1e-3)) / value}
        gcw.close()
        del gcw
        torch.cuda.empty_cache()

    fsi = fsi_form(ib, barrier, max_ranks, world) if (fp32 and args.compare) else None

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks, peak_kind = measured_peaks()
    fl = flops_per_cell(args.scheme)
    fl["finish"] = fl["finish"] + (fl["visc_div"] if fp32 else 0)  # FP32 finish fuses the divergence
    by = bytes_per_cell(args.precision)
    sm_mhz = clk["sm_mhz"] or 2070.0
    if fp32:
        peak_tf = FP32_FLOP_PER_CLK_PER_SM * SMS * sm_mhz * 1e6 / 1e12
        note = "FP32 pipe: 256 flop/clk/SM (128 FMA lanes) x 152 SMs x median SM clock of the run"
    else:
        peak_tf = FP64_FLOP_PER_CLK_PER_SM * SMS * sm_mhz * 1e6 / 1e12
        note = "FP64 pipe: 4 flop/clk/SM x 152 SMs x median SM clock of the run"
    hbm_peak = peaks.get("hbm_gbs", HBM_FALLBACK_GBS)

    def kernel_roofline(k):
        v = prof[k]
        avg_ms = v["ms"] / v["timed"]
        f_tf = fl.get(k, 0.0) * spec.cells / (avg_ms * 1e-3) / 1e12
        b_gbs = by.get(k, 0.0) * spec.cells / (avg_ms * 1e-3) / 1e9
        # the binding resource is the one the kernel's algorithmic work fills the most
        if f_tf / peak_tf >= b_gbs / hbm_peak:
            return {"bound": "alu", "kernel": k, "achieved": f_tf, "peak": peak_tf,
                    "unit": "TFLOP/s", "frac": f_tf / peak_tf, "peak_note": note,
                    "flops_per_cell": fl.get(k, 0.0), "avg_launch_ms": avg_ms}
        return {"bound": "hbm", "kernel": k, "achieved": b_gbs, "peak": hbm_peak,
                "unit": "GB/s", "frac": b_gbs / hbm_peak, "peak_note": f"{peak_kind} copy bandwidth",
                "bytes_per_cell": by.get(k, 0.0), "avg_launch_ms": avg_ms}

    classes = {k: v for k, v in prof.items() if v["timed"] > 0}
    dom = max(classes, key=lambda k: classes[k]["ms"])
    dominant = kernel_roofline(dom)
    dominant["traffic"] = ncu_traffic(dom, args.precision)
    kernel_rooflines = {k: {kk: kernel_roofline(k)[kk] for kk in ("bound", "frac", "avg_launch_ms")}
                        for k in classes if k in fl or k in by}
    kernel_rooflines["dominant"] = dominant
    stage_ms = ms / world / (3 * args.steps)
    bpc = bytes_per_cell_stage()
    roofline = stage_roofline(bpc, spec.cells, stage_ms, hbm_peak, peak_kind,
                              fl["total"], peak_tf, stage_traffic(classes, args.precision))
    out = {
        "metric": "stage-RHS cell-updates/s", "value": value, "unit": "cell-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if fp32 else "f64", "data": "synthetic",
        "config": config_dict(args, args.n),
        "roofline": roofline,
        "kernel_ms_per_step": {k: v["ms"] / args.steps for k, v in prof.items() if v["timed"]},
        "kernel_rooflines": kernel_rooflines,
        "flops_per_cell_stage": fl["total"],
        "clocks": clk, "gpu_launches": gpu_launches, "device_status": status,
    }
    if compare is not None:
        out["forms"] = compare
        if learned is not None:
            out["forms"]["learned"] = learned
        if fsi is not None:
            out["forms"]["fsi"] = fsi
        if charwise is not None:
            out["forms"]["charwise_fp32"] = charwise
    if e2e is not None:
        out["e2e"] = e2e
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(args)
        out["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args)
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_fsi_only(args, rank, world, local_rank):
    """The coupled flapping-plate step alone (one JSON line from rank 0)."""
    import torch
    from paper_1905_00182_gb300 import ibfsa as ib
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    barrier = (lambda: dist.barrier()) if dist is not None else (lambda: None)
    r = fsi_form(ib, barrier, lambda x: max_over_ranks(x, dist, "cuda"), world,
                 warmup=args.warmup, steps=args.steps, steps64=min(2, args.steps))
    if rank == 0:
        print(json.dumps({"metric": "coupled plate-fluid step cell-updates/s",
                          "value": r["fp32"]["value"], "unit": "cell-updates/s",
                          "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "higher_is_better": True, "scaling": "weak", "dtype": "f32",
                          "data": "synthetic", "config": {"workload": r["workload"]},
                          "fsi": r}), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "fsi":
        run_fsi_only(args, rank, world, local_rank)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
