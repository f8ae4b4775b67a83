"""GPU parity of the flexible plate (Eq. 1, ANCF; clamp of Eq. 17) and of the coupled
plate-fluid step against the FP64 CPU oracle.

The kernel and the oracle solve the same Newton systems of the implicit midpoint rule by
different methods: the kernel by block cyclic reduction over the 4 x 4 node blocks with fused
multiply-adds, the oracle by Gaussian elimination with partial pivoting in natural order, every
operation rounded on its own.  Two backward-stable solutions of one Newton step differ by a few
roundings of the residual amplified by the condition number kappa of the Newton matrix
A = M + (dt^2/4) dQ_int/de (computed here from the oracle's dense mass and tangent matrices):
per step |de| <= 64 kappa eps max|e| and |dv| <= (2/dt) of that, summed over the steps.  Marker
positions follow the plate state within the same bound; the coupled fluid state, whose markers
move by that much, within 1e-10 of its perturbation.  The fast and FP32 fluid forms are
compared with the strict GPU run within the tolerances of their arithmetic."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00182_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ib():
    from paper_1905_00182_gb300 import ibfsa
    ibfsa.lib()
    return ibfsa


def _forces(ps, seed, scale):
    r = W.splitmix64(seed, 2 * ps.n_markers)
    return scale * (r.reshape(2, ps.n_markers) - 0.5)


EPS = float(np.finfo(np.float64).eps)


def _kappa(ps, e, dt):
    """condition number of the Newton matrix M + (dt^2/4) dQ_int/de at the state e"""
    _, K, Mm = O.plate_internal(ps, e, tangent=True, mass=True)
    A = Mm + 0.25 * dt * dt * K
    if ps.clamped:  # node 0's position is prescribed: its rows and columns are not unknowns
        A = A[2:, 2:]
    return float(np.linalg.cond(A))


def _bounds(ps, e, dt, steps):
    """(|de|, |dv|) bounds between two backward-stable Newton solutions after `steps` steps"""
    de = 64.0 * _kappa(ps, e, dt) * EPS * max(1.0, float(np.max(np.abs(e)))) * steps
    return de, 2.0 * de / dt


def _close(got, want, tol):
    err = float(np.max(np.abs(np.asarray(got) - np.asarray(want))))
    return err <= tol, err


def _deformed(ps, seed=11, amp=0.05, vamp=0.5, **kw):
    r = W.splitmix64(seed, 2 * ps.ndof)
    e, v = W.plate_straight(ps, **kw)
    return e + amp * (r[: ps.ndof] - 0.5), v + vamp * (r[ps.ndof:] - 0.5)


@pytest.mark.parametrize("kind", ["free", "clamped", "flapping"])
def test_plate_steps_match_oracle(kind):
    ib = _ib()
    if kind == "free":
        ps = W.PlateSpec(n_el=10, n_markers=37, K_S=40.0, K_B=0.05, clamped=0)
        e, v = _deformed(ps, origin=(0.2, -0.1), theta=0.4)
        dt, scale = 0.01, 2.0
    elif kind == "clamped":
        ps = W.PlateSpec(n_el=17, n_markers=101, K_S=300.0, K_B=0.2, clamped=1, x0=(0.1, 0.2),
                         theta0=-0.3, A0=0.4, freq=1.3, beta=1.2, alpha_m=0.8, phi=0.5)
        e, v = W.plate_straight(ps)
        dt, scale = 0.004, 0.5
    else:
        w = W.flapping_plate_2d(n=(64, 32))
        ps, e, v = w["plate"], w["e"], w["v"]
        dt, scale = w["dt"], 1e-3
    P = ib.Plate(ps)
    P.set_state(e, v, 0.0)
    eo, vo, t = e.copy(), v.copy(), 0.0
    for n in range(12):
        F = _forces(ps, 100 + n, scale)
        P.step(dt, F)
        eb, vb = eo.copy(), vo.copy()
        t_new = t + dt
        eo, vo, _ = O.plate_step(ps, eo, vo, t_new, dt, Qf=O.plate_load(ps, F))
        t = t_new
    eg, vg, tg = P.get_state()
    flags, iters = P.status()
    assert flags == 0 and 1 <= iters <= 8
    assert tg == t
    tol_e, tol_v = _bounds(ps, e, dt, 12)
    ok_e, err_e = _close(eg.cpu().numpy(), eo, tol_e)
    ok_v, err_v = _close(vg.cpu().numpy(), vo, tol_v)
    print(f"{kind}: kappa {_kappa(ps, e, dt):.3e}, |de| {err_e:.3e} (bound {tol_e:.3e}), "
          f"|dv| {err_v:.3e} (bound {tol_v:.3e})")
    assert ok_e and ok_v
    assert np.max(np.abs(eo - e)) > 1e3 * tol_e  # the comparison resolves the motion
    X, U, dS = P.markers()
    Xo, Uo, dSo = O.plate_markers(ps, eo, vo)
    assert _close(X.cpu().numpy(), Xo, 4 * tol_e)[0] and _close(U.cpu().numpy(), Uo, 4 * tol_v)[0]
    assert np.array_equal(dS.cpu().numpy(), dSo)
    # force and power of the last step: its load and the markers' velocities before it
    fg, pg = P.force()
    _, Ub, _ = O.plate_markers(ps, eb, vb)
    fo, po = O.plate_force(ps, F, Ub)
    assert np.array_equal(fg, fo)  # the load alone: summed in marker order on both sides
    assert abs(pg - po) <= 4 * tol_v * np.sum(np.abs(F)) * ps.length / ps.n_markers
    P.close()


@pytest.mark.parametrize("n_el,nm", [(1, 1), (2, 3), (128, 3001)])
def test_plate_extreme_sizes_match_oracle(n_el, nm):
    ib = _ib()
    ps = W.PlateSpec(n_el=n_el, n_markers=nm, K_S=80.0, K_B=0.1, clamped=1, A0=0.3, freq=0.9,
                     beta=1.5, alpha_m=0.5)
    e, v = W.plate_straight(ps)
    P = ib.Plate(ps)
    P.set_state(e, v, 0.25)
    eo, vo, t = e.copy(), v.copy(), 0.25
    dt = 0.003
    for n in range(4):
        F = _forces(ps, 7 + n, 0.3)
        P.step(dt, F)
        eo, vo, _ = O.plate_step(ps, eo, vo, t + dt, dt, Qf=O.plate_load(ps, F))
        t = t + dt
    eg, vg, _ = P.get_state()
    assert P.status()[0] == 0
    tol_e, tol_v = _bounds(ps, e, dt, 4)
    assert _close(eg.cpu().numpy(), eo, tol_e)[0] and _close(vg.cpu().numpy(), vo, tol_v)[0]


def test_newton_limit_is_reported_not_faulted():
    ib = _ib()
    ps = W.PlateSpec(n_el=8, n_markers=16, K_S=100.0, K_B=0.1, clamped=0, newton_max=1,
                     newton_tol=1e-15)
    e, v = _deformed(ps, vamp=2.0)
    P = ib.Plate(ps)
    P.set_state(e, v)
    P.step(0.05)
    flags, iters = P.status()
    assert flags & ib.IBFSA_STATUS_NOCONV and iters == 1
    # the state after the capped iteration is the oracle's capped iterate: one linear solve
    eo, vo, _ = O.plate_step(ps, e, v, 0.05, 0.05, check=False)
    eg, vg, _ = P.get_state()
    tol_e, tol_v = _bounds(ps, e, 0.05, 1)
    assert _close(eg.cpu().numpy(), eo, tol_e)[0] and _close(vg.cpu().numpy(), vo, tol_v)[0]
    assert P.status() == (0, 0)  # cleared by the read


def _coupled_case(n=(96, 64), scheme=W.TENO5, precision=W.FP64):
    """Flapping clamped plate in a stream on a small grid (the 4096x2048 set-up, coarse)."""
    g = 1.4
    U0 = 0.2
    spec = W.GridSpec(dim=2, n=(n[0], n[1], 1), lo=(-3.0, -2.0, 0.0), hi=(3.0, 2.0, 1.0),
                      gamma=g, Re=500.0, qinf=W.freestream(2, g, vel=(U0, 0.0, 0.0)),
                      scheme=scheme, precision=precision, bc=((1, 1), (1, 1), (0, 0)),
                      sponge_cells=6, max_markers=60)
    h = spec.h[0]
    dt = 0.5 / ((1.0 + U0) / h + 1.0 / spec.h[1])
    spec.alpha_pen, spec.beta_pen = W.penalty_defaults(h, dt)
    spec.sponge_sigma = 0.5 * (1.0 + U0) / h
    ps = W.PlateSpec(n_el=8, n_markers=60, length=1.0, rho_s=1.0, K_S=400.0, K_B=0.05,
                     clamped=1, x0=(-0.5, 0.0), A0=0.4, freq=0.5, beta=0.5 * math.pi,
                     alpha_m=math.radians(40.0))
    e, v = W.plate_straight(ps)
    Q = W.random_smooth_state(spec, seed=5, amp=1e-3, vel0=(U0, 0.0, 0.0))
    return spec, ps, Q, e, v, dt


def _coupled_gpu(spec, ps, Q, e, v, dt, steps, strict, force=None):
    ib = _ib()
    G = ib.Grid(spec, strict=strict)
    G.set_state(Q)
    X, U, dS = O.plate_markers(ps, e, v)
    G.set_markers(X, U, dS)  # zeroes the penalty integral
    P = ib.Plate(ps)
    P.set_state(e, v, 0.0)
    ib.fsi_step(G, P, dt, steps)
    out = (G.get_state().cpu().numpy(), G.penalty_integral().cpu().numpy(),
           *[t.cpu().numpy() if hasattr(t, "cpu") else t for t in P.get_state()])
    if force is not None:
        force.append(P.force())
    flags = (G.status(), P.status())
    G.close()
    P.close()
    return out, flags


def test_coupled_step_matches_oracle():
    spec, ps, Q, e, v, dt = _coupled_case()
    steps = 3
    fl = []
    (Qg, xig, eg, vg, tg), (gs, (ps_flags, iters)) = _coupled_gpu(spec, ps, Q, e, v, dt, steps,
                                                                  strict=True, force=fl)
    xi0 = np.zeros((2, ps.n_markers))
    Q2, xi2, e2, v2, t2, _ = O.fsi_step(spec, ps, Q, xi0, e, v, 0.0, dt, nsteps=steps - 1)
    Qo, xio, eo, vo, to, it_o = O.fsi_step(spec, ps, Q2, xi2, e2, v2, t2, dt, nsteps=1)
    _, Ul, _ = O.plate_markers(ps, e2, v2)
    fo, po = O.plate_force(ps, O.fsi_last_load(ps), Ul)
    assert gs == 0 and ps_flags == 0 and iters >= max(it_o) - 1
    assert tg == to
    tol_e, tol_v = _bounds(ps, e, dt, steps)
    ok_e, err_e = _close(eg, eo, tol_e)
    ok_v, err_v = _close(vg, vo, tol_v)
    qinf = np.array(spec.qinf[:4])[:, None, None, None]
    pert = np.max(np.abs(Qo - qinf), axis=(1, 2, 3))
    errq = np.max(np.abs(Qg - Qo), axis=(1, 2, 3))
    print(f"coupled: |de| {err_e:.3e} ({tol_e:.3e}), |dv| {err_v:.3e} ({tol_v:.3e}), "
          f"|dQ|/pert {errq / pert}")
    assert ok_e and ok_v
    # the fluid sees markers that moved by ~|de|: its state within 1e-10 of its perturbation
    assert np.all(errq <= 1e-10 * pert)
    assert np.max(np.abs(xig - xio)) <= 1e-10 * np.max(np.abs(xio))
    sc = np.max(np.abs(fo))
    assert np.max(np.abs(np.asarray(fl[0][0]) - fo)) <= 1e-9 * sc
    assert abs(fl[0][1] - po) <= 1e-9 * (abs(po) + sc)
    assert np.max(np.abs(eo - e)) > 1e-3  # the plate moved


def test_coupled_step_fast_and_fp32_forms_track_strict():
    spec, ps, Q, e, v, dt = _coupled_case()
    steps = 6
    (Qs, _, es, vs, _), _ = _coupled_gpu(spec, ps, Q, e, v, dt, steps, strict=True)
    (Qf, _, ef, vf, _), (gs, (pf, _)) = _coupled_gpu(spec, ps, Q, e, v, dt, steps, strict=False)
    assert gs == 0 and pf == 0
    spec32 = W.GridSpec(**{**spec.__dict__, "precision": W.FP32_PERTURB})
    (Q3, _, e3, v3, _), (gs3, (p3, _)) = _coupled_gpu(spec32, ps, Q, e, v, dt, steps,
                                                      strict=False)
    assert gs3 == 0 and p3 == 0
    disp = np.max(np.abs(es - e))
    # fast FP64: a few roundings per operation; FP32 perturbation form: 1e-3 of the motion
    assert np.max(np.abs(ef - es)) <= 1e-10 * disp
    assert np.max(np.abs(e3 - es)) <= 1e-3 * disp
    qinf = np.array(spec.qinf[:4])[:, None, None, None]
    pert = np.max(np.abs(Qs - qinf), axis=(1, 2, 3))
    for c in range(4):
        assert np.max(np.abs(Qf[c] - Qs[c])) <= 1e-9 * pert[c]
        assert np.max(np.abs(Q3[c] - Qs[c])) <= 1e-3 * pert[c]


def test_flapping_plate_full_size_fp32_vs_fp64():
    """4096x2048 flapping plate (40 elements, 800 markers, TENO5): the FP32 perturbation form
    with the FP64 plate against the FP64 form over the same 300 coupled steps: plate motion
    and the pressure fluctuation on a ring of 360 probes at r = 1.3 around the plate (reached by
    the plate's waves) within 1e-3 relative RMS; Newton converges every step.  The flow field
    itself differs most at the plate's sharp trailing edge, where FP32 and FP64 reach different
    TENO stencil decisions: bounded in RMS, not cell by cell."""
    ib = _ib()
    w = W.flapping_plate_2d()
    ps, e, v, dt = w["plate"], w["e"], w["v"], w["dt"]
    ring = W.ring_probes(360, 1.3)
    steps = 300
    res = {}
    for prec in (W.FP64, W.FP32_PERTURB):
        spec = W.GridSpec(**{**w["spec"].__dict__, "precision": prec})
        G = ib.Grid(spec, strict=False, max_probes=ring.shape[1])
        G.set_state(w["Q"])
        X, U, dS = O.plate_markers(ps, e, v)
        G.set_markers(X, U, dS)
        P = ib.Plate(ps)
        P.set_state(e, v, 0.0)
        ib.fsi_step(G, P, dt, steps)
        eg, vg, _ = P.get_state()
        dp = G.probe(ring).cpu().numpy()
        Q = G.get_state().cpu().numpy()
        res[prec] = (eg.cpu().numpy(), dp, Q, G.status(), P.status())
        G.close()
        P.close()
    e64, dp64, Q64, gs64, (pf64, it64) = res[W.FP64]
    e32, dp32, Q32, gs32, (pf32, it32) = res[W.FP32_PERTURB]
    assert gs64 == 0 and gs32 == 0 and pf64 == 0 and pf32 == 0
    assert it64 <= 6 and it32 <= 6
    disp = np.max(np.abs(e64 - e))
    assert disp > 0.05
    assert np.max(np.abs(e32 - e64)) <= 1e-3 * disp
    rms = lambda a: float(np.sqrt(np.mean(a * a)))
    assert rms(dp64) > 1e-6  # the plate's waves reached the ring
    assert rms(dp32 - dp64) <= 1e-3 * rms(dp64)
    qinf = np.array(w["spec"].qinf[:4])
    for c in range(4):
        assert rms(Q32[c] - Q64[c]) <= 1e-2 * rms(Q64[c] - qinf[c])
