"""ctypes binding of the plain FP64 CPU oracle (oracle/ibfsa_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and by the bench's
CPU-baseline leg, never by the product path.  It shares no code with the CUDA library; both
read the same GridSpec (a plain description of the problem) and marshal it into their own
structs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ibfsa_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "plate_oracle.c"), os.path.join(_HERE, "ibfsa_oracle.h")]
_LIB = os.path.join(_HERE, "libibfsa_oracle.so")

ORC_OK = 0
ORC_ERR_ARG = -1
ORC_ERR_BOUNDS = -4


def build(force: bool = False) -> str:
    """Compile the oracle (fluid stage and plate) with plain gcc: -O2, no fused multiply-add
    contraction."""
    newest = max(os.path.getmtime(f) for f in _SRCS)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
               "-o", _LIB, *[f for f in _SRCS if f.endswith(".c")], "-lm"]
        subprocess.check_call(cmd)
    return _LIB


class OrcDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("gamma", ctypes.c_double),
        ("Re", ctypes.c_double),
        ("qinf", ctypes.c_double * 5),
        ("scheme", ctypes.c_int),
        ("bc", (ctypes.c_int * 2) * 3),
        ("sponge_cells", ctypes.c_int),
        ("sponge_sigma", ctypes.c_double),
        ("alpha_pen", ctypes.c_double),
        ("beta_pen", ctypes.c_double),
        ("src_amp", ctypes.c_double),
        ("src_b", ctypes.c_double),
        ("src_omega", ctypes.c_double),
        ("src_xc", ctypes.c_double * 3),
        ("time", ctypes.c_double),
        ("charwise", ctypes.c_int),
        ("xnode", ctypes.POINTER(ctypes.c_double) * 3),
        ("xmetric", ctypes.POINTER(ctypes.c_double) * 3),
        ("mlp_params", ctypes.POINTER(ctypes.c_double)),
        ("mlp_round", ctypes.c_int),
        ("mlp_floor", ctypes.c_double),
    ]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.orc_lambda.restype = ctypes.c_double
        _lib.orc_lambda.argtypes = [ctypes.c_double]
        for f in ("orc_weno5js", "orc_teno5"):
            getattr(_lib, f).restype = ctypes.c_double
            getattr(_lib, f).argtypes = [_D]
        _lib.orc_rhs.argtypes = [ctypes.POINTER(OrcDesc), _D, ctypes.c_int, _D, _D, _D, _D, _D, _D,
                                 _D, _D]
        _lib.orc_rhs_given_alpha.argtypes = [ctypes.POINTER(OrcDesc), _D, ctypes.c_int, _D, _D,
                                             _D, _D, _D, _D]
        _lib.orc_rk3.argtypes = [ctypes.POINTER(OrcDesc), _D, ctypes.c_int, _D, _D, _D, _D,
                                 ctypes.c_double, ctypes.c_int]
        _lib.orc_probe.argtypes = [ctypes.POINTER(OrcDesc), _D, ctypes.c_int, _D, _D]
        _lib.orc_wavespeeds.argtypes = [ctypes.POINTER(OrcDesc), _D, _D]
        _lib.orc_interp_scalar.argtypes = [ctypes.POINTER(OrcDesc), _D, ctypes.c_int, _D, _D]
        _lib.orc_spread_scalar.argtypes = [ctypes.POINTER(OrcDesc), ctypes.c_int, _D, _D, _D, _D]
        _lib.orc_mlp_weights.restype = None
        _lib.orc_mlp_weights.argtypes = [_D, ctypes.c_int, _D, _D]
        _lib.orc_learned_recon.restype = ctypes.c_double
        _lib.orc_learned_recon.argtypes = [_D, ctypes.c_int, ctypes.c_double, _D,
                                           ctypes.POINTER(ctypes.c_int)]
        _lib.orc_mlp_counts.restype = None
        _lib.orc_mlp_counts.argtypes = [ctypes.POINTER(ctypes.c_longlong)] * 2
    return _lib


class Learned:
    """The learned reconstruction weights as the oracle evaluates them: the 2403 parameters used
    as given (pass the bfloat16-rounded values the tensor cores see), the network's input and
    hidden activations rounded to bfloat16 when round_act, and the guard's amplitude floor."""

    def __init__(self, params, round_act: bool = True, floor: float = 1e-9):
        self.params = np.ascontiguousarray(params, dtype=np.float64)
        if self.params.shape != (2403,):
            raise ValueError("the network has 2403 parameters")
        self.round_act = bool(round_act)
        self.floor = float(floor)


def desc(spec, t: float = 0.0, charwise: bool = False, stretch=None, mlp=None) -> OrcDesc:
    """The oracle's descriptor.  stretch: None (uniform) or, per direction, None or a pair
    (x nodes, dx/dxi at the nodes) over the padded range i = -4 .. n+3.  mlp: a Learned (the
    learned-weight scheme), else the spec's WENO5-JS or TENO5 (TENO5 for the learned scheme:
    its end-to-end oracle)."""
    d = OrcDesc()
    d.dim = spec.dim
    for a in range(3):
        d.n[a] = int(spec.n[a])
        d.lo[a] = float(spec.lo[a])
        d.hi[a] = float(spec.hi[a])
        d.bc[a][0] = int(spec.bc[a][0])
        d.bc[a][1] = int(spec.bc[a][1])
    d.gamma = spec.gamma
    d.Re = spec.Re
    for c in range(5):
        d.qinf[c] = float(spec.qinf[c])
    d.scheme = 1 if spec.scheme != 0 else 0  # the learned variant's end-to-end oracle is TENO5
    d.sponge_cells = spec.sponge_cells
    d.sponge_sigma = spec.sponge_sigma
    d.alpha_pen = spec.alpha_pen
    d.beta_pen = spec.beta_pen
    d.src_amp = float(spec.src_amp)
    d.src_b = float(spec.src_b)
    d.src_omega = float(spec.src_omega)
    for a in range(3):
        d.src_xc[a] = float(spec.src_xc[a])
    d.time = float(t)
    d.charwise = 1 if (charwise or getattr(spec, "charwise", False)) else 0
    d._keep = []
    if mlp is not None:
        d.scheme = 2
        d._keep.append(mlp.params)
        d.mlp_params = mlp.params.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.mlp_round = 1 if mlp.round_act else 0
        d.mlp_floor = mlp.floor
    if stretch is not None:
        for a, pair in enumerate(stretch):
            if pair is None or a >= spec.dim:
                continue
            xn, xm = (np.ascontiguousarray(v, dtype=np.float64) for v in pair)
            if xn.shape != (spec.n[a] + 8,) or xm.shape != (spec.n[a] + 8,):
                raise ValueError(f"direction {a}: node and metric arrays need n + 8 entries")
            d._keep += [xn, xm]
            d.xnode[a] = xn.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            d.xmetric[a] = xm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return d


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def lam(r: float) -> float:
    return lib().orc_lambda(float(r))


def weno5js(v) -> float:
    v = _f64(np.asarray(v))
    return lib().orc_weno5js(_p(v))


def teno5(v) -> float:
    v = _f64(np.asarray(v))
    return lib().orc_teno5(_p(v))


def _markers(spec, X, U, dS, xi):
    if X is None:
        return 0, None, None, None, None
    X = _f64(X)
    nm = X.shape[1]
    U = _f64(U) if U is not None else np.zeros_like(X)
    dS = _f64(dS)
    xi = _f64(xi) if xi is not None else np.zeros_like(X)
    return nm, X, U, dS, xi


def rhs(spec, Q, X=None, U=None, dS=None, xi=None, return_markers=False, t=0.0, charwise=False,
        stretch=None, mlp=None):
    """RHS L(Q) + S of every interior cell at time t, shape [nv][nz][ny][nx] (charwise: the
    characteristic-wise reconstruction; mlp: a Learned, the learned-weight scheme)."""
    Q = _f64(Q)
    nm, X, U, dS, xi = _markers(spec, X, U, dS, xi)
    L = np.zeros_like(Q)
    F = np.zeros((spec.dim, max(nm, 1)))
    rate = np.zeros((spec.dim, max(nm, 1)))
    alpha = np.zeros(3)
    d = desc(spec, t, charwise, stretch, mlp)
    rc = lib().orc_rhs(ctypes.byref(d), _p(Q), nm, _p(X), _p(U), _p(dS), _p(xi), _p(L), _p(F),
                       _p(rate), _p(alpha))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle rhs failed: {rc}")
    if return_markers:
        return L, F[:, :nm], rate[:, :nm], alpha
    return L


def rhs_given_alpha(spec, Q, alpha, X=None, U=None, dS=None, xi=None, mlp=None, charwise=False):
    """Right-hand side with the split speeds alpha[3] supplied (for crops of a large state)."""
    Q = _f64(Q)
    nm, X, U, dS, xi = _markers(spec, X, U, dS, xi)
    L = np.zeros_like(Q)
    a = _f64(np.asarray(alpha, dtype=np.float64).reshape(3))
    d = desc(spec, charwise=charwise, mlp=mlp)
    rc = lib().orc_rhs_given_alpha(ctypes.byref(d), _p(Q), nm, _p(X), _p(U), _p(dS), _p(xi),
                                   _p(L), _p(a))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle rhs failed: {rc}")
    return L


def rk3(spec, Q, dt, nsteps=1, X=None, U=None, dS=None, xi=None, t=0.0, charwise=False,
        stretch=None, mlp=None):
    """nsteps SSP-RK3 steps from time t; returns (Q, xi)."""
    Q = _f64(Q).copy()
    nm, X, U, dS, xi = _markers(spec, X, U, dS, xi)
    xi = xi.copy() if xi is not None else None
    d = desc(spec, t, charwise, stretch, mlp)
    rc = lib().orc_rk3(ctypes.byref(d), _p(Q), nm, _p(X), _p(U), _p(dS), _p(xi), float(dt),
                       int(nsteps))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle rk3 failed: {rc}")
    return Q, xi


def probe(spec, Q, xp, stretch=None):
    Q = _f64(Q)
    xp = _f64(xp)
    out = np.zeros(xp.shape[1])
    d = desc(spec, stretch=stretch)
    rc = lib().orc_probe(ctypes.byref(d), _p(Q), xp.shape[1], _p(xp), _p(out))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle probe failed: {rc}")
    return out


def wavespeeds(spec, Q):
    Q = _f64(Q)
    out = np.zeros(3)
    d = desc(spec)
    lib().orc_wavespeeds(ctypes.byref(d), _p(Q), _p(out))
    return out


def interp_scalar(spec, phi, X):
    phi = _f64(phi)
    X = _f64(X)
    out = np.zeros(X.shape[1])
    d = desc(spec)
    rc = lib().orc_interp_scalar(ctypes.byref(d), _p(phi), X.shape[1], _p(X), _p(out))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle interp failed: {rc}")
    return out


def spread_scalar(spec, X, Fk, dS):
    X = _f64(X)
    Fk = _f64(Fk)
    dS = _f64(dS)
    nx, ny, nz = spec.n
    f = np.zeros((nz, ny, nx))
    d = desc(spec)
    rc = lib().orc_spread_scalar(ctypes.byref(d), X.shape[1], _p(X), _p(Fk), _p(dS), _p(f))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle spread failed: {rc}")
    return f


# --------------------------------------------------------------------------------------------
# Flexible plate (Eq. 1, ANCF) and the coupled plate-fluid step (oracle/plate_oracle.c)
# --------------------------------------------------------------------------------------------

class OrcPlate(ctypes.Structure):
    _fields_ = [
        ("n_el", ctypes.c_int),
        ("n_markers", ctypes.c_int),
        ("length", ctypes.c_double),
        ("rho_s", ctypes.c_double),
        ("K_S", ctypes.c_double),
        ("K_B", ctypes.c_double),
        ("clamped", ctypes.c_int),
        ("x0", ctypes.c_double * 2),
        ("theta0", ctypes.c_double),
        ("A0", ctypes.c_double),
        ("freq", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("alpha_m", ctypes.c_double),
        ("phi", ctypes.c_double),
        ("newton_max", ctypes.c_int),
        ("newton_tol", ctypes.c_double),
    ]


ORC_PLATE_NOCONV = -8
_I = ctypes.POINTER(ctypes.c_int)
_plate_ready = False


def _plate_lib():
    global _plate_ready
    L = lib()
    if not _plate_ready:
        P = ctypes.POINTER(OrcPlate)
        L.orc_plate_motion.restype = None
        L.orc_plate_motion.argtypes = [P, ctypes.c_double, _D, _D]
        L.orc_plate_markers.argtypes = [P, _D, _D, _D, _D, _D]
        L.orc_plate_load.argtypes = [P, _D, _D]
        L.orc_plate_internal.argtypes = [P, _D, _D, _D, _D]
        L.orc_plate_step.argtypes = [P, _D, _D, ctypes.c_double, ctypes.c_double, _D, _I]
        L.orc_plate_static.argtypes = [P, _D, _D, _I]
        L.orc_fsi_step.argtypes = [ctypes.POINTER(OrcDesc), P, _D, _D, _D, _D, _D,
                                   ctypes.c_double, ctypes.c_int, _I]
        L.orc_plate_force.argtypes = [P, _D, _D, _D, _D]
        L.orc_fsi_last_load.argtypes = [_D, ctypes.c_int]
        _plate_ready = True
    return L


def plate_desc(ps) -> OrcPlate:
    d = OrcPlate()
    d.n_el = int(ps.n_el)
    d.n_markers = int(ps.n_markers)
    d.length = float(ps.length)
    d.rho_s = float(ps.rho_s)
    d.K_S = float(ps.K_S)
    d.K_B = float(ps.K_B)
    d.clamped = int(ps.clamped)
    d.x0[0], d.x0[1] = float(ps.x0[0]), float(ps.x0[1])
    d.theta0 = float(ps.theta0)
    d.A0 = float(ps.A0)
    d.freq = float(ps.freq)
    d.beta = float(ps.beta)
    d.alpha_m = float(ps.alpha_m)
    d.phi = float(ps.phi)
    d.newton_max = int(ps.newton_max)
    d.newton_tol = float(ps.newton_tol)
    return d


def plate_motion(ps, t):
    """Prescribed clamp coordinates and rates of node 0 at time t (Eq. 17)."""
    e4, v4 = np.zeros(4), np.zeros(4)
    d = plate_desc(ps)
    _plate_lib().orc_plate_motion(ctypes.byref(d), float(t), _p(e4), _p(v4))
    return e4, v4


def plate_markers(ps, e, v):
    e, v = _f64(e), _f64(v)
    nm = ps.n_markers
    X, U, dS = np.zeros((2, nm)), np.zeros((2, nm)), np.zeros(nm)
    d = plate_desc(ps)
    rc = _plate_lib().orc_plate_markers(ctypes.byref(d), _p(e), _p(v), _p(X), _p(U), _p(dS))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle plate markers failed: {rc}")
    return X, U, dS


def plate_load(ps, F):
    F = _f64(F)
    Qf = np.zeros(4 * (ps.n_el + 1))
    d = plate_desc(ps)
    rc = _plate_lib().orc_plate_load(ctypes.byref(d), _p(F), _p(Qf))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle plate load failed: {rc}")
    return Qf


def plate_internal(ps, e, tangent=False, mass=False):
    """Internal force Q_int(e); optionally the dense tangent dQ_int/de and mass matrix."""
    e = _f64(e)
    nd = 4 * (ps.n_el + 1)
    Q = np.zeros(nd)
    K = np.zeros((nd, nd)) if tangent else None
    M = np.zeros((nd, nd)) if mass else None
    d = plate_desc(ps)
    rc = _plate_lib().orc_plate_internal(ctypes.byref(d), _p(e), _p(Q), _p(K), _p(M))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle plate internal failed: {rc}")
    return Q, K, M


def plate_step(ps, e, v, t_new, dt, Qf=None, nsteps=1, check=True):
    """nsteps implicit-midpoint steps under the generalised load Qf (constant); the clamp is
    taken to t_new, t_new + dt, ... Returns (e, v, iterations of the last step).  check=False
    returns the state of a step whose Newton iteration hit its limit instead of raising."""
    e, v = _f64(e).copy(), _f64(v).copy()
    Qf = None if Qf is None else _f64(Qf)
    it = ctypes.c_int(0)
    d = plate_desc(ps)
    t = float(t_new)
    for _ in range(nsteps):
        rc = _plate_lib().orc_plate_step(ctypes.byref(d), _p(e), _p(v), t, float(dt), _p(Qf),
                                         ctypes.byref(it))
        if rc != ORC_OK and (check or rc != ORC_PLATE_NOCONV):
            raise RuntimeError(f"oracle plate step failed: {rc}")
        t = t + float(dt)
    return e, v, it.value


def plate_static(ps, e0, Qf):
    e = _f64(e0).copy()
    Qf = _f64(Qf)
    it = ctypes.c_int(0)
    d = plate_desc(ps)
    rc = _plate_lib().orc_plate_static(ctypes.byref(d), _p(e), _p(Qf), ctypes.byref(it))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle plate static failed: {rc}")
    return e, it.value


def fsi_step(spec, ps, Q, xi, e, v, t, dt, nsteps=1, tf=None):
    """nsteps coupled plate-fluid steps (plate clock t, fluid clock tf, default t); returns
    (Q, xi, e, v, t, Newton iterations per step)."""
    Q = _f64(Q).copy()
    xi = _f64(xi).copy()
    e, v = _f64(e).copy(), _f64(v).copy()
    tt = ctypes.c_double(float(t))
    iters = (ctypes.c_int * max(1, nsteps))()
    d = desc(spec, t if tf is None else tf)
    pd = plate_desc(ps)
    rc = _plate_lib().orc_fsi_step(ctypes.byref(d), ctypes.byref(pd), _p(Q), _p(xi), _p(e), _p(v),
                                   ctypes.cast(ctypes.pointer(tt), _D), float(dt), int(nsteps),
                                   ctypes.cast(iters, _I))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle fsi step failed: {rc}")
    return Q, xi, e, v, tt.value, list(iters)[:nsteps]


def plate_force(ps, F, U):
    """(force [2], power) of the load F on markers moving with U (Eq. 19 numerators)."""
    F, U = _f64(F), _f64(U)
    force = np.zeros(2)
    pw = ctypes.c_double(0.0)
    d = plate_desc(ps)
    rc = _plate_lib().orc_plate_force(ctypes.byref(d), _p(F), _p(U), _p(force),
                                      ctypes.cast(ctypes.pointer(pw), _D))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle plate force failed: {rc}")
    return force, pw.value


def fsi_last_load(ps):
    """The stage-weighted load of the last coupled step, [2][n_markers]."""
    F = np.zeros((2, ps.n_markers))
    rc = _plate_lib().orc_fsi_last_load(_p(F), 2 * ps.n_markers)
    if rc != ORC_OK:
        raise RuntimeError("no coupled step ran")
    return F


def probe_stats(history):
    """Time statistics of probe signals, Sec. 3.2: for each probe (columns of history [T][np]),
    the time mean of dp and the root mean square of dp~ = dp - mean, by the definition (two
    passes over the samples, population form).  A probe with no samples gives 0 and 0."""
    h = np.asarray(history, dtype=np.float64)
    if h.ndim != 2:
        raise ValueError("history must be [T][np]")
    if h.shape[0] == 0:
        return np.zeros(h.shape[1]), np.zeros(h.shape[1])
    mean = h.sum(axis=0) / h.shape[0]
    dev = h - mean
    return mean, np.sqrt((dev * dev).sum(axis=0) / h.shape[0])


def char_eigen(dim, gamma, a, Ql, Qr=None):
    """(R, L, lam): right eigenvectors (columns), left eigenvectors (rows) and eigenvalues of the
    Euler flux Jacobian along direction a at the Roe average of Ql and Qr (Qr = Ql: at Ql)."""
    nv = dim + 2
    Ql = _f64(Ql)
    Qr = Ql if Qr is None else _f64(Qr)
    R = np.zeros((nv, nv))
    L = np.zeros((nv, nv))
    lam = np.zeros(nv)
    rc = lib().orc_char_eigen(int(dim), ctypes.c_double(gamma), int(a), _p(Ql), _p(Qr), _p(R),
                              _p(L), _p(lam))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle eigen-system failed: {rc}")
    return R, L, lam


# --------------------------------------------------------------------------------------------
# learned reconstruction weights (scheme 2 of the oracle)
# --------------------------------------------------------------------------------------------

def mlp_weights(params, x, round_act=True):
    """The network's three softmax weights for normalised stencils x [B, 5]."""
    p = _f64(np.asarray(params))
    x = np.atleast_2d(_f64(np.asarray(x)))
    out = np.zeros((x.shape[0], 3))
    for b in range(x.shape[0]):
        xb = np.ascontiguousarray(x[b])
        wb = np.zeros(3)
        lib().orc_mlp_weights(_p(p), 1 if round_act else 0, _p(xb), _p(wb))
        out[b] = wb
    return out


def learned_recon(mlp, v):
    """The learned reconstruction of stencils v [B, 5] (upwind-ordered): (face values, mask of
    the stencils whose weights came from the network)."""
    v = np.atleast_2d(_f64(np.asarray(v)))
    out = np.zeros(v.shape[0])
    used = np.zeros(v.shape[0], dtype=bool)
    u = ctypes.c_int(0)
    for b in range(v.shape[0]):
        vb = np.ascontiguousarray(v[b])
        out[b] = lib().orc_learned_recon(_p(mlp.params), 1 if mlp.round_act else 0, mlp.floor,
                                         _p(vb), ctypes.byref(u))
        used[b] = bool(u.value)
    return out, used


def mlp_counts():
    """(reconstructions that used the network, all reconstructions) of the last oracle
    right-hand side of the learned scheme."""
    a, b = ctypes.c_longlong(0), ctypes.c_longlong(0)
    lib().orc_mlp_counts(ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value
