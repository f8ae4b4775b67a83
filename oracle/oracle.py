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
_LIB = os.path.join(_HERE, "libibfsa_oracle.so")

ORC_OK = 0
ORC_ERR_ARG = -1
ORC_ERR_BOUNDS = -4


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc: -O2, no fused multiply-add contraction."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
               "-o", _LIB, _SRC, "-lm"]
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
    return _lib


def desc(spec) -> OrcDesc:
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


def rhs(spec, Q, X=None, U=None, dS=None, xi=None, return_markers=False):
    """RHS L(Q) + S of every interior cell, shape [nv][nz][ny][nx]."""
    Q = _f64(Q)
    nm, X, U, dS, xi = _markers(spec, X, U, dS, xi)
    L = np.zeros_like(Q)
    F = np.zeros((spec.dim, max(nm, 1)))
    rate = np.zeros((spec.dim, max(nm, 1)))
    alpha = np.zeros(3)
    d = desc(spec)
    rc = lib().orc_rhs(ctypes.byref(d), _p(Q), nm, _p(X), _p(U), _p(dS), _p(xi), _p(L), _p(F),
                       _p(rate), _p(alpha))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle rhs failed: {rc}")
    if return_markers:
        return L, F[:, :nm], rate[:, :nm], alpha
    return L


def rhs_given_alpha(spec, Q, alpha, X=None, U=None, dS=None, xi=None):
    """Right-hand side with the split speeds alpha[3] supplied (for crops of a large state)."""
    Q = _f64(Q)
    nm, X, U, dS, xi = _markers(spec, X, U, dS, xi)
    L = np.zeros_like(Q)
    a = _f64(np.asarray(alpha, dtype=np.float64).reshape(3))
    d = desc(spec)
    rc = lib().orc_rhs_given_alpha(ctypes.byref(d), _p(Q), nm, _p(X), _p(U), _p(dS), _p(xi),
                                   _p(L), _p(a))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle rhs failed: {rc}")
    return L


def rk3(spec, Q, dt, nsteps=1, X=None, U=None, dS=None, xi=None):
    """nsteps SSP-RK3 steps; returns (Q, xi)."""
    Q = _f64(Q).copy()
    nm, X, U, dS, xi = _markers(spec, X, U, dS, xi)
    xi = xi.copy() if xi is not None else None
    d = desc(spec)
    rc = lib().orc_rk3(ctypes.byref(d), _p(Q), nm, _p(X), _p(U), _p(dS), _p(xi), float(dt),
                       int(nsteps))
    if rc != ORC_OK:
        raise RuntimeError(f"oracle rk3 failed: {rc}")
    return Q, xi


def probe(spec, Q, xp):
    Q = _f64(Q)
    xp = _f64(xp)
    out = np.zeros(xp.shape[1])
    d = desc(spec)
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
