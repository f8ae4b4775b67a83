"""Thin Python binding of the libibfsa C ABI (include/ibfsa.h).

The functions carry the C names and only marshal arguments: every step of the stage
right-hand side runs in the CUDA kernels of libibfsa.so.  PyTorch supplies device memory (the
workspace) and the CUDA stream.  There is no CPU fallback: if the library is missing or no GPU
is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libibfsa.so")

IBFSA_OK = 0
IBFSA_ERR_ARG = -1
IBFSA_ERR_CUDA = -2
IBFSA_ERR_NONFINITE = -3
IBFSA_ERR_BOUNDS = -4
IBFSA_ERR_UNSUPPORTED = -5
IBFSA_ERR_WORKSPACE = -6
IBFSA_STATUS_BOUNDS = 1
IBFSA_STATUS_NONFINITE = 2
IBFSA_STATUS_TIMEOUT = 4
IBFSA_STATUS_NOCONV = 8
IBFSA_PLATE_FREE = 0
IBFSA_PLATE_CLAMPED = 1
IBFSA_PLATE_MAX_EL = 128

# every symbol include/ibfsa.h declares
EXPORTS = (
    "ibfsa_workspace_bytes", "ibfsa_create_grid", "ibfsa_destroy_grid", "ibfsa_set_state",
    "ibfsa_get_state", "ibfsa_set_markers", "ibfsa_get_marker_forces",
    "ibfsa_get_penalty_integral", "ibfsa_set_penalty_integral", "ibfsa_rhs", "ibfsa_rk3_step",
    "ibfsa_max_wavespeed", "ibfsa_probe", "ibfsa_probe_accumulate", "ibfsa_probe_stats",
    "ibfsa_get_status", "ibfsa_last_error",
    "ibfsa_profile_enable", "ibfsa_profile_read", "ibfsa_rhs_noalloc",
    "ibfsa_mlp_state_bytes", "ibfsa_mlp_init", "ibfsa_mlp_train_step", "ibfsa_mlp_read",
    "ibfsa_mlp_eval", "ibfsa_set_mlp", "ibfsa_mlp_stats", "ibfsa_mlp_sample",
    "ibfsa_body_force", "ibfsa_plate_workspace_bytes", "ibfsa_plate_create",
    "ibfsa_plate_destroy", "ibfsa_plate_set_state", "ibfsa_plate_get_state", "ibfsa_plate_step",
    "ibfsa_plate_markers", "ibfsa_plate_get_status", "ibfsa_fsi_step", "ibfsa_plate_force",
    "ibfsa_set_source", "ibfsa_set_time", "ibfsa_get_time", "ibfsa_set_mesh",
    "ibfsa_selftest_wait",
)
MLP_NPARAM = 2403

KERNEL_CLASSES = ("pad", "ib_interp", "conv_x", "conv_y", "conv_z", "visc_flux", "visc_div",
                  "ib_spread", "finish", "probe", "plate")


class IbfsaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libibfsa error {code}: {msg}")
        self.code = code


class GridDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("gamma", ctypes.c_double),
        ("Re", ctypes.c_double),
        ("qinf", ctypes.c_double * 5),
        ("scheme", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("strict_fp", ctypes.c_int),
        ("bc", (ctypes.c_int * 2) * 3),
        ("sponge_cells", ctypes.c_int),
        ("sponge_sigma", ctypes.c_double),
        ("alpha_pen", ctypes.c_double),
        ("beta_pen", ctypes.c_double),
        ("max_markers", ctypes.c_int),
        ("max_probes", ctypes.c_int),
        ("charwise", ctypes.c_int),
    ]


class PlateDesc(ctypes.Structure):
    _fields_ = [
        ("n_el", ctypes.c_int),
        ("n_markers", ctypes.c_int),
        ("length", ctypes.c_double),
        ("rho_s", ctypes.c_double),
        ("K_S", ctypes.c_double),
        ("K_B", ctypes.c_double),
        ("clamp", ctypes.c_int),
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


_lib = None
_P = ctypes.c_void_p


def lib():
    """Load libibfsa.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        D = ctypes.POINTER(GridDesc)
        L.ibfsa_workspace_bytes.argtypes = [D, ctypes.POINTER(ctypes.c_size_t)]
        L.ibfsa_create_grid.argtypes = [D, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]
        L.ibfsa_destroy_grid.argtypes = [_P]
        L.ibfsa_set_state.argtypes = [_P, _P]
        L.ibfsa_get_state.argtypes = [_P, _P]
        L.ibfsa_set_markers.argtypes = [_P, ctypes.c_int, _P, _P, _P, ctypes.c_int]
        L.ibfsa_get_marker_forces.argtypes = [_P, _P]
        L.ibfsa_get_penalty_integral.argtypes = [_P, _P]
        L.ibfsa_set_penalty_integral.argtypes = [_P, _P]
        L.ibfsa_rhs.argtypes = [_P, _P]
        L.ibfsa_rk3_step.argtypes = [_P, ctypes.c_double, ctypes.c_int]
        L.ibfsa_max_wavespeed.argtypes = [_P, ctypes.POINTER(ctypes.c_double)]
        L.ibfsa_probe.argtypes = [_P, ctypes.c_int, _P, _P]
        L.ibfsa_probe_accumulate.argtypes = [_P, ctypes.c_int, _P, _P, _P]
        L.ibfsa_probe_stats.argtypes = [_P, ctypes.c_int, _P, _P, _P]
        L.ibfsa_get_status.argtypes = [_P, ctypes.POINTER(ctypes.c_int)]
        L.ibfsa_last_error.restype = ctypes.c_char_p
        L.ibfsa_profile_enable.argtypes = [_P, ctypes.c_int]
        L.ibfsa_profile_read.argtypes = [_P, ctypes.c_int, _P, _P, _P]
        L.ibfsa_mlp_state_bytes.restype = ctypes.c_size_t
        L.ibfsa_mlp_state_bytes.argtypes = []
        L.ibfsa_mlp_init.argtypes = [_P, _P, _P]
        L.ibfsa_mlp_train_step.argtypes = [_P, ctypes.c_int, _P, _P, ctypes.c_float, ctypes.c_int, _P]
        L.ibfsa_mlp_read.argtypes = [_P, _P, _P, _P, _P]
        L.ibfsa_mlp_eval.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P]
        L.ibfsa_body_force.argtypes = [_P, _P, _P]
        L.ibfsa_set_mlp.argtypes = [_P, _P]
        L.ibfsa_mlp_stats.argtypes = [_P, _P]
        L.ibfsa_mlp_sample.argtypes = [_P, ctypes.c_int, ctypes.c_ulonglong, ctypes.c_int, _P, _P,
                                       _P]
        L.ibfsa_rhs_noalloc.argtypes = [D, _P, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P, _P]
        PD = ctypes.POINTER(PlateDesc)
        L.ibfsa_plate_workspace_bytes.argtypes = [PD, ctypes.POINTER(ctypes.c_size_t)]
        L.ibfsa_plate_create.argtypes = [PD, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]
        L.ibfsa_plate_destroy.argtypes = [_P]
        L.ibfsa_plate_set_state.argtypes = [_P, _P, _P, ctypes.c_double]
        L.ibfsa_plate_get_state.argtypes = [_P, _P, _P, ctypes.POINTER(ctypes.c_double)]
        L.ibfsa_plate_step.argtypes = [_P, ctypes.c_double, _P]
        L.ibfsa_plate_markers.argtypes = [_P, _P, _P, _P]
        L.ibfsa_plate_get_status.argtypes = [_P, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_int)]
        L.ibfsa_fsi_step.argtypes = [_P, _P, ctypes.c_double, ctypes.c_int]
        L.ibfsa_plate_force.argtypes = [_P, _P, _P]
        L.ibfsa_set_source.argtypes = [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double, _P]
        L.ibfsa_set_time.argtypes = [_P, ctypes.c_double]
        L.ibfsa_set_mesh.argtypes = [_P, ctypes.c_int, _P, _P]
        L.ibfsa_selftest_wait.argtypes = [_P]
        L.ibfsa_get_time.argtypes = [_P, ctypes.POINTER(ctypes.c_double)]
        _lib = L
    return _lib


def _check(rc):
    if rc != IBFSA_OK:
        raise IbfsaError(rc, lib().ibfsa_last_error().decode())


def desc_from_spec(spec: W.GridSpec, strict: bool = False, max_probes: int = 0) -> GridDesc:
    d = GridDesc()
    d.dim = spec.dim
    for a in range(3):
        d.n[a] = int(spec.n[a])
        d.lo[a] = float(spec.lo[a])
        d.hi[a] = float(spec.hi[a])
        d.bc[a][0] = int(spec.bc[a][0])
        d.bc[a][1] = int(spec.bc[a][1])
    d.gamma = float(spec.gamma)
    d.Re = float(spec.Re)
    for c in range(5):
        d.qinf[c] = float(spec.qinf[c])
    d.scheme = int(spec.scheme)
    d.precision = int(spec.precision)
    d.strict_fp = 1 if strict else 0
    d.sponge_cells = int(spec.sponge_cells)
    d.sponge_sigma = float(spec.sponge_sigma)
    d.alpha_pen = float(spec.alpha_pen)
    d.beta_pen = float(spec.beta_pen)
    d.max_markers = int(spec.max_markers)
    d.max_probes = int(max_probes)
    d.charwise = int(spec.charwise)
    return d


# ---- the C entry points, same names --------------------------------------------------------

def ibfsa_workspace_bytes(desc: GridDesc) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().ibfsa_workspace_bytes(ctypes.byref(desc), ctypes.byref(n)))
    return n.value


def ibfsa_create_grid(desc: GridDesc, workspace_ptr: int, workspace_bytes: int, stream_ptr: int):
    h = _P()
    _check(lib().ibfsa_create_grid(ctypes.byref(desc), _P(workspace_ptr), workspace_bytes,
                                   _P(stream_ptr), ctypes.byref(h)))
    return h


def ibfsa_destroy_grid(g):
    _check(lib().ibfsa_destroy_grid(g))


def ibfsa_set_state(g, ptr: int):
    _check(lib().ibfsa_set_state(g, _P(ptr)))


def ibfsa_get_state(g, ptr: int):
    _check(lib().ibfsa_get_state(g, _P(ptr)))


def ibfsa_set_markers(g, n: int, X: int, U: int, dS: int, reset_integral: int = 1):
    _check(lib().ibfsa_set_markers(g, n, _P(X), _P(U), _P(dS), reset_integral))


def ibfsa_get_marker_forces(g, ptr: int):
    _check(lib().ibfsa_get_marker_forces(g, _P(ptr)))


def ibfsa_get_penalty_integral(g, ptr: int):
    _check(lib().ibfsa_get_penalty_integral(g, _P(ptr)))


def ibfsa_set_penalty_integral(g, ptr: int):
    _check(lib().ibfsa_set_penalty_integral(g, _P(ptr)))


def ibfsa_rhs(g, ptr: int):
    _check(lib().ibfsa_rhs(g, _P(ptr)))


def ibfsa_rk3_step(g, dt: float, nsteps: int = 1):
    _check(lib().ibfsa_rk3_step(g, float(dt), int(nsteps)))


def ibfsa_max_wavespeed(g):
    out = (ctypes.c_double * 3)()
    _check(lib().ibfsa_max_wavespeed(g, out))
    return list(out)


def ibfsa_probe(g, np_: int, xp: int, out: int):
    _check(lib().ibfsa_probe(g, int(np_), _P(xp), _P(out)))


def ibfsa_probe_accumulate(g, np_: int, xp: int, out: int, acc: int):
    _check(lib().ibfsa_probe_accumulate(g, int(np_), _P(xp), _P(out), _P(acc)))


def ibfsa_probe_stats(g, np_: int, acc: int, mean: int, rms: int):
    _check(lib().ibfsa_probe_stats(g, int(np_), _P(acc), _P(mean), _P(rms)))


def ibfsa_get_status(g) -> int:
    v = ctypes.c_int(0)
    _check(lib().ibfsa_get_status(g, ctypes.byref(v)))
    return v.value


def ibfsa_profile_enable(g, enable: bool):
    _check(lib().ibfsa_profile_enable(g, 1 if enable else 0))


def ibfsa_profile_read(g):
    n = len(KERNEL_CLASSES)
    ms = (ctypes.c_double * n)()
    launches = (ctypes.c_longlong * n)()
    timed = (ctypes.c_longlong * n)()
    _check(lib().ibfsa_profile_read(g, n, ctypes.cast(ms, _P), ctypes.cast(launches, _P),
                                    ctypes.cast(timed, _P)))
    return {k: dict(ms=ms[i], launches=launches[i], timed=timed[i])
            for i, k in enumerate(KERNEL_CLASSES)}


def ibfsa_rhs_noalloc(desc: GridDesc, Q: int, n_markers: int, X: int, U: int, dS: int, xi: int,
                      L: int, F: int = 0, status: int = 0, stream: int = 0):
    """Right-hand side without a grid or workspace (device pointers in and out); see the
    header for who needs it and its scratch limit."""
    _check(lib().ibfsa_rhs_noalloc(ctypes.byref(desc), _P(Q), int(n_markers), _P(X), _P(U),
                                   _P(dS), _P(xi), _P(L), _P(F or None), _P(status or None),
                                   _P(stream)))


def ibfsa_mlp_state_bytes() -> int:
    return int(lib().ibfsa_mlp_state_bytes())


def ibfsa_mlp_init(state: int, params: int, stream: int = 0):
    _check(lib().ibfsa_mlp_init(_P(state), _P(params), _P(stream)))


def ibfsa_mlp_train_step(state: int, n: int, stencils: int, targets: int, lr: float, step: int,
                         stream: int = 0):
    _check(lib().ibfsa_mlp_train_step(_P(state), int(n), _P(stencils), _P(targets), float(lr),
                                      int(step), _P(stream)))


def ibfsa_mlp_read(state: int, params: int = 0, grad: int = 0, loss: int = 0, stream: int = 0):
    _check(lib().ibfsa_mlp_read(_P(state), _P(params or None), _P(grad or None),
                                _P(loss or None), _P(stream)))


def ibfsa_mlp_eval(state: int, n: int, stencils: int, targets: int = 0, face: int = 0,
                   omega: int = 0, loss: int = 0, stream: int = 0):
    _check(lib().ibfsa_mlp_eval(_P(state), int(n), _P(stencils), _P(targets or None),
                                _P(face or None), _P(omega or None), _P(loss or None),
                                _P(stream)))


def ibfsa_body_force(g):
    f = (ctypes.c_double * 3)()
    pw = ctypes.c_double(0.0)
    _check(lib().ibfsa_body_force(g, ctypes.cast(f, _P), ctypes.cast(ctypes.byref(pw), _P)))
    return list(f), pw.value


def ibfsa_set_mlp(g, state: int):
    _check(lib().ibfsa_set_mlp(g, _P(state)))


def ibfsa_mlp_stats(g):
    c = (ctypes.c_ulonglong * 2)()
    _check(lib().ibfsa_mlp_stats(g, ctypes.cast(c, _P)))
    return int(c[0]), int(c[1])


def ibfsa_mlp_sample(g, n_max: int, seed: int, attempts: int, stencils: int, targets: int,
                     count: int):
    _check(lib().ibfsa_mlp_sample(g, int(n_max), int(seed), int(attempts), _P(stencils),
                                  _P(targets), _P(count)))


class MLP:
    """Training state of the learned weights in device memory (torch-allocated)."""

    def __init__(self, params):
        import torch
        self.nbytes = ibfsa_mlp_state_bytes()
        self.buf = torch.zeros(self.nbytes // 4 + 64, dtype=torch.float32, device="cuda")
        self.ptr = (self.buf.data_ptr() + 255) & ~255
        p = torch.as_tensor(np.ascontiguousarray(params, dtype=np.float32)).cuda()
        ibfsa_mlp_init(self.ptr, p.data_ptr(), torch.cuda.current_stream().cuda_stream)
        self.step = 0

    def train_step(self, stencils, targets, lr):
        import torch
        self.step += 1
        ibfsa_mlp_train_step(self.ptr, stencils.shape[0], stencils.data_ptr(),
                             targets.data_ptr(), lr, self.step,
                             torch.cuda.current_stream().cuda_stream)

    def gradient(self, stencils, targets):
        import torch
        ibfsa_mlp_train_step(self.ptr, stencils.shape[0], stencils.data_ptr(),
                             targets.data_ptr(), 0.0, max(1, self.step),
                             torch.cuda.current_stream().cuda_stream)
        g = np.zeros(MLP_NPARAM, np.float32)
        loss = np.zeros(1, np.float32)
        ibfsa_mlp_read(self.ptr, 0, g.ctypes.data, loss.ctypes.data,
                       torch.cuda.current_stream().cuda_stream)
        return float(loss[0]), g

    def params(self):
        import torch
        p = np.zeros(MLP_NPARAM, np.float32)
        loss = np.zeros(1, np.float32)
        ibfsa_mlp_read(self.ptr, p.ctypes.data, 0, loss.ctypes.data,
                       torch.cuda.current_stream().cuda_stream)
        return p, float(loss[0])

    def eval(self, stencils, targets=None):
        import torch
        n = stencils.shape[0]
        face = torch.empty(n, dtype=torch.float32, device="cuda")
        omega = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        ibfsa_mlp_eval(self.ptr, n, stencils.data_ptr(),
                       targets.data_ptr() if targets is not None else 0, face.data_ptr(),
                       omega.data_ptr(), loss.data_ptr() if targets is not None else 0,
                       torch.cuda.current_stream().cuda_stream)
        return face, omega, (float(loss.item()) if targets is not None else None)


def plate_desc_from_spec(ps: W.PlateSpec) -> PlateDesc:
    d = PlateDesc()
    d.n_el = int(ps.n_el)
    d.n_markers = int(ps.n_markers)
    d.length = float(ps.length)
    d.rho_s = float(ps.rho_s)
    d.K_S = float(ps.K_S)
    d.K_B = float(ps.K_B)
    d.clamp = IBFSA_PLATE_CLAMPED if ps.clamped else IBFSA_PLATE_FREE
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


def ibfsa_plate_workspace_bytes(desc: PlateDesc) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().ibfsa_plate_workspace_bytes(ctypes.byref(desc), ctypes.byref(n)))
    return n.value


def ibfsa_plate_create(desc: PlateDesc, workspace_ptr: int, workspace_bytes: int,
                       stream_ptr: int):
    h = _P()
    _check(lib().ibfsa_plate_create(ctypes.byref(desc), workspace_ptr, workspace_bytes,
                                    stream_ptr, ctypes.byref(h)))
    return h


def ibfsa_plate_destroy(p):
    _check(lib().ibfsa_plate_destroy(p))


def ibfsa_plate_set_state(p, e: int, v: int, t: float):
    _check(lib().ibfsa_plate_set_state(p, e, v, float(t)))


def ibfsa_plate_get_state(p, e: int, v: int) -> float:
    t = ctypes.c_double(0.0)
    _check(lib().ibfsa_plate_get_state(p, e, v, ctypes.byref(t)))
    return t.value


def ibfsa_plate_step(p, dt: float, F: int = 0):
    _check(lib().ibfsa_plate_step(p, float(dt), F))


def ibfsa_plate_markers(p, X: int, U: int, dS: int):
    _check(lib().ibfsa_plate_markers(p, X, U, dS))


def ibfsa_plate_get_status(p):
    f, it = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().ibfsa_plate_get_status(p, ctypes.byref(f), ctypes.byref(it)))
    return f.value, it.value


def ibfsa_plate_force(p):
    f = (ctypes.c_double * 2)()
    pw = ctypes.c_double(0.0)
    _check(lib().ibfsa_plate_force(p, ctypes.cast(f, _P), ctypes.cast(ctypes.pointer(pw), _P)))
    return np.array([f[0], f[1]]), pw.value


def ibfsa_set_source(g, amp: float, b: float, omega: float, xc):
    c = (ctypes.c_double * 3)(*[float(x) for x in list(xc) + [0.0] * (3 - len(xc))])
    _check(lib().ibfsa_set_source(g, float(amp), float(b), float(omega), ctypes.cast(c, _P)))


def ibfsa_set_time(g, t: float):
    _check(lib().ibfsa_set_time(g, float(t)))


def ibfsa_get_time(g) -> float:
    t = ctypes.c_double(0.0)
    _check(lib().ibfsa_get_time(g, ctypes.byref(t)))
    return t.value


def ibfsa_set_mesh(g, a: int, x_nodes: int, dxdxi: int):
    """Stretched mesh along direction a: node coordinates and dx/dxi at i = -4 .. n+3 (pointers;
    both 0: uniform again)."""
    _check(lib().ibfsa_set_mesh(g, int(a), _P(x_nodes or None), _P(dxdxi or None)))


def ibfsa_selftest_wait(g):
    """Run the bounded-wait self-test on the grid's stream (it reports IBFSA_STATUS_TIMEOUT)."""
    _check(lib().ibfsa_selftest_wait(g))


def ibfsa_fsi_step(g, p, dt: float, nsteps: int = 1):
    _check(lib().ibfsa_fsi_step(g, p, float(dt), int(nsteps)))


# ---- convenience wrapper over torch tensors -------------------------------------------------

def _dev_f64(x, device):
    import torch
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    return x.to(device=device, dtype=torch.float64).contiguous()


class Grid:
    """A grid with its torch-allocated workspace on the current CUDA device and stream."""

    def __init__(self, spec: W.GridSpec, strict: bool = False, max_probes: int = 0,
                 stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libibfsa needs a CUDA device")
        self.spec = spec
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.desc = desc_from_spec(spec, strict=strict, max_probes=max_probes)
        self.ws_bytes = ibfsa_workspace_bytes(self.desc)
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self.ws_ptr = (base + 255) & ~255
        self.h = ibfsa_create_grid(self.desc, self.ws_ptr, self.ws_bytes, self.stream.cuda_stream)
        self.nm = 0
        if spec.src_amp != 0.0:
            ibfsa_set_source(self.h, spec.src_amp, spec.src_b, spec.src_omega, spec.src_xc)
        self._state_src = None
        self._marker_src = None

    def close(self):
        if self.h is not None:
            ibfsa_destroy_grid(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, Q):
        t = _dev_f64(Q, self.device)
        assert tuple(t.shape) == self.spec.shape()
        ibfsa_set_state(self.h, t.data_ptr())
        self._state_src = t  # kept alive until the next set_state (the copy is asynchronous)

    def get_state(self):
        import torch
        out = torch.empty(self.spec.shape(), dtype=torch.float64, device=self.device)
        ibfsa_get_state(self.h, out.data_ptr())
        return out

    def set_markers(self, X, U, dS, reset_integral=True):
        X = _dev_f64(X, self.device)
        U = _dev_f64(U, self.device)
        dS = _dev_f64(dS, self.device)
        n = X.shape[1]
        ibfsa_set_markers(self.h, n, X.data_ptr(), U.data_ptr(), dS.data_ptr(),
                          1 if reset_integral else 0)
        self.nm = n
        self._marker_src = (X, U, dS)

    def marker_forces(self):
        import torch
        out = torch.empty((self.spec.dim, self.nm), dtype=torch.float64, device=self.device)
        ibfsa_get_marker_forces(self.h, out.data_ptr())
        return out

    def penalty_integral(self):
        import torch
        out = torch.empty((self.spec.dim, self.nm), dtype=torch.float64, device=self.device)
        ibfsa_get_penalty_integral(self.h, out.data_ptr())
        return out

    def rhs(self):
        import torch
        out = torch.empty(self.spec.shape(), dtype=torch.float64, device=self.device)
        ibfsa_rhs(self.h, out.data_ptr())
        return out

    def rk3_step(self, dt, nsteps=1):
        ibfsa_rk3_step(self.h, dt, nsteps)

    def max_wavespeed(self):
        return ibfsa_max_wavespeed(self.h)[: self.spec.dim]

    def probe(self, xp):
        import torch
        xp = _dev_f64(xp, self.device)
        out = torch.empty(xp.shape[1], dtype=torch.float64, device=self.device)
        ibfsa_probe(self.h, xp.shape[1], xp.data_ptr(), out.data_ptr())
        return out

    def probe_accumulate(self, xp, acc):
        """Samples dp at xp [dim][np] into a fresh tensor and folds it into acc, a zero-filled
        float64 device tensor of 3*np entries (count, running mean, running M2)."""
        import torch
        xp = _dev_f64(xp, self.device)
        npr = xp.shape[1]
        if acc.dtype != torch.float64 or acc.device != self.device or acc.numel() != 3 * npr \
                or not acc.is_contiguous():
            raise ValueError("acc must be a contiguous float64 tensor of 3*np entries on the "
                             "grid's device")
        out = torch.empty(npr, dtype=torch.float64, device=self.device)
        ibfsa_probe_accumulate(self.h, npr, xp.data_ptr(), out.data_ptr(), acc.data_ptr())
        return out

    def probe_stats(self, acc):
        """(time mean of dp, RMS of dp about that mean) per probe from an accumulator."""
        import torch
        npr = acc.numel() // 3
        mean = torch.empty(npr, dtype=torch.float64, device=self.device)
        rms = torch.empty_like(mean)
        ibfsa_probe_stats(self.h, npr, acc.data_ptr(), mean.data_ptr(), rms.data_ptr())
        return mean, rms

    def status(self) -> int:
        return ibfsa_get_status(self.h)

    def time(self) -> float:
        return ibfsa_get_time(self.h)

    def set_time(self, t: float):
        ibfsa_set_time(self.h, t)

    def set_mesh(self, a: int, nodes=None, metric=None):
        """Stretch direction a: node coordinates and dx/dxi at i = -4 .. n[a]+3 (arrays of
        n[a] + 8 entries); None: uniform again."""
        if nodes is None:
            ibfsa_set_mesh(self.h, a, 0, 0)
            return
        x = np.ascontiguousarray(nodes, dtype=np.float64)
        m = np.ascontiguousarray(metric, dtype=np.float64)
        if x.shape != (self.spec.n[a] + 8,) or m.shape != x.shape:
            raise ValueError(f"direction {a}: nodes and metric need n + 8 = "
                             f"{self.spec.n[a] + 8} entries")
        ibfsa_set_mesh(self.h, a, x.ctypes.data, m.ctypes.data)  # copied, synchronised


class Plate:
    """A flexible plate with its torch-allocated workspace on the current device and stream."""

    def __init__(self, ps: W.PlateSpec, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libibfsa needs a CUDA device")
        self.ps = ps
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.desc = plate_desc_from_spec(ps)
        self.ws_bytes = ibfsa_plate_workspace_bytes(self.desc)
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        self.ws_ptr = (self.ws.data_ptr() + 255) & ~255
        self.h = ibfsa_plate_create(self.desc, self.ws_ptr, self.ws_bytes,
                                    self.stream.cuda_stream)
        self._src = None
        self._load = None

    def close(self):
        if self.h is not None:
            ibfsa_plate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, e, v, t=0.0):
        e = _dev_f64(e, self.device)
        v = _dev_f64(v, self.device)
        ibfsa_plate_set_state(self.h, e.data_ptr(), v.data_ptr(), t)
        self._src = (e, v)

    def get_state(self):
        import torch
        nd = self.ps.ndof
        e = torch.empty(nd, dtype=torch.float64, device=self.device)
        v = torch.empty(nd, dtype=torch.float64, device=self.device)
        t = ibfsa_plate_get_state(self.h, e.data_ptr(), v.data_ptr())
        return e, v, t

    def step(self, dt, F=None):
        """One step under marker forces F [2][n_markers] (None: no load)."""
        if F is None:
            ibfsa_plate_step(self.h, dt, 0)
        else:
            F = _dev_f64(F, self.device)
            ibfsa_plate_step(self.h, dt, F.data_ptr())
            self._load = F  # the copy into the workspace is asynchronous

    def markers(self):
        import torch
        nm = self.ps.n_markers
        X = torch.empty((2, nm), dtype=torch.float64, device=self.device)
        U = torch.empty((2, nm), dtype=torch.float64, device=self.device)
        dS = torch.empty(nm, dtype=torch.float64, device=self.device)
        ibfsa_plate_markers(self.h, X.data_ptr(), U.data_ptr(), dS.data_ptr())
        return X, U, dS

    def status(self):
        """(status bits, largest Newton iteration count) since the last call."""
        return ibfsa_plate_get_status(self.h)

    def force(self):
        """(force [2], power) of the last step's load (Eq. 19 numerators)."""
        return ibfsa_plate_force(self.h)


def fsi_step(grid: Grid, plate: Plate, dt: float, nsteps: int = 1):
    """nsteps coupled plate-fluid steps (ibfsa_fsi_step)."""
    ibfsa_fsi_step(grid.h, plate.h, dt, nsteps)
    grid.nm = plate.ps.n_markers
