"""ctypes front end of the FP64 CPU oracle (``prost_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it to check and time the CUDA path.  The
library in ``paper_1302_2073_gb300`` never imports it.

The C source is compiled with gcc on first use (or by :func:`build`) into
``oracle/_build/liboracle.so``.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prost_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")

MAX_CG = 64
FRAME_U8, FRAME_F32, FRAME_F64 = 0, 1, 2
_DT = {"u8": FRAME_U8, "f32": FRAME_F32, "f64": FRAME_F64}
_NP = {FRAME_U8: np.uint8, FRAME_F32: np.float32, FRAME_F64: np.float64}


class OrcParams(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("channels", C.c_int32),
                ("k", C.c_int32), ("p", C.c_double), ("mu", C.c_double),
                ("delta", C.c_double), ("omega", C.c_double), ("t_init", C.c_double),
                ("t_min", C.c_double), ("i_init", C.c_int32), ("n_cg", C.c_int32),
                ("in_scale", C.c_double), ("in_offset", C.c_double),
                ("mask_from", C.c_int32), ("reorth", C.c_int32)]


class OrcTrace(C.Structure):
    _fields_ = [("cost", C.c_double * (MAX_CG + 1)), ("alpha", C.c_double * MAX_CG),
                ("beta", C.c_double * MAX_CG), ("gnorm", C.c_double * (MAX_CG + 1)),
                ("pi_norm", C.c_double), ("y_norm", C.c_double), ("sigma", C.c_double),
                ("t", C.c_double), ("theta", C.c_double), ("updated", C.c_int32),
                ("pad", C.c_int32), ("n_foreground", C.c_int64)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, -O2, no fast-math)."""
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared",
                           "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _OUT)
    return _OUT


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        u8p = C.POINTER(C.c_uint8)
        prm = C.POINTER(OrcParams)
        tr = C.POINTER(OrcTrace)
        L.orc_check_params.argtypes = [prm]
        L.orc_h.restype = C.c_double
        L.orc_h.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_mu_heuristic.restype = C.c_double
        L.orc_mu_heuristic.argtypes = [C.c_double, C.c_double]
        L.orc_step_size.restype = C.c_double
        L.orc_step_size.argtypes = [prm, C.c_int64]
        L.orc_preprocess.argtypes = [prm, C.c_void_p, C.c_int, dp]
        L.orc_weights.argtypes = [prm, u8p, dp]
        L.orc_residual.argtypes = [C.c_int64, C.c_int, dp, dp, dp, dp]
        L.orc_cost.restype = C.c_double
        L.orc_cost.argtypes = [prm, dp, dp, dp, dp]
        L.orc_eta.argtypes = [prm, dp, dp, dp]
        L.orc_ut.argtypes = [C.c_int64, C.c_int, dp, dp, dp]
        L.orc_grad_U.argtypes = [C.c_int64, C.c_int, dp, dp, dp]
        L.orc_project.argtypes = [C.c_int64, C.c_int, dp, dp, dp]
        L.orc_cg.argtypes = [prm, dp, dp, dp, dp, tr]
        L.orc_grassmann_step.argtypes = [prm, dp, dp, dp, C.c_double, tr]
        L.orc_labels.restype = C.c_int64
        L.orc_labels.argtypes = [prm, dp, dp, dp, u8p, dp]
        L.orc_reorthonormalize.argtypes = [C.c_int64, C.c_int, dp, dp]
        L.orc_frame_step.argtypes = [prm, dp, dp, u8p, C.c_int64, C.c_void_p, C.c_int, tr, dp]
        _lib = L
    return _lib


def _d(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _u8(a):
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def params(width, height, channels, k, p=0.25, mu=None, delta=0.35, omega=5e-5,
           t_init=5e-3, t_min=1e-4, i_init=100, n_cg=5, in_scale=1.0, in_offset=0.0,
           mask_from=0, reorth=1, **_ignored) -> OrcParams:
    if mu is None:
        mu = lib().orc_mu_heuristic(delta, p)
    return OrcParams(int(width), int(height), int(channels), int(k), float(p), float(mu),
                     float(delta), float(omega), float(t_init), float(t_min), int(i_init),
                     int(n_cg), float(in_scale), float(in_offset), int(mask_from), int(reorth))


def _m(prm):
    return prm.width * prm.height * prm.channels


def _P(prm):
    return prm.width * prm.height


# ---- thin wrappers over the C functions --------------------------------------

def h(r, mu, p):
    return lib().orc_h(float(r), float(mu), float(p))


def mu_heuristic(delta, p):
    return lib().orc_mu_heuristic(float(delta), float(p))


def step_size(prm, i):
    return lib().orc_step_size(C.byref(prm), int(i))


def preprocess(prm, frame):
    frame = np.ascontiguousarray(frame)
    dt = {np.dtype(np.uint8): FRAME_U8, np.dtype(np.float32): FRAME_F32,
          np.dtype(np.float64): FRAME_F64}[frame.dtype]
    assert frame.size == _m(prm)
    x = np.empty(_m(prm))
    lib().orc_preprocess(C.byref(prm), frame.ctypes.data_as(C.c_void_p), dt, _d(x))
    return x


def weights(prm, labels):
    w = np.empty(_P(prm))
    lab = None if labels is None else _u8(np.ascontiguousarray(labels, dtype=np.uint8).ravel())
    lib().orc_weights(C.byref(prm), lab, _d(w))
    return w


def residual(U, y, x):
    U, y, x = _f64(U), _f64(y), _f64(x)
    r = np.empty(U.shape[0])
    lib().orc_residual(U.shape[0], U.shape[1], _d(U), _d(y), _d(x), _d(r))
    return r


def cost(prm, U, y, x, w):
    U, y, x, w = _f64(U), _f64(y), _f64(x), _f64(w)
    return lib().orc_cost(C.byref(prm), _d(U), _d(y), _d(x), _d(w))


def eta(prm, r, w):
    r, w = _f64(r), _f64(w)
    out = np.empty_like(r)
    lib().orc_eta(C.byref(prm), _d(r), _d(w), _d(out))
    return out


def ut(U, v):
    U, v = _f64(U), _f64(v)
    out = np.empty(U.shape[1])
    lib().orc_ut(U.shape[0], U.shape[1], _d(U), _d(v), _d(out))
    return out


def grad_U(eta_, y):
    eta_, y = _f64(eta_), _f64(y)
    G = np.empty((eta_.size, y.size))
    lib().orc_grad_U(eta_.size, y.size, _d(eta_), _d(y), _d(G))
    return G


def project(U, hcol):
    U, hcol = _f64(U), _f64(hcol)
    out = np.empty(U.shape[0])
    lib().orc_project(U.shape[0], U.shape[1], _d(U), _d(hcol), _d(out))
    return out


def cg(prm, U, x, w, y0):
    U, x, w = _f64(U), _f64(x), _f64(w)
    y = _f64(y0).copy()
    tr = OrcTrace()
    rc = lib().orc_cg(C.byref(prm), _d(U), _d(x), _d(w), _d(y), C.byref(tr))
    if rc:
        raise RuntimeError(f"orc_cg failed: {rc}")
    return y, tr


def grassmann_step(prm, U, y, eta_, t):
    Un = _f64(U).copy()
    tr = OrcTrace()
    rc = lib().orc_grassmann_step(C.byref(prm), _d(Un), _d(_f64(y)), _d(_f64(eta_)),
                                  float(t), C.byref(tr))
    if rc:
        raise RuntimeError(f"orc_grassmann_step failed: {rc}")
    return Un, tr


def labels(prm, U, y, x):
    lab = np.empty(_P(prm), dtype=np.uint8)
    mx = np.empty(_P(prm))
    n = lib().orc_labels(C.byref(prm), _d(_f64(U)), _d(_f64(y)), _d(_f64(x)), _u8(lab), _d(mx))
    return lab, mx, int(n)


def reorthonormalize(U, y=None):
    Un = _f64(U).copy()
    yn = None if y is None else _f64(y).copy()
    rc = lib().orc_reorthonormalize(Un.shape[0], Un.shape[1], _d(Un),
                                    None if yn is None else _d(yn))
    if rc:
        raise RuntimeError(f"orc_reorthonormalize failed: {rc}")
    return Un, yn


@dataclass
class OracleState:
    """pROST state between frames: subspace, coefficients, previous labels, frame counter."""
    U: np.ndarray
    y: np.ndarray
    labels: np.ndarray
    i: int = 0

    def copy(self):
        return OracleState(self.U.copy(), self.y.copy(), self.labels.copy(), self.i)


@dataclass
class StepResult:
    trace: OrcTrace
    residual: np.ndarray | None = None
    labels: np.ndarray | None = None
    extra: dict = field(default_factory=dict)


def frame_step(prm, state: OracleState, frame, want_residual=True) -> StepResult:
    """Advance ``state`` by one frame in place (Steps 1-3); returns the trace."""
    frame = np.ascontiguousarray(frame)
    dt = {np.dtype(np.uint8): FRAME_U8, np.dtype(np.float32): FRAME_F32,
          np.dtype(np.float64): FRAME_F64}[frame.dtype]
    assert frame.size == _m(prm)
    assert state.U.shape == (_m(prm), prm.k) and state.U.flags.c_contiguous
    tr = OrcTrace()
    res = np.empty(_m(prm)) if want_residual else None
    rc = lib().orc_frame_step(C.byref(prm), _d(state.U), _d(state.y), _u8(state.labels),
                              int(state.i), frame.ctypes.data_as(C.c_void_p), dt,
                              C.byref(tr), None if res is None else _d(res))
    if rc:
        raise RuntimeError(f"orc_frame_step failed: {rc}")
    state.i += 1
    return StepResult(tr, res, state.labels.copy())


def initial_state(U0, P) -> OracleState:
    U0 = _f64(U0).copy()
    return OracleState(U0, np.zeros(U0.shape[1]), np.zeros(P, dtype=np.uint8), 0)
