"""Python binding of libprost (include/prost.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Buffers may be
torch tensors (device or host) or numpy arrays (host); ``on_device`` is taken
from the tensors.  Negative return codes raise :class:`ProstError`, except
the frame status PROST_EBADFRAME, which prost_step() and prost_sync() return.
The library is built in-tree on first use; without it every call fails.
"""

from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import build as _build

PROST_OK, PROST_EINVAL, PROST_ENOMEM, PROST_ECUDA = 0, -1, -2, -3
PROST_EBADFRAME, PROST_ETIMEOUT, PROST_ENOTSPD = -4, -5, -6
PROST_U8, PROST_F32, PROST_BF16 = 0, 1, 2
PROST_MASK_POST_UPDATE, PROST_MASK_PRE_UPDATE = 0, 1
PROST_MAX_K, PROST_MAX_K_SINGLE, PROST_STATIC_MAX_K, PROST_MAX_CG = 32, 16, 16, 32
PROST_FORM_AUTO, PROST_FORM_GRID, PROST_FORM_CLUSTER, PROST_FORM_PASSES, PROST_FORM_RESIDENT = 0, 1, 2, 3, 4
PROST_CLUSTER_MAX_U_BYTES = 1 << 20

HEADER = os.path.join(_build.INCLUDE, "prost.h")


class ProstError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class prost_params(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("channels", C.c_int32),
                ("k", C.c_int32), ("p", C.c_double), ("mu", C.c_double), ("delta", C.c_double),
                ("omega", C.c_double), ("t_init", C.c_double), ("t_min", C.c_double),
                ("i_init", C.c_int32), ("n_cg", C.c_int32), ("in_scale", C.c_double),
                ("in_offset", C.c_double), ("frame_dtype", C.c_int32), ("u_dtype", C.c_int32),
                ("mask_from", C.c_int32), ("form", C.c_int32), ("seed", C.c_uint64)]


class prost_stats(C.Structure):
    _fields_ = [("frames", C.c_int64), ("bad_frames", C.c_int64), ("n_cg", C.c_int32),
                ("status", C.c_int32), ("cost", C.c_double * (PROST_MAX_CG + 1)),
                ("gnorm", C.c_double * (PROST_MAX_CG + 1)), ("alpha", C.c_double * PROST_MAX_CG),
                ("beta", C.c_double * (PROST_MAX_CG + 1)), ("pi_norm", C.c_double),
                ("y_norm", C.c_double), ("sigma", C.c_double), ("t", C.c_double),
                ("theta", C.c_double), ("updated", C.c_int32), ("pad0", C.c_int32),
                ("n_foreground", C.c_int64), ("orth_err", C.c_double),
                ("eta_norm", C.c_double), ("pi_explicit", C.c_int32), ("form", C.c_int32)]


_lib = None


def lib():
    """The loaded library (built in-tree if missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, sz = C.c_void_p, C.c_size_t
        P = C.POINTER
        L.prost_state_bytes.argtypes = [P(prost_params), P(sz)]
        L.prost_init.argtypes = [P(prost_params), vp, P(vp)]
        L.prost_step.argtypes = [vp, vp, C.c_int, vp, vp]
        L.prost_step_many.argtypes = [vp, vp, C.c_int32, C.c_int, vp]
        L.prost_step_many_async.argtypes = [vp, vp, C.c_int32, vp]
        L.prost_sync.argtypes = [vp]
        L.prost_step_async.argtypes = [vp, vp, vp, vp]
        L.prost_wait.argtypes = [vp]
        L.prost_inject_barrier_skew.argtypes = [vp, C.c_int64]
        L.prost_inject_wait_timeout.argtypes = [vp, C.c_int32, C.c_int64]
        L.prost_get_subspace.argtypes = [vp, vp, vp, C.c_int]
        L.prost_set_subspace.argtypes = [vp, vp, vp, C.c_int]
        L.prost_set_labels.argtypes = [vp, vp, C.c_int]
        L.prost_set_frame_index.argtypes = [vp, C.c_int64]
        L.prost_get_stats.argtypes = [vp, P(prost_stats)]
        L.prost_get_state.argtypes = [vp, vp, P(sz)]
        L.prost_set_state.argtypes = [vp, vp, sz]
        L.prost_set_timing.argtypes = [vp, C.c_int]
        L.prost_get_timing.argtypes = [vp, P(C.c_float), P(C.c_int)]
        L.prost_get_trace.argtypes = [vp, P(C.c_uint64)]
        L.prost_cost_grad_static.argtypes = [P(prost_params), vp, P(C.c_double), vp, vp, vp,
                                             vp, vp]
        L.prost_destroy.argtypes = [vp]
        L.prost_destroy.restype = None
        L.prost_strerror.argtypes = [C.c_int]
        L.prost_strerror.restype = C.c_char_p
        L.prost_last_error.argtypes = [vp]
        L.prost_last_error.restype = C.c_char_p
        L.prost_version.argtypes = []
        L.prost_pre_init.argtypes = [C.c_int32] * 7 + [vp, P(vp)]
        L.prost_pre_apply.argtypes = [vp, vp, C.c_int, vp]
        L.prost_pre_get_stats.argtypes = [vp, vp, P(C.c_double), P(C.c_int32)]
        L.prost_pre_get_state.argtypes = [vp, vp, P(sz)]
        L.prost_pre_set_state.argtypes = [vp, vp, sz]
        L.prost_pre_last_error.argtypes = [vp]
        L.prost_pre_last_error.restype = C.c_char_p
        L.prost_pre_destroy.argtypes = [vp]
        L.prost_pre_destroy.restype = None
        L.prost_median3x3.argtypes = [vp, vp, C.c_int32, C.c_int32, C.c_int, vp]
        L.prost_batch_init.argtypes = [P(prost_params), C.c_int32, vp, P(vp)]
        L.prost_batch_step.argtypes = [vp, P(vp), P(vp)]
        L.prost_batch_sync.argtypes = [vp]
        L.prost_batch_stream.argtypes = [vp, C.c_int32, P(vp)]
        L.prost_batch_set_graph.argtypes = [vp, C.c_int]
        L.prost_batch_set_concurrent.argtypes = [vp, C.c_int]
        L.prost_batch_get_concurrent.argtypes = [vp, P(C.c_int32)]
        L.prost_batch_tune.argtypes = [vp, P(vp), C.c_int32, P(C.c_float)]
        L.prost_batch_plan.argtypes = [vp, P(C.c_int32), P(C.c_int32), P(C.c_float), P(C.c_int32)]
        L.prost_batch_split.argtypes = [C.c_int32, C.c_int32, P(C.c_double), P(C.c_int32), P(C.c_int32)]
        L.prost_batch_last_error.argtypes = [vp]
        L.prost_batch_last_error.restype = C.c_char_p
        L.prost_batch_destroy.argtypes = [vp]
        L.prost_batch_destroy.restype = None
        L.prost_window_init.argtypes = [C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double, vp,
                                        P(vp)]
        L.prost_window_eval.argtypes = [vp] + [vp] * 10
        L.prost_window_ustep.argtypes = [vp, vp, vp, C.c_float, vp, vp]
        L.prost_window_inject_wait_timeout.argtypes = [vp, C.c_int32, C.c_int64]
        L.prost_window_last_error.argtypes = [vp]
        L.prost_window_last_error.restype = C.c_char_p
        L.prost_window_destroy.argtypes = [vp]
        L.prost_window_destroy.restype = None
        _lib = L
    return _lib


def header_functions():
    """Names of the entry points declared in include/prost.h."""
    src = open(HEADER).read()
    return sorted(set(re.findall(r"\b(prost_[a-z_]+)\s*\(", src)))


# ---- marshalling helpers ---------------------------------------------------

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)}")


def _where(*bufs):
    flags = {bool(b.is_cuda) for b in bufs if b is not None and _is_torch(b)}
    flags |= {False for b in bufs if isinstance(b, np.ndarray)}
    if len(flags) > 1:
        raise ValueError("buffers must be all on the device or all on the host")
    return 1 if flags == {True} else 0


def _check(rc, h=None, allow=()):
    if rc < 0 and rc not in allow:
        detail = lib().prost_last_error(h).decode()
        raise ProstError(rc, f"{prost_strerror(rc)}: {detail}" if detail else prost_strerror(rc))
    return rc


_DTYPES = {"u8": PROST_U8, "uint8": PROST_U8, "f32": PROST_F32, "float32": PROST_F32,
           "bf16": PROST_BF16, "bfloat16": PROST_BF16}


def make_params(width, height, channels=1, k=5, p=0.25, mu=0.0, delta=0.35, omega=5e-5,
                t_init=5e-3, t_min=1e-4, i_init=100, n_cg=5, in_scale=1.0, in_offset=0.0,
                frame_dtype="u8", u_dtype="f32", mask_from=PROST_MASK_POST_UPDATE, seed=0,
                form=PROST_FORM_AUTO, **_ignored) -> prost_params:
    fd = _DTYPES[frame_dtype] if isinstance(frame_dtype, str) else int(frame_dtype)
    ud = _DTYPES[u_dtype] if isinstance(u_dtype, str) else int(u_dtype)
    return prost_params(int(width), int(height), int(channels), int(k), float(p), float(mu),
                        float(delta), float(omega), float(t_init), float(t_min), int(i_init),
                        int(n_cg), float(in_scale), float(in_offset), fd, ud, int(mask_from), int(form),
                        int(seed))


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


# ---- the C entry points ------------------------------------------------------

def prost_version():
    return lib().prost_version()


def prost_strerror(code):
    return lib().prost_strerror(int(code)).decode()


def prost_last_error(h=None):
    return lib().prost_last_error(h).decode()


def prost_state_bytes(params):
    n = C.c_size_t()
    _check(lib().prost_state_bytes(C.byref(params), C.byref(n)))
    return n.value


def prost_init(params, stream=None):
    h = C.c_void_p()
    _check(lib().prost_init(C.byref(params), _stream_ptr(stream), C.byref(h)))
    return h


def prost_step(h, frame, mask_out=None, background_out=None):
    """Steps 1-3 for one frame; returns PROST_OK or PROST_EBADFRAME (host
    buffers: the frame's status; device buffers: PROST_OK once enqueued)."""
    od = _where(frame, mask_out, background_out)
    return _check(lib().prost_step(h, _ptr(frame), od, _ptr(mask_out), _ptr(background_out)), h,
                  allow=(PROST_EBADFRAME,))


def prost_step_many(h, frames, n, masks_out=None):
    """Steps 1-3 for n consecutive frames (frames: n * m entries, masks_out:
    n * P bytes); host buffers: the last frame's status, device buffers:
    PROST_OK once enqueued."""
    od = _where(frames, masks_out)
    return _check(lib().prost_step_many(h, _ptr(frames), int(n), od, _ptr(masks_out)), h,
                  allow=(PROST_EBADFRAME,))


def prost_step_async(h, frame, mask_out=None, background_out=None):
    """Enqueue a host frame (numpy arrays or CPU tensors, page-locked for
    overlap) and return at once; the buffers must stay alive until
    prost_wait has returned this frame."""
    for b in (frame, mask_out, background_out):
        if b is not None and _is_torch(b) and b.is_cuda:
            raise ProstError(PROST_EINVAL, "prost_step_async takes host buffers")
    return _check(lib().prost_step_async(h, _ptr(frame), _ptr(mask_out), _ptr(background_out)), h)


def prost_step_many_async(h, frames, n, masks_out=None):
    """Enqueue n host frames (numpy arrays or CPU tensors, page-locked for
    overlap) as one pipelined call and return at once; prost_wait returns
    the call's last frame's status."""
    for b in (frames, masks_out):
        if b is not None and _is_torch(b) and b.is_cuda:
            raise ProstError(PROST_EINVAL, "prost_step_many_async takes host buffers")
    return _check(lib().prost_step_many_async(h, _ptr(frames), int(n), _ptr(masks_out)), h)


def prost_wait(h):
    """Status of the oldest frame of prost_step_async (raises on errors other
    than PROST_EBADFRAME)."""
    return _check(lib().prost_wait(h), h, allow=(PROST_EBADFRAME,))


def prost_sync(h):
    return _check(lib().prost_sync(h), h, allow=(PROST_EBADFRAME,))


def prost_inject_barrier_skew(h, delta):
    """Failure-detection tests: leave the grid barrier as an aborted launch
    would (host-side injection); the next frame is refused and prost_sync
    raises PROST_ETIMEOUT, then the tracker recovers."""
    return _check(lib().prost_inject_barrier_skew(h, int(delta)), h)


def prost_inject_wait_timeout(h, pass_index, cycles):
    """Failure-detection tests: the next frame's grid barrier of residual
    pass pass_index waits for an arrival that never comes and gives up after
    `cycles` SM clock cycles (the bounded wait runs out)."""
    return _check(lib().prost_inject_wait_timeout(h, int(pass_index), int(cycles)), h)


def prost_get_subspace(h, U_out=None, y_out=None):
    od = _where(U_out, y_out)
    return _check(lib().prost_get_subspace(h, _ptr(U_out), _ptr(y_out), od), h)


def prost_set_subspace(h, U, y=None):
    od = _where(U, y)
    return _check(lib().prost_set_subspace(h, _ptr(U), _ptr(y), od), h)


def prost_set_labels(h, labels=None):
    od = _where(labels)
    return _check(lib().prost_set_labels(h, _ptr(labels), od), h)


def prost_set_frame_index(h, i):
    return _check(lib().prost_set_frame_index(h, int(i)), h)


def prost_get_stats(h):
    st = prost_stats()
    _check(lib().prost_get_stats(h, C.byref(st)), h)
    return st


def prost_get_state(h):
    n = C.c_size_t(0)
    _check(lib().prost_get_state(h, None, C.byref(n)), h)
    buf = (C.c_char * n.value)()
    _check(lib().prost_get_state(h, buf, C.byref(n)), h)
    return bytes(buf[: n.value])


def prost_set_state(h, state: bytes):
    buf = C.create_string_buffer(state, len(state))
    return _check(lib().prost_set_state(h, buf, len(state)), h)


def prost_set_timing(h, enable=True):
    return _check(lib().prost_set_timing(h, 1 if enable else 0), h)


def prost_get_timing(h):
    """Per-launch device times (ms) of the last traced frame."""
    buf = (C.c_float * (PROST_MAX_CG + 2))()
    n = C.c_int(0)
    _check(lib().prost_get_timing(h, buf, C.byref(n)), h)
    return [buf[j] for j in range(n.value)]


PROST_TRACE_LEN = PROST_MAX_CG + 13


def prost_get_trace(h):
    """Raw %globaltimer stamps (ns) of the last frame (see include/prost.h)."""
    buf = (C.c_uint64 * PROST_TRACE_LEN)()
    _check(lib().prost_get_trace(h, buf), h)
    return [int(v) for v in buf]


def prost_cost_grad_static(params, U, y, frame, labels, out, status_out=None, stream=None):
    """Cost and gradient of one frame with no device allocation (static
    library scratch); U, frame, labels, out, status_out are device tensors,
    y a sequence of k floats.  Enqueues only."""
    yk = (C.c_double * max(1, len(y)))(*[float(v) for v in y])
    return _check(lib().prost_cost_grad_static(C.byref(params), _ptr(U), yk, _ptr(frame),
                                               _ptr(labels), _ptr(out), _ptr(status_out),
                                               _stream_ptr(stream)))


def prost_destroy(h):
    if h:
        lib().prost_destroy(h)


# ---- many streams per tick ----------------------------------------------------

def _check_batch(rc, b=None):
    if rc < 0:
        detail = lib().prost_batch_last_error(b).decode()
        raise ProstError(rc, f"{prost_strerror(rc)}: {detail}" if detail else prost_strerror(rc))
    return rc


def _ptr_array(bufs):
    arr = (C.c_void_p * len(bufs))()
    for i, x in enumerate(bufs):
        arr[i] = _ptr(x)
    return arr


def prost_batch_init(params_list, stream=None):
    """A batch of streams, one prost_params each; returns the batch handle."""
    n = len(params_list)
    arr = (prost_params * n)(*params_list)
    out = C.c_void_p()
    _check_batch(lib().prost_batch_init(arr, n, _stream_ptr(stream), C.byref(out)))
    return out.value


def prost_batch_step(b, frames, masks=None):
    """One tick: frames[i] (device tensor) for stream i, masks[i] (device
    tensor of P bytes) receives its labels.  Enqueues only."""
    fa = _ptr_array(frames)
    ma = _ptr_array(masks) if masks is not None else None
    return _check_batch(lib().prost_batch_step(b, fa, ma), b)


def prost_batch_sync(b):
    return _check_batch(lib().prost_batch_sync(b), b)


def prost_batch_stream(b, i):
    h = C.c_void_p()
    _check_batch(lib().prost_batch_stream(b, int(i), C.byref(h)), b)
    return h.value


def prost_batch_set_graph(b, enable=True):
    return _check_batch(lib().prost_batch_set_graph(b, 1 if enable else 0), b)


def prost_batch_set_concurrent(b, enable=True):
    return _check_batch(lib().prost_batch_set_concurrent(b, 1 if enable else 0), b)


def prost_batch_get_concurrent(b):
    v = C.c_int32()
    _check_batch(lib().prost_batch_get_concurrent(b, C.byref(v)), b)
    return bool(v.value)


def prost_batch_tune(b, frames, ticks=5):
    """Autotune the batch plan on these frames; returns the chosen ms per tick."""
    ms = C.c_float(0.0)
    _check_batch(lib().prost_batch_tune(b, _ptr_array(frames), int(ticks), C.byref(ms)), b)
    return ms.value


def prost_batch_plan(b, n):
    """(CTAs per stream, kernel groups, alpha, graph on)."""
    ctas = (C.c_int32 * n)()
    ng, gr = C.c_int32(0), C.c_int32(0)
    al = C.c_float(0.0)
    _check_batch(lib().prost_batch_plan(b, ctas, C.byref(ng), C.byref(al), C.byref(gr)), b)
    return list(ctas), ng.value, al.value, bool(gr.value)


def prost_batch_split(budget, weights, caps):
    """The batch's split of `budget` CTAs between streams of these weights and
    caps (host only); returns the CTAs per stream."""
    n = len(weights)
    if len(caps) != n:
        raise ValueError("weights and caps differ in length")
    w = (C.c_double * max(n, 1))(*[float(x) for x in weights])
    cp = (C.c_int32 * max(n, 1))(*[int(x) for x in caps])
    out = (C.c_int32 * max(n, 1))()
    rc = lib().prost_batch_split(int(budget), n, w, cp, out)
    if rc < 0:
        raise ProstError(rc, prost_strerror(rc))
    return list(out)[:n]


def prost_batch_last_error(b=None):
    return lib().prost_batch_last_error(b).decode()


def prost_batch_destroy(b):
    if b:
        lib().prost_batch_destroy(b)


# ---- the cost over a window of frames -----------------------------------------

def _check_win(rc, w=None):
    if rc < 0:
        detail = lib().prost_window_last_error(w).decode()
        raise ProstError(rc, f"{prost_strerror(rc)}: {detail}" if detail else prost_strerror(rc))
    return rc


def prost_window_init(m, channels, k, n, p=0.25, omega=5e-5, stream=None):
    out = C.c_void_p()
    _check_win(lib().prost_window_init(int(m), int(channels), int(k), int(n), float(p), float(omega),
                                       _stream_ptr(stream), C.byref(out)))
    return out.value


def prost_window_eval(w, U, Y, X, labels, mu, cost, dU=None, dY=None, dmu=None, gscale=None):
    """Cost into cost (device float); gradients too when dU, dY, dmu are given."""
    return _check_win(lib().prost_window_eval(w, _ptr(U), _ptr(Y), _ptr(X), _ptr(labels), _ptr(mu),
                                              _ptr(gscale), _ptr(cost), _ptr(dU), _ptr(dY), _ptr(dmu)), w)


def prost_window_ustep(w, U, dU, t, U_out, status_out=None):
    return _check_win(lib().prost_window_ustep(w, _ptr(U), _ptr(dU), float(t), _ptr(U_out), _ptr(status_out)), w)


def prost_window_inject_wait_timeout(w, barrier, cycles):
    """Failure-detection tests: the next U-step's grid barrier `barrier` (1 or
    2) gives up after `cycles` SM clock cycles; that U-step reports -2."""
    return _check_win(lib().prost_window_inject_wait_timeout(w, int(barrier), int(cycles)), w)


def prost_window_last_error(w=None):
    return lib().prost_window_last_error(w).decode()


def prost_window_destroy(w):
    if w:
        lib().prost_window_destroy(w)


# ---- pre- and post-processing (Section 3.4) ---------------------------------

def _check_pre(rc, p=None):
    if rc < 0:
        detail = lib().prost_pre_last_error(p).decode()
        raise ProstError(rc, f"{prost_strerror(rc)}: {detail}" if detail else prost_strerror(rc))
    return rc


def prost_pre_init(w_in, h_in, channels, w_out, h_out, frame_dtype="u8", i_init=100, stream=None):
    """Resampling to w_out x h_out and running mean/deviation normalisation
    over the first i_init frames; returns the handle."""
    fd = _DTYPES[frame_dtype] if isinstance(frame_dtype, str) else int(frame_dtype)
    out = C.c_void_p()
    _check_pre(lib().prost_pre_init(int(w_in), int(h_in), int(channels), int(w_out), int(h_out), fd,
                                    int(i_init), _stream_ptr(stream), C.byref(out)))
    return out.value


def prost_pre_apply(p, frame, out):
    """One frame into out (channels x h_out x w_out float32), both on the
    device (enqueued) or both on the host (synchronous)."""
    return _check_pre(lib().prost_pre_apply(p, _ptr(frame), _where(frame, out), _ptr(out)), p)


def prost_pre_get_stats(p, mean_out=None):
    """(deviation, frames counted); fills mean_out (host float32) if given."""
    sd = C.c_double(0.0)
    n = C.c_int32(0)
    _check_pre(lib().prost_pre_get_stats(p, _ptr(mean_out), C.byref(sd), C.byref(n)), p)
    return sd.value, n.value


def prost_pre_get_state(p):
    """The pre-processor's running statistics as bytes (checkpoint)."""
    n = C.c_size_t(0)
    _check_pre(lib().prost_pre_get_state(p, None, C.byref(n)), p)
    buf = C.create_string_buffer(n.value)
    _check_pre(lib().prost_pre_get_state(p, buf, C.byref(n)), p)
    return buf.raw[:n.value]


def prost_pre_set_state(p, state: bytes):
    buf = C.create_string_buffer(state, len(state))
    return _check_pre(lib().prost_pre_set_state(p, buf, len(state)), p)


def prost_pre_last_error(p=None):
    return lib().prost_pre_last_error(p).decode()


def prost_pre_destroy(p):
    if p:
        lib().prost_pre_destroy(p)


def prost_median3x3(mask_in, mask_out, width, height, stream=None):
    """3 x 3 median of a binary mask (border replicated), device or host buffers."""
    return _check(lib().prost_median3x3(_ptr(mask_in), _ptr(mask_out), int(width), int(height),
                                        _where(mask_in, mask_out), _stream_ptr(stream)))


__all__ = [n for n in dir() if n.startswith(("prost_", "PROST_"))] + [
    "ProstError", "make_params", "header_functions", "lib"]
