"""ctypes binding of the C ABI in ``include/pml.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls.  Pointers are passed
as plain integers (``tensor.data_ptr()`` for device memory, numpy ``ctypes.data`` for
host memory).  There is no fallback: if ``libpml.so`` has not been built, loading
fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpml.so")

PML_OK = 0
PML_EINVAL = 1
PML_ENOMEM = 2
PML_ECUDA = 3
PML_ESTATE = 4
PML_EUNSTABLE = 5
PML_ENONFINITE = 6
PML_ETIMEOUT = 7

PML_SIGMA_CONSTANT = 0
PML_SIGMA_POWER = 1
PML_SIGMA_RANDOM = 2
PML_SIGMA_USER = 3

PML_FLAG_ADJOINT = 1
PML_FLAG_WALL = 2

PML_FIELD_U = 0
PML_FIELD_V = 1


def PML_FIELD_PHI(a):
    return 2 + 2 * a


def PML_FIELD_PSI(a):
    return 3 + 2 * a


# every symbol the header declares (checked by the CPU test suite)
EXPORTED = (
    "pml_workspace_bytes", "pml_create", "pml_set_initial", "pml_set_sources",
    "pml_set_receivers", "pml_step", "pml_read_field", "pml_norms", "pml_get_step", "pml_sync",
    "pml_set_check_interval", "pml_set_wait_limit",
    "pml_query_layout", "pml_query_sigma", "pml_plan_layer_items", "pml_adjoint_reset", "pml_adjoint_step",
    "pml_adjoint_read_field", "pml_sigma_gradient", "pml_sigma_gradient_bytes", "pml_state_bytes", "pml_save_state", "pml_load_state",
    "pml_get_variant", "pml_set_variant", "pml_get_time_block", "pml_autotune",
    "pml_profile_enable", "pml_profile_read", "pml_norms_dense_static",
    "pml_batch_create", "pml_batch_step", "pml_batch_get_variant", "pml_batch_set_variant",
    "pml_batch_get_time_block",
    "pml_batch_autotune", "pml_batch_profile_enable", "pml_batch_profile_read", "pml_batch_info",
    "pml_batch_destroy", "pml_residual_factor", "pml_design_width", "pml_fma_peak", "pml_destroy", "pml_last_error", "pml_status_string",
)


class pml_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int64 * 3)]


class pml_sigma_profile(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("sigma_max", ctypes.c_double), ("order", ctypes.c_double),
                ("user", ctypes.c_void_p * 3)]


class PMLError(RuntimeError):
    def __init__(self, status, text):
        super().__init__("pml status %d: %s" % (status, text))
        self.status = status


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libpml.so (built by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libpml.so is not built (%s); run `python -c \"import __graft_entry__ as g; "
                           "g.build()\"` first" % p)
    lib = ctypes.CDLL(p)
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    st = ctypes.c_int
    sig = {
        "pml_workspace_bytes": [ctypes.POINTER(pml_grid), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_size_t)],
        "pml_create": [ctypes.POINTER(pml_grid), ctypes.c_double, ctypes.c_double, ctypes.c_int,
                       ctypes.POINTER(pml_sigma_profile), ctypes.c_int, P, P, ctypes.c_size_t,
                       ctypes.c_int, ctypes.POINTER(P)],
        "pml_set_initial": [P, P, P, ctypes.c_int],
        "pml_set_sources": [P, ctypes.c_int, P, P, ctypes.c_double, ctypes.c_double],
        "pml_set_receivers": [P, ctypes.c_int, P, P, i64],
        "pml_step": [P, i64],
        "pml_read_field": [P, ctypes.c_int, P, ctypes.c_int],
        "pml_norms": [P, P, P],
        "pml_get_step": [P, ctypes.POINTER(i64)],
        "pml_sync": [P],
        "pml_set_check_interval": [P, i64],
        "pml_set_wait_limit": [P, ctypes.c_uint64],
        "pml_query_layout": [P, ctypes.c_int, P, P, P],
        "pml_plan_layer_items": [ctypes.POINTER(pml_grid), ctypes.c_int, ctypes.POINTER(pml_sigma_profile),
                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_int64,
                                 ctypes.POINTER(ctypes.c_int64)],
        "pml_query_sigma": [P, ctypes.c_int, P],
        "pml_adjoint_reset": [P],
        "pml_adjoint_step": [P, i64, P, P, P],
        "pml_adjoint_read_field": [P, ctypes.c_int, P, ctypes.c_int],
        "pml_sigma_gradient": [P, i64, P, P, i64, P, P, P],
        "pml_sigma_gradient_bytes": [P, i64, i64, ctypes.POINTER(ctypes.c_size_t)],
        "pml_state_bytes": [P, ctypes.POINTER(ctypes.c_size_t)],
        "pml_save_state": [P, P, ctypes.c_int],
        "pml_load_state": [P, P, ctypes.c_int],
        "pml_profile_enable": [P, ctypes.c_int],
        "pml_get_variant": [P, P, P],
        "pml_set_variant": [P, ctypes.c_int],
        "pml_get_time_block": [P, P],
        "pml_autotune": [P, ctypes.c_int, P, P],
        "pml_norms_dense_static": [ctypes.c_int, P, ctypes.c_int, P, P, P, P, ctypes.c_double, P, P, P],
        "pml_profile_read": [P, P, P],
        "pml_batch_create": [ctypes.c_int, P, ctypes.POINTER(P)],
        "pml_batch_step": [P, i64],
        "pml_batch_get_variant": [P, P, P],
        "pml_batch_set_variant": [P, ctypes.c_int],
        "pml_batch_get_time_block": [P, P],
        "pml_batch_autotune": [P, ctypes.c_int, P, P],
        "pml_batch_profile_enable": [P, ctypes.c_int],
        "pml_batch_profile_read": [P, P, P],
        "pml_batch_info": [P, P],
        "pml_residual_factor": [ctypes.c_int, P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, P],
        "pml_fma_peak": [ctypes.c_int, P, i64, P, P],
        "pml_design_width": [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = st
    lib.pml_batch_destroy.argtypes = [P]
    lib.pml_batch_destroy.restype = None
    lib.pml_destroy.argtypes = [P]
    lib.pml_destroy.restype = None
    lib.pml_last_error.argtypes = [P]
    lib.pml_last_error.restype = ctypes.c_char_p
    lib.pml_status_string.argtypes = [ctypes.c_int]
    lib.pml_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status, ctx=None):
    if status != PML_OK:
        txt = load().pml_last_error(ctx)
        raise PMLError(status, txt.decode() if txt else "")
    return status


# ---- one Python function per C entry point -------------------------------------------

def pml_workspace_bytes(ndim, n, pml_width, precision, flags=0) -> int:
    g = pml_grid(ndim, (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - len(n)))))
    out = ctypes.c_size_t(0)
    _check(load().pml_workspace_bytes(ctypes.byref(g), int(pml_width), int(precision), int(flags),
                                      ctypes.byref(out)))
    return int(out.value)


def pml_create(ndim, n, h, dt, pml_width, kind, sigma_max, order, user, precision, stream,
               workspace, workspace_bytes, flags=0):
    """user: sequence of host pointers (int) or None per axis."""
    g = pml_grid(ndim, (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - len(n)))))
    u = [None, None, None]
    if user is not None:
        for a, p in enumerate(user):
            u[a] = p
    prof = pml_sigma_profile(int(kind), float(sigma_max), float(order), (ctypes.c_void_p * 3)(*u))
    ctx = ctypes.c_void_p(0)
    _check(load().pml_create(ctypes.byref(g), float(h), float(dt), int(pml_width), ctypes.byref(prof),
                             int(precision), stream, workspace, int(workspace_bytes), int(flags),
                             ctypes.byref(ctx)))
    return ctx.value


def pml_set_initial(ctx, u0, v0, on_device):
    _check(load().pml_set_initial(ctx, u0, v0, int(on_device)), ctx)


def pml_set_sources(ctx, ns, coords, amp, f_peak, t_delay):
    _check(load().pml_set_sources(ctx, int(ns), coords, amp, float(f_peak), float(t_delay)), ctx)


def pml_set_receivers(ctx, nr, coords, trace_buf, capacity):
    _check(load().pml_set_receivers(ctx, int(nr), coords, trace_buf, int(capacity)), ctx)


def pml_step(ctx, n):
    _check(load().pml_step(ctx, int(n)), ctx)


def pml_read_field(ctx, field, dst, on_device):
    _check(load().pml_read_field(ctx, int(field), dst, int(on_device)), ctx)


def pml_norms(ctx, ref, out):
    _check(load().pml_norms(ctx, ref, out), ctx)


def pml_get_step(ctx) -> int:
    v = ctypes.c_int64(0)
    _check(load().pml_get_step(ctx, ctypes.byref(v)), ctx)
    return int(v.value)


def pml_sync(ctx):
    _check(load().pml_sync(ctx), ctx)


def pml_set_check_interval(ctx, steps):
    _check(load().pml_set_check_interval(ctx, int(steps)), ctx)


def pml_set_wait_limit(ctx, ns):
    _check(load().pml_set_wait_limit(ctx, int(ns)), ctx)


def pml_plan_layer_items(ndim, n, pml_width, kind, sigma_max, order, user, precision, flags, sm_count, which):
    """Layer work items of a box (host only, no context): an int32 array [count][10] of
    x0, y0, z0, xlo, xhi, ylo, yhi, zlo, zhi, flags.  user: host pointers (int) or None."""
    import numpy as np
    g = pml_grid(ndim, (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - len(n)))))
    u = [None, None, None]
    if user is not None:
        for a, p in enumerate(user):
            u[a] = p
    prof = pml_sigma_profile(int(kind), float(sigma_max), float(order), (ctypes.c_void_p * 3)(*u))
    count = ctypes.c_int64(0)
    args = (ctypes.byref(g), int(pml_width), ctypes.byref(prof), int(precision), int(flags), int(sm_count),
            int(which))
    _check(load().pml_plan_layer_items(*args, None, 0, ctypes.byref(count)))
    out = np.zeros((max(count.value, 1), 10), dtype=np.int32)
    _check(load().pml_plan_layer_items(*args, out.ctypes.data, int(count.value), ctypes.byref(count)))
    return out[:count.value]


def pml_query_layout(ctx, axis, phi, psi, interior):
    _check(load().pml_query_layout(ctx, int(axis), phi, psi, interior), ctx)


def pml_query_sigma(ctx, axis, out):
    _check(load().pml_query_sigma(ctx, int(axis), out), ctx)


def pml_adjoint_reset(ctx):
    _check(load().pml_adjoint_reset(ctx), ctx)


def pml_adjoint_step(ctx, n, residual, grad_u, grad_amp):
    _check(load().pml_adjoint_step(ctx, int(n), residual, grad_u, grad_amp), ctx)


def pml_adjoint_read_field(ctx, field, dst, on_device):
    _check(load().pml_adjoint_read_field(ctx, int(field), dst, int(on_device)), ctx)


def pml_sigma_gradient(ctx, n, target, residual, interval, grad_sigma, grad_amp=None):
    """Runs n forward steps and the adjoint; fills grad_sigma (numpy float64, sum of T[a])
    and grad_amp (numpy float64 [ns] or None); returns the misfit J (0 with a residual)."""
    J = ctypes.c_double(0.0)
    _check(load().pml_sigma_gradient(ctx, int(n), target, residual, int(interval), grad_sigma.ctypes.data,
                                     ctypes.byref(J), None if grad_amp is None else grad_amp.ctypes.data), ctx)
    return float(J.value)


def pml_sigma_gradient_bytes(ctx, n, interval=0) -> int:
    v = ctypes.c_size_t(0)
    _check(load().pml_sigma_gradient_bytes(ctx, int(n), int(interval), ctypes.byref(v)), ctx)
    return int(v.value)


def pml_state_bytes(ctx) -> int:
    v = ctypes.c_size_t(0)
    _check(load().pml_state_bytes(ctx, ctypes.byref(v)), ctx)
    return int(v.value)


def pml_save_state(ctx, dst, on_device):
    _check(load().pml_save_state(ctx, dst, int(on_device)), ctx)


def pml_load_state(ctx, src, on_device):
    _check(load().pml_load_state(ctx, src, int(on_device)), ctx)


def pml_get_variant(ctx):
    """Returns (current variant, number of variants)."""
    v = ctypes.c_int(0)
    n = ctypes.c_int(0)
    _check(load().pml_get_variant(ctx, ctypes.byref(v), ctypes.byref(n)), ctx)
    return int(v.value), int(n.value)


def pml_set_variant(ctx, variant):
    _check(load().pml_set_variant(ctx, int(variant)), ctx)


def pml_get_time_block(ctx):
    """Steps per pass of the current variant (1, or 2 for a two-step variant)."""
    d = ctypes.c_int(0)
    _check(load().pml_get_time_block(ctx, ctypes.byref(d)), ctx)
    return int(d.value)


def pml_autotune(ctx, steps):
    """Returns (chosen variant, per-variant ms per step)."""
    import numpy as np
    _, n = pml_get_variant(ctx)
    times = np.zeros(n, dtype=np.float64)
    ch = ctypes.c_int(0)
    _check(load().pml_autotune(ctx, int(steps), times.ctypes.data, ctypes.byref(ch)), ctx)
    return int(ch.value), times


def pml_profile_enable(ctx, enable):
    _check(load().pml_profile_enable(ctx, int(enable)), ctx)


def pml_profile_read(ctx):
    """Returns (ms[3], launches[3]) for kinds interior, layer, point kernels."""
    import numpy as np
    ms = np.zeros(3, dtype=np.float64)
    n = np.zeros(3, dtype=np.int64)
    _check(load().pml_profile_read(ctx, ms.ctypes.data, n.ctypes.data), ctx)
    return ms, n


def pml_norms_dense_static(ndim, T, precision, U, V, wlo, whi, h, ref, stream):
    """Energy and norms of dense device arrays U, V (pointers) over the inclusive window
    wlo..whi, with no device allocation.  Returns a numpy array of 5 doubles."""
    import numpy as np
    Ta = np.ascontiguousarray(list(T) + [1] * (3 - len(T)), dtype=np.int64)
    lo = np.ascontiguousarray(list(wlo) + [0] * (3 - len(wlo)), dtype=np.int64)
    hi = np.ascontiguousarray(list(whi) + [0] * (3 - len(whi)), dtype=np.int64)
    out = np.zeros(5, dtype=np.float64)
    _check(load().pml_norms_dense_static(int(ndim), Ta.ctypes.data, int(precision), U, V, lo.ctypes.data,
                                         hi.ctypes.data, float(h), ref, stream, out.ctypes.data))
    return out


def pml_batch_create(ctxs):
    """Batch of 2D contexts (a list of context handles); returns the batch handle."""
    arr = (ctypes.c_void_p * len(ctxs))(*ctxs)
    out = ctypes.c_void_p(0)
    _check(load().pml_batch_create(len(ctxs), arr, ctypes.byref(out)))
    return out.value


def pml_batch_step(batch, n):
    _check(load().pml_batch_step(batch, int(n)))


def pml_batch_get_variant(batch):
    """Returns (current variant, number of variants)."""
    v = ctypes.c_int(0)
    n = ctypes.c_int(0)
    _check(load().pml_batch_get_variant(batch, ctypes.byref(v), ctypes.byref(n)))
    return int(v.value), int(n.value)


def pml_batch_set_variant(batch, variant):
    _check(load().pml_batch_set_variant(batch, int(variant)))


def pml_batch_get_time_block(b):
    """Steps per pass of the batch's current variant (1 or 2)."""
    d = ctypes.c_int(0)
    _check(load().pml_batch_get_time_block(b, ctypes.byref(d)))
    return int(d.value)


def pml_batch_autotune(batch, steps):
    """Returns (chosen variant, per-variant ms per step)."""
    import numpy as np
    _, n = pml_batch_get_variant(batch)
    times = np.zeros(n, dtype=np.float64)
    ch = ctypes.c_int(0)
    _check(load().pml_batch_autotune(batch, int(steps), times.ctypes.data, ctypes.byref(ch)))
    return int(ch.value), times


def pml_batch_profile_enable(batch, enable):
    _check(load().pml_batch_profile_enable(batch, int(enable)))


def pml_batch_profile_read(batch):
    """Returns (ms[2], launches[2]) for kinds interior, layer."""
    import numpy as np
    ms = np.zeros(2, dtype=np.float64)
    n = np.zeros(2, dtype=np.int64)
    _check(load().pml_batch_profile_read(batch, ms.ctypes.data, n.ctypes.data))
    return ms, n


def pml_batch_info(batch):
    """Returns (grids, interior work items, layer tiles, interior CTAs)."""
    import numpy as np
    info = np.zeros(4, dtype=np.int64)
    _check(load().pml_batch_info(batch, info.ctypes.data))
    return tuple(int(x) for x in info)


def pml_batch_destroy(batch):
    load().pml_batch_destroy(batch)


def pml_residual_factor(sigma_h, kh, omega_h, backed=False):
    """Residual-wave amplitude factor of one pass through the edges sigma_h (sigma * h)."""
    import numpy as np
    s = np.ascontiguousarray(sigma_h, dtype=np.float64)
    out = ctypes.c_double(0.0)
    kh = complex(kh)
    _check(load().pml_residual_factor(int(s.shape[0]), s.ctypes.data if s.size else None, kh.real, kh.imag,
                                      float(omega_h), int(bool(backed)), ctypes.byref(out)))
    return float(out.value)


def pml_design_width(kind, sigma_max_h, order, cos_min, omega_h_max, eps, backed=False, w_max=512):
    """(smallest width meeting eps or -1, largest factor of the sweep at that width)."""
    w = ctypes.c_int(0)
    worst = ctypes.c_double(0.0)
    _check(load().pml_design_width(int(kind), float(sigma_max_h), float(order), float(cos_min), float(omega_h_max),
                                   float(eps), int(bool(backed)), int(w_max), ctypes.byref(w), ctypes.byref(worst)))
    return int(w.value), float(worst.value)


def pml_fma_peak(precision, stream, iters):
    """(TFLOP/s, ms) of the library's FMA-throughput kernel in FP32 or FP64."""
    tf = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    _check(load().pml_fma_peak(int(precision), stream, int(iters), ctypes.byref(tf), ctypes.byref(ms)))
    return float(tf.value), float(ms.value)


def pml_destroy(ctx):
    load().pml_destroy(ctx)


def pml_last_error(ctx) -> str:
    t = load().pml_last_error(ctx)
    return t.decode() if t else ""


def pml_status_string(status) -> str:
    return load().pml_status_string(int(status)).decode()
