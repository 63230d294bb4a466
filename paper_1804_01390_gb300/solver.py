"""Torch-facing wrapper of the C ABI: device memory and streams come from PyTorch.

``PMLSolver`` owns one ``pml_ctx``.  Its workspace is a torch ``uint8`` tensor on the
solver's device, the stream is a torch CUDA stream, and fields are returned as torch
tensors shaped like the padded box in numpy order ([T2][T1][T0], x fastest).  All
arithmetic runs in the library's kernels; this module only marshals arguments.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

_KINDS = {"constant": _lib.PML_SIGMA_CONSTANT, "power": _lib.PML_SIGMA_POWER,
          "quadratic": _lib.PML_SIGMA_POWER, "random": _lib.PML_SIGMA_RANDOM,
          "user": _lib.PML_SIGMA_USER}


def _host_ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class PMLSolver:
    """Discrete PML solver (eq:DiscretePML + RK4) on the periodic box N + 2w.

    Parameters mirror ``pml_create``: ``N`` interior vertices per axis (2 or 3 axes),
    layer width ``w``, spacing ``h``, step ``dt``, damping profile ``sigma`` (one of
    "constant", "quadratic"/"power", "random", "user"), ``precision`` 32 or 64.
    ``draws`` (random) or ``user_sigma`` (user) are per-axis host arrays of length T.
    ``wall=True`` ends every axis with a reflecting wall instead of the periodic wrap.
    """

    def __init__(self, N, w, h=1.0, dt=0.5, sigma="quadratic", sigma_max=2.0, order=2.0,
                 draws=None, user_sigma=None, precision=32, device=None, stream=None,
                 adjoint=False, wall=False):
        self.N = tuple(int(n) for n in N)
        self.ndim = len(self.N)
        self.w = int(w)
        self.T = tuple(n + 2 * self.w for n in self.N)
        self.h = float(h)
        self.dt = float(dt)
        self.precision = int(precision)
        self.dtype = torch.float32 if self.precision == 32 else torch.float64
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.type != "cuda":
            raise ValueError("PMLSolver runs on CUDA devices only")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        kind = _KINDS[sigma]
        user = None
        self._keep = []
        if kind in (_lib.PML_SIGMA_RANDOM, _lib.PML_SIGMA_USER):
            src = draws if kind == _lib.PML_SIGMA_RANDOM else user_sigma
            if src is None or len(src) != self.ndim:
                raise ValueError("sigma=%r needs one array per axis" % sigma)
            user = []
            for a, arr in enumerate(src):
                arr = np.ascontiguousarray(arr, dtype=np.float64)
                assert arr.shape == (self.T[a],)
                self._keep.append(arr)
                user.append(_host_ptr(arr))
        flags = (_lib.PML_FLAG_ADJOINT if adjoint else 0) | (_lib.PML_FLAG_WALL if wall else 0)
        self.wall = bool(wall)
        nbytes = _lib.pml_workspace_bytes(self.ndim, self.N, self.w, self.precision, flags)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.ctx = _lib.pml_create(self.ndim, self.N, self.h, self.dt, self.w, kind, sigma_max, order,
                                   user, self.precision, self.stream.cuda_stream,
                                   self.workspace.data_ptr(), nbytes, flags)
        self.adjoint = adjoint
        self.ns = 0
        self.nr = 0
        self.traces = None

    # -- lifecycle -----------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            _lib.pml_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return self.T[::-1]

    def _dense(self, x):
        if isinstance(x, np.ndarray):
            x = torch.from_numpy(x)
        x = x.to(self.dtype)
        if x.device.type == "cuda":
            x = x.to(self.device).contiguous()
        else:
            x = x.contiguous()
        assert tuple(x.shape) == self.shape, (tuple(x.shape), self.shape)
        return x

    # -- state ---------------------------------------------------------------------
    def set_initial(self, u0, v0=None):
        u = self._dense(u0)
        v = self._dense(v0) if v0 is not None else None
        on_dev = u.device.type == "cuda"
        if v is not None and (v.device.type == "cuda") != on_dev:
            v = v.to(u.device)
        self._init_keep = (u, v)
        _lib.pml_set_initial(self.ctx, u.data_ptr(), v.data_ptr() if v is not None else None, on_dev)

    def set_sources(self, coords, amp, f_peak, t_delay):
        c = np.ascontiguousarray(np.asarray(coords, dtype=np.int64).reshape(-1, self.ndim))
        a = np.ascontiguousarray(np.asarray(amp, dtype=np.float64).reshape(-1))
        self.ns = int(a.shape[0])
        _lib.pml_set_sources(self.ctx, self.ns, _host_ptr(c) if self.ns else None,
                             _host_ptr(a) if self.ns else None, f_peak, t_delay)

    def set_receivers(self, coords, capacity):
        c = np.ascontiguousarray(np.asarray(coords, dtype=np.int64).reshape(-1, self.ndim))
        self.nr = int(c.shape[0])
        self.traces = torch.zeros((int(capacity), self.nr), dtype=self.dtype, device=self.device)
        _lib.pml_set_receivers(self.ctx, self.nr, _host_ptr(c), self.traces.data_ptr(), int(capacity))
        return self.traces

    def step(self, n=1):
        _lib.pml_step(self.ctx, int(n))

    @property
    def step_count(self):
        return _lib.pml_get_step(self.ctx)

    def sync(self):
        _lib.pml_sync(self.ctx)

    def set_check_interval(self, steps):
        """Scan U and V for non-finite values every `steps` steps (0: off)."""
        _lib.pml_set_check_interval(self.ctx, int(steps))

    def set_wait_limit(self, ns):
        """Limit of every bounded device wait in nanoseconds (0: the default)."""
        _lib.pml_set_wait_limit(self.ctx, int(ns))

    def read(self, field=0, out=None):
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device=self.device)
        _lib.pml_read_field(self.ctx, int(field), out.data_ptr(), out.device.type == "cuda")
        return out

    def norms(self, ref=None):
        """Energy eq:Energy, max|U|, ||U||, ||U-ref||, max|U-ref| over the physical window."""
        out = np.zeros(5, dtype=np.float64)
        r = None
        if ref is not None:
            ref = ref.to(device=self.device, dtype=torch.float64).contiguous()
            assert tuple(ref.shape) == self.N[::-1]
            r = ref.data_ptr()
        _lib.pml_norms(self.ctx, r, _host_ptr(out))
        return {"energy": out[0], "max": out[1], "l2": out[2], "diff_l2": out[3], "diff_max": out[4]}

    def layout(self, axis):
        T = self.T[axis]
        phi = np.zeros(T, np.uint8)
        psi = np.zeros(T, np.uint8)
        inner = np.zeros(T, np.uint8)
        _lib.pml_query_layout(self.ctx, axis, _host_ptr(phi), _host_ptr(psi), _host_ptr(inner))
        return phi, psi, inner

    def sigma(self, axis):
        out = np.zeros(self.T[axis], np.float64)
        _lib.pml_query_sigma(self.ctx, axis, _host_ptr(out))
        return out

    # -- adjoint -------------------------------------------------------------------
    def adjoint_reset(self):
        _lib.pml_adjoint_reset(self.ctx)

    def adjoint_step(self, n, residual=None, want_grad_u=True):
        """Reverse n steps; residual: device tensor [n, nr] (row k = step clock-k)."""
        res = None
        if residual is not None:
            residual = residual.to(device=self.device, dtype=self.dtype).contiguous()
            assert tuple(residual.shape) == (int(n), self.nr)
            res = residual.data_ptr()
        gu = torch.empty(self.shape, dtype=self.dtype, device=self.device) if want_grad_u else None
        ga = np.zeros(max(self.ns, 1), dtype=np.float64)
        _lib.pml_adjoint_step(self.ctx, int(n), res, gu.data_ptr() if gu is not None else None,
                              _host_ptr(ga) if self.ns else None)
        return gu, (ga[: self.ns] if self.ns else None)

    def adjoint_read(self, field=0):
        out = torch.empty(self.shape, dtype=self.dtype, device=self.device)
        _lib.pml_adjoint_read_field(self.ctx, int(field), out.data_ptr(), True)
        return out

    def sigma_gradient(self, n, target=None, residual=None, interval=0):
        """Runs n steps from the current state; returns (J, [dJ/dsigma_a per axis],
        dJ/da or None) for J = 1/2 sum (U_m(x_r) - target[m-1, r])^2, or for the misfit
        whose trace gradient is `residual` (then J is 0) (pml_sigma_gradient)."""
        g = np.zeros(int(sum(self.T)), dtype=np.float64)
        ga = np.zeros(max(self.ns, 1), dtype=np.float64) if self.ns else None
        args = []
        for a in (target, residual):   # device copies in the context precision, kept alive
            if a is not None:
                a = a.to(device=self.device, dtype=self.dtype).contiguous()
                assert tuple(a.shape) == (int(n), self.nr)
            args.append(a)
        ptr = [None if a is None else a.data_ptr() for a in args]
        J = _lib.pml_sigma_gradient(self.ctx, int(n), ptr[0], ptr[1], int(interval), g, ga)
        out, off = [], 0
        for t in self.T:
            out.append(g[off:off + t].copy())
            off += t
        return J, out, ga

    # -- checkpoints -----------------------------------------------------------------
    def state_bytes(self):
        return _lib.pml_state_bytes(self.ctx)

    def save_state(self, dst=None):
        if dst is None:
            dst = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        _lib.pml_save_state(self.ctx, dst.data_ptr(), dst.device.type == "cuda")
        return dst

    def load_state(self, src):
        _lib.pml_load_state(self.ctx, src.data_ptr(), src.device.type == "cuda")


class PMLBatch:
    """Many independent 2D solvers advanced together (``pml_batch_*``).

    All solvers must be 2D, of one precision and on one stream; they keep working on
    their own between batch steps (``read``, ``norms``, ``step``).  The batch holds
    references to them so that they outlive it.
    """

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.handle = _lib.pml_batch_create([s.ctx for s in self.solvers])

    def close(self):
        if getattr(self, "handle", None):
            _lib.pml_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        _lib.pml_batch_step(self.handle, int(n))

    @property
    def variant(self):
        return _lib.pml_batch_get_variant(self.handle)[0]

    @property
    def variant_count(self):
        return _lib.pml_batch_get_variant(self.handle)[1]

    def time_block(self):
        """Steps per pass of the current variant (1, or 2 for a two-step shape)."""
        return _lib.pml_batch_get_time_block(self.handle)

    def set_variant(self, v):
        _lib.pml_batch_set_variant(self.handle, int(v))

    def autotune(self, steps):
        return _lib.pml_batch_autotune(self.handle, int(steps))

    def profile(self, enable=True):
        _lib.pml_batch_profile_enable(self.handle, int(enable))

    def profile_read(self):
        return _lib.pml_batch_profile_read(self.handle)

    def info(self):
        return _lib.pml_batch_info(self.handle)
