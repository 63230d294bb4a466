"""Plain FP64 CPU oracle for the reflectionless discrete PML (arXiv 1804.01390).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The CUDA library never imports, links or calls it, and it shares no code with the
library; the only module both sides use is the seeded input generator
``paper_1804_01390_gb300.workloads`` (which holds none of the method's arithmetic).

The arithmetic lives in ``pml_oracle.c`` (plain C, FP64, ``-O2 -ffp-contract=off``);
this module compiles it with gcc and marshals numpy arrays through ctypes.  Each
function names the part of the paper it follows:

* ``sigma_profile``   -- damping coefficients sigma_a(i) >= 0, zero in the physical
                         domain (Sec. 1.1.2, text after Eq. 3; Fig. HalfSpaceGauss /
                         HalfSpaceRand profiles), edge-centred as in eq:IntroSolution.
* ``layout_axis``     -- supports of Phi / Psi (Sec. 1.1.2) and the interior run.
* ``rhs``             -- A y + b(t), eq:DiscretePML (Eq. 3a-3c) in first-order form.
* ``rk4``             -- classic RK4 (Sec. 1.1.3), stage by stage.
* ``energy``          -- eq:Energy (Sec. 1.1.5).
* ``rhs_transpose`` / ``adjoint`` -- transpose of A and the reverse of the RK4
                         stage graph (discrete adjoint of the scheme above).
* ``misfit_grad_sigma`` -- receiver misfit and its gradient with respect to every edge
                         damping sigma_a[e], from the reverse stage graph and the sigma
                         entries of eq:DiscretePML.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pml_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[bool, ctypes.CDLL] = {}

KIND_CONSTANT = 0
KIND_POWER = 1
KIND_RANDOM = 2


def _lib_path(openmp: bool) -> str:
    return os.path.join(_BUILD, "liboracle_omp.so" if openmp else "liboracle.so")


def build(force: bool = False) -> list[str]:
    """Compile the serial oracle and its OpenMP twin (same source) with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    out = []
    for openmp in (False, True):
        dst = _lib_path(openmp)
        if (not force and os.path.exists(dst)
                and os.path.getmtime(dst) >= os.path.getmtime(_SRC)):
            out.append(dst)
            continue
        tmp = dst + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-fPIC",
               "-shared", _SRC, "-o", tmp, "-lm"]
        if openmp:
            cmd.insert(1, "-fopenmp")
        subprocess.run(cmd, check=True)
        os.replace(tmp, dst)
        out.append(dst)
    return out


def _lib(openmp: bool = False) -> ctypes.CDLL:
    with _LOCK:
        if openmp in _LIBS:
            return _LIBS[openmp]
        build()
        lib = ctypes.CDLL(_lib_path(openmp))
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        dbl = ctypes.c_double
        cint = ctypes.c_int
        lib.orc_ricker.restype = dbl
        lib.orc_ricker.argtypes = [dbl, dbl, dbl]
        lib.orc_sigma_profile.restype = cint
        lib.orc_sigma_profile.argtypes = [i64, i64, cint, dbl, dbl, P, P]
        lib.orc_layout_axis.restype = None
        lib.orc_layout_axis.argtypes = [P, i64, i64, P, P, P]
        lib.orc_rhs.restype = None
        lib.orc_rhs.argtypes = [cint, P, dbl, P, P, P, cint, P, P, dbl, dbl, dbl]
        lib.orc_rk4.restype = cint
        lib.orc_rk4.argtypes = [cint, P, dbl, P, P, i64, dbl, i64, cint, P, P, dbl, dbl,
                                cint, P, P]
        lib.orc_energy.restype = dbl
        lib.orc_energy.argtypes = [cint, P, dbl, P, P, P]
        lib.orc_norms.restype = None
        lib.orc_norms.argtypes = [cint, P, P, P, P, P, P]
        lib.orc_rhs_transpose.restype = None
        lib.orc_rhs_transpose.argtypes = [cint, P, dbl, P, P, P]
        lib.orc_adjoint.restype = cint
        lib.orc_adjoint.argtypes = [cint, P, dbl, P, P, i64, dbl, i64, cint, P, dbl, dbl, P,
                                    cint, P, P]
        lib.orc_set_boundary.restype = None
        lib.orc_set_boundary.argtypes = [cint]
        lib.orc_misfit_grad_sigma.restype = cint
        lib.orc_misfit_grad_sigma.argtypes = [cint, P, dbl, P, P, i64, dbl, i64, cint, P, P, dbl,
                                              dbl, cint, P, P, P, P]
        _LIBS[openmp] = lib
        return lib


def _bc(grid, openmp=False):
    """The library to call for `grid`, with its boundary (periodic or wall) selected."""
    lib = _lib(openmp)
    lib.orc_set_boundary(int(grid.wall))
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


class Grid:
    """A box of shape T (x fastest, length ndim), spacing h, sigma per axis; periodic, or
    with wall=True zero beyond both ends of every axis (sigma[T-1] must then be 0)."""

    def __init__(self, T, h, sigmas, wall=False):
        self.wall = bool(wall)
        self.T = tuple(int(t) for t in T)
        self.ndim = len(self.T)
        assert 1 <= self.ndim <= 3 and len(sigmas) == self.ndim
        self.h = float(h)
        self.sigmas = [_f64(s) for s in sigmas]
        for t, s in zip(self.T, self.sigmas):
            assert s.shape == (t,)
        if self.wall:
            assert all(s_[-1] == 0.0 for s_ in self.sigmas), "a wall leaves no edge T-1 -> 0"
        self._T = _i64(self.T)
        self._sig = _f64(np.concatenate(self.sigmas))

    @property
    def n(self) -> int:
        return int(np.prod(self.T))

    @property
    def nfields(self) -> int:
        return 2 + 2 * self.ndim

    def zeros_state(self):
        return np.zeros((self.nfields, self.n), dtype=np.float64)

    def flat(self, coords) -> int:
        """Flat index of vertex coords=(x[, y[, z]])."""
        idx, stride = 0, 1
        for c, t in zip(coords, self.T):
            idx += (int(c) % t) * stride
            stride *= t
        return idx

    def field(self, state, k):
        """View field k of a state as an array indexed [z][y][x] (numpy order)."""
        return state[k].reshape(self.T[::-1])


def ricker(t, f_peak, t_delay):
    return _lib().orc_ricker(float(t), float(f_peak), float(t_delay))


def sigma_profile(N, w, kind=KIND_POWER, sigma_max=2.0, order=2.0, draws=None):
    """Edge-centred damping profile of length N + 2w (Sec. 1.1.2): sigma[e] belongs to the
    edge (e, e+1); the physical edges w-1 .. w+N-1 carry 0, the layer edges
    sigma_max (d/w)^order with d the edge's depth into the layer (kind POWER), sigma_max
    (CONSTANT) or sigma_max times a given uniform draw (RANDOM)."""
    T = int(N) + 2 * int(w)
    out = np.zeros(T, dtype=np.float64)
    d = None if draws is None else _f64(draws)
    if kind == KIND_RANDOM:
        assert d is not None and d.shape == (T,)
    rc = _lib().orc_sigma_profile(int(N), int(w), int(kind), float(sigma_max), float(order),
                                 _ptr(d), _ptr(out))
    if rc != 0:
        raise ValueError("bad sigma profile arguments")
    return out


def layout_axis(sigma, centre):
    """(phi_active, psi_active, interior) uint8 masks along one axis."""
    s = _f64(sigma)
    T = s.shape[0]
    pa = np.zeros(T, np.uint8)
    qa = np.zeros(T, np.uint8)
    it = np.zeros(T, np.uint8)
    _lib().orc_layout_axis(_ptr(s), T, int(centre), _ptr(pa), _ptr(qa), _ptr(it))
    return pa, qa, it


def _src_args(sources):
    if sources is None:
        return 0, None, None, 0.0, 0.0, None, None
    idx = _i64(sources["idx"])
    amp = _f64(sources["amp"])
    return (int(idx.shape[0]), idx, amp, float(sources["f_peak"]), float(sources["t_delay"]),
            idx, amp)


def rhs(grid: Grid, y, sources=None, t=0.0):
    """A y (+ b(t)), eq:DiscretePML."""
    y = _f64(y).reshape(grid.nfields, grid.n)
    out = np.empty_like(y)
    ns, idx, amp, fp, td, _k1, _k2 = _src_args(sources)
    _bc(grid).orc_rhs(grid.ndim, _ptr(grid._T), grid.h, _ptr(grid._sig), _ptr(y), _ptr(out), ns,
                   _ptr(idx), _ptr(amp), fp, td, float(t))
    return out


def rk4(grid: Grid, y, nsteps, dt, step0=0, sources=None, receivers=None, openmp=False):
    """nsteps classic RK4 steps (Sec. 1.1.3).  Returns (state, traces or None)."""
    y = _f64(y).reshape(grid.nfields, grid.n).copy()
    ns, idx, amp, fp, td, _k1, _k2 = _src_args(sources)
    nr = 0
    ridx = None
    trace = None
    if receivers is not None:
        ridx = _i64(receivers)
        nr = int(ridx.shape[0])
        trace = np.zeros((int(nsteps), nr), dtype=np.float64)
    rc = _bc(grid, openmp).orc_rk4(grid.ndim, _ptr(grid._T), grid.h, _ptr(grid._sig), _ptr(y),
                              int(nsteps), float(dt), int(step0), ns, _ptr(idx), _ptr(amp), fp,
                              td, nr, _ptr(ridx), _ptr(trace))
    if rc != 0:
        raise MemoryError("oracle scratch allocation failed")
    return y, trace


def energy(grid: Grid, y, lo=None, hi=None):
    """eq:Energy over the inclusive window lo..hi (default: the whole box)."""
    y = _f64(y).reshape(grid.nfields, grid.n)
    lo = _i64([0] * grid.ndim if lo is None else lo)
    hi = _i64([t - 1 for t in grid.T] if hi is None else hi)
    return _bc(grid).orc_energy(grid.ndim, _ptr(grid._T), grid.h, _ptr(y), _ptr(lo), _ptr(hi))


def norms(grid: Grid, U, ref=None, lo=None, hi=None):
    """(max|U|, ||U||_2, ||U-ref||_2) over the inclusive window."""
    U = _f64(U).reshape(grid.n)
    r = None if ref is None else _f64(ref).reshape(grid.n)
    lo = _i64([0] * grid.ndim if lo is None else lo)
    hi = _i64([t - 1 for t in grid.T] if hi is None else hi)
    out = np.zeros(3)
    _lib().orc_norms(grid.ndim, _ptr(grid._T), _ptr(U), _ptr(r), _ptr(lo), _ptr(hi), _ptr(out))
    return out


def rhs_transpose(grid: Grid, yb):
    yb = _f64(yb).reshape(grid.nfields, grid.n)
    out = np.empty_like(yb)
    _bc(grid).orc_rhs_transpose(grid.ndim, _ptr(grid._T), grid.h, _ptr(grid._sig), _ptr(yb),
                             _ptr(out))
    return out


def adjoint(grid: Grid, yb, nsteps, dt, step_end, sources=None, receivers=None, residual=None):
    """Reverse nsteps RK4 steps from step_end.  Returns (yb, grad_amp or None)."""
    yb = _f64(yb).reshape(grid.nfields, grid.n).copy()
    ns, idx, _amp, fp, td, _k1, _k2 = _src_args(sources)
    gamp = np.zeros(ns, dtype=np.float64) if ns else None
    nr = 0
    ridx = None
    res = None
    if receivers is not None:
        ridx = _i64(receivers)
        nr = int(ridx.shape[0])
        res = _f64(residual).reshape(int(nsteps), nr)
    rc = _bc(grid).orc_adjoint(grid.ndim, _ptr(grid._T), grid.h, _ptr(grid._sig), _ptr(yb),
                            int(nsteps), float(dt), int(step_end), ns, _ptr(idx), fp, td,
                            _ptr(gamp), nr, _ptr(ridx), _ptr(res))
    if rc != 0:
        raise MemoryError("oracle scratch allocation failed")
    return yb, gamp


def misfit_grad_sigma(grid: Grid, y0, nsteps, dt, receivers, target, sources=None, step0=0):
    """J = 1/2 sum_m sum_r (U_m(x_r) - target[m-1, r])^2 of the RK4 run from y0 and dJ/dsigma
    per axis (list of arrays of length T[a]; zero where sigma is zero).  Keeps every
    forward state: small problems only."""
    y0 = _f64(y0).reshape(grid.nfields, grid.n)
    ns, idx, amp, fp, td, _k1, _k2 = _src_args(sources)
    ridx = _i64(receivers)
    nr = int(ridx.shape[0])
    tgt = _f64(target).reshape(int(nsteps), nr)
    J = ctypes.c_double(0.0)
    grad = np.zeros(int(sum(grid.T)), dtype=np.float64)
    rc = _bc(grid).orc_misfit_grad_sigma(grid.ndim, _ptr(grid._T), grid.h, _ptr(grid._sig), _ptr(y0),
                                      int(nsteps), float(dt), int(step0), ns, _ptr(idx), _ptr(amp), fp,
                                      td, nr, _ptr(ridx), _ptr(tgt), ctypes.byref(J), _ptr(grad))
    if rc != 0:
        raise MemoryError("oracle scratch allocation failed")
    out, off = [], 0
    for t in grid.T:
        out.append(grad[off:off + t].copy())
        off += t
    return J.value, out
