"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds none of the method's arithmetic: no damping profile, no stencil,
no time stepping.  It draws the random numbers and builds the initial data that
both sides receive as plain arrays, so that the two implementations can be compared
on identical inputs.  Only numpy is used (PCG64 via ``numpy.random.default_rng``).

Workloads follow the shape of the paper's experiments (Sec. 1.1.3: a Gauss bump
with zero initial velocity, white noise in a disk; Sec. 1.1.4: residual waves in a
periodic box; Sec. 1.1.5: long-time energy) scaled to the benchmark configurations:

* ``cfg1``  2D 128^2 interior + 16-cell layer, one Gaussian (s=4) near an interface;
* ``cfg2``  2D 8192^2 interior + 32-cell layer, 16 Gaussians (s in [2,8], amp in [-1,1]);
* ``cfg3``  3D 512^3 interior + 24-cell layer, one Gaussian (s=6) plus 8 point sources;
* ``cfg4``  96 independent 2D grids with sides in [256, 2048], layer 16..32, one Gaussian each;
* ``cfg5``  2D 2048^2 interior + 32-cell layer, Gaussian (s=8), 16 sources, 64 receivers.

Every Gaussian is exp(-|x - c|^2 / (2 s^2)) with a real-valued centre c (in vertex
units) and is multiplied by the indicator of the physical window, so the layer
starts at rest (the initial data of the paper's runs have compact support inside the
physical domain).  Arrays are numpy-ordered [z][y][x] (x fastest).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Gaussian:
    centre: tuple          # (cx[, cy[, cz]]) in vertex units of the padded box
    width: float           # s
    amp: float = 1.0


@dataclass
class Workload:
    name: str
    ndim: int
    N: tuple               # interior vertices per axis (x, y[, z])
    w: int                 # layer width per side
    h: float = 1.0
    dt: float = 0.5
    steps: int = 1000
    sigma_kind: str = "quadratic"   # "quadratic" | "constant" | "random"
    sigma_max: float = 2.0
    sigma_order: float = 2.0
    sigma_draws: list = None        # per-axis uniform [0,1) draws for "random"
    gaussians: list = field(default_factory=list)
    sources: dict = None            # {"coords": [[x,y(,z)],...], "amp": [...], "f_peak", "t_delay"}
    receivers: list = None          # [[x,y(,z)], ...]
    seed: int = 0

    @property
    def T(self):
        return tuple(n + 2 * self.w for n in self.N)

    @property
    def points(self) -> int:
        return int(np.prod(self.T))

    def window(self):
        """Inclusive physical window per axis (x, y[, z])."""
        lo = tuple(self.w for _ in self.N)
        hi = tuple(self.w + n - 1 for n in self.N)
        return lo, hi


def gaussian_field(T, gaussians, window=None, dtype=np.float64):
    """Sum of Gaussians on the padded box T=(Tx, Ty[, Tz]); zero outside `window`.

    Each Gaussian is evaluated on a +-7s box around its centre only (exp(-24.5) is
    below 1e-10 of the peak), so 8k^2 and 512^3 fields build in seconds.
    """
    T = tuple(int(t) for t in T)
    nd = len(T)
    out = np.zeros(T[::-1], dtype=np.float64)
    for g in gaussians:
        r = 7.0 * g.width
        sl = []
        axes = []
        for a in range(nd):
            lo = max(0, int(np.floor(g.centre[a] - r)))
            hi = min(T[a], int(np.ceil(g.centre[a] + r)) + 1)
            sl.append(slice(lo, hi))
            axes.append(np.arange(lo, hi, dtype=np.float64) - g.centre[a])
        # numpy order is reversed (z, y, x)
        d2 = np.zeros([len(ax) for ax in axes[::-1]], dtype=np.float64)
        for a in range(nd):
            shape = [1] * nd
            shape[nd - 1 - a] = len(axes[a])
            d2 = d2 + (axes[a] ** 2).reshape(shape)
        out[tuple(sl[::-1])] += g.amp * np.exp(-d2 / (2.0 * g.width * g.width))
    if window is not None:
        lo, hi = window
        mask = np.zeros_like(out, dtype=bool)
        mask[tuple(slice(l, h + 1) for l, h in zip(lo[::-1], hi[::-1]))] = True
        out = np.where(mask, out, 0.0)
    return out.astype(dtype, copy=False)


def initial_field(wl: Workload, dtype=np.float64):
    return gaussian_field(wl.T, wl.gaussians, wl.window(), dtype)


def sigma_draws(T, seed):
    """Uniform [0,1) draws, one per edge, for a random damping profile (Fig. HalfSpaceRand)."""
    return np.random.default_rng(seed).random(int(T))


def white_noise_disk(T, centre, radius, variance, seed, window=None):
    """Gaussian white noise of the given variance inside a disk / ball (Fig. HalfSpaceRand)."""
    T = tuple(int(t) for t in T)
    rng = np.random.default_rng(seed)
    noise = rng.normal(0.0, np.sqrt(variance), size=T[::-1])
    grids = np.meshgrid(*[np.arange(t, dtype=np.float64) for t in T[::-1]], indexing="ij")
    d2 = sum((grids[len(T) - 1 - a] - centre[a]) ** 2 for a in range(len(T)))
    out = np.where(d2 <= radius * radius, noise, 0.0)
    if window is not None:
        lo, hi = window
        mask = np.zeros_like(out, dtype=bool)
        mask[tuple(slice(l, h + 1) for l, h in zip(lo[::-1], hi[::-1]))] = True
        out = np.where(mask, out, 0.0)
    return out


def cfg1(N=128, w=16, steps=1000, seed=1, sigma_kind="quadratic", sigma_max=2.0):
    """2D Gauss bump near one interface (Sec. 1.1.3, Fig. HalfSpaceGauss geometry)."""
    rng = np.random.default_rng(seed)
    off = rng.uniform(8.0, 24.0)
    cy = w + N / 2.0 + rng.uniform(-N / 8.0, N / 8.0)
    g = Gaussian((w + off, cy), 4.0, 1.0)
    return Workload("cfg1", 2, (N, N), w, steps=steps, gaussians=[g], seed=seed,
                    sigma_kind=sigma_kind, sigma_max=sigma_max)


def reference_box(wl: Workload, M):
    """The same initial data placed in a periodic M^d box without layer (sigma = 0).

    The physical window of `wl` maps to vertices off..off+N-1 of the big box with
    off = (M - N)/2 along each axis, vertex for vertex.
    Returns (big workload, offsets).
    """
    offs = tuple((M - n) // 2 for n in wl.N)
    shift = tuple(o - wl.w for o in offs)
    gs = [Gaussian(tuple(c + s for c, s in zip(g.centre, shift)), g.width, g.amp)
          for g in wl.gaussians]
    big = Workload(wl.name + "-ref", wl.ndim, tuple(M for _ in wl.N), 0, wl.h, wl.dt, wl.steps,
                   "constant", 0.0, gaussians=gs, seed=wl.seed)
    return big, offs


def reference_initial_field(wl: Workload, M, dtype=np.float64):
    """Initial field of the big reference box: the masked window data of `wl`, embedded."""
    big, offs = reference_box(wl, M)
    u_small = initial_field(wl)
    out = np.zeros(big.T[::-1], dtype=np.float64)
    lo, hi = wl.window()
    src = tuple(slice(l, h + 1) for l, h in zip(lo[::-1], hi[::-1]))
    dst = tuple(slice(o, o + n) for o, n in zip(offs[::-1], wl.N[::-1]))
    out[dst] = u_small[src]
    return out.astype(dtype, copy=False)


def cfg2(N=8192, w=32, steps=5000, seed=2, npulses=16):
    """2D large single grid: 16 Gaussians, s in [2,8], amplitudes in [-1,1]."""
    rng = np.random.default_rng(seed)
    gs = []
    for _ in range(npulses):
        s = rng.uniform(2.0, 8.0)
        c = tuple(w + rng.uniform(3 * s, n - 1 - 3 * s) for n in (N, N))
        gs.append(Gaussian(c, s, rng.uniform(-1.0, 1.0)))
    return Workload("cfg2", 2, (N, N), w, steps=steps, gaussians=gs, seed=seed)


def cfg3(N=512, w=24, steps=2000, seed=3, nsrc=8, dt=0.5):
    """3D: one Gaussian (s=6) near the centre plus 8 Ricker point sources (0.05 / step)."""
    rng = np.random.default_rng(seed)
    c = tuple(w + N / 2.0 + rng.uniform(-N / 8.0, N / 8.0) for _ in range(3))
    g = Gaussian(c, 6.0, 1.0)
    coords = [[int(rng.integers(w + 8, w + N - 8)) for _ in range(3)] for _ in range(nsrc)]
    amps = list(rng.uniform(-1.0, 1.0, size=nsrc))
    f_peak = 0.05 / dt
    src = {"coords": coords, "amp": amps, "f_peak": f_peak, "t_delay": 1.5 / f_peak}
    return Workload("cfg3", 3, (N, N, N), w, dt=dt, steps=steps, gaussians=[g], sources=src,
                    seed=seed)


def cfg4(ngrids=96, seed=4, steps=3000, lo=256, hi=2048):
    """96 independent 2D grids of uneven sizes, one Gaussian (s=4) each."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(ngrids):
        N = (int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1)))
        w = int(rng.integers(16, 33))
        c = tuple(w + rng.uniform(0.25 * n, 0.75 * n) for n in N)
        out.append(Workload("cfg4[%d]" % k, 2, N, w, steps=steps,
                            gaussians=[Gaussian(c, 4.0, 1.0)], seed=seed))
    return out


def cfg5(N=2048, w=32, steps=10000, seed=5, nsrc=16, nrec=64, dt=0.5):
    """2D adjoint workload: Gaussian (s=8), 16 Ricker sources, 64 receivers on a line."""
    rng = np.random.default_rng(seed)
    c = tuple(w + N / 2.0 + rng.uniform(-N / 8.0, N / 8.0) for _ in range(2))
    g = Gaussian(c, 8.0, 1.0)
    coords = [[int(rng.integers(w + 8, w + N - 8)) for _ in range(2)] for _ in range(nsrc)]
    amps = list(rng.uniform(-1.0, 1.0, size=nsrc))
    f_peak = 0.05 / dt
    src = {"coords": coords, "amp": amps, "f_peak": f_peak, "t_delay": 1.5 / f_peak}
    ry = w + 32
    rxs = np.linspace(w + 8, w + N - 9, nrec).round().astype(int)
    rec = [[int(x), ry] for x in rxs]
    return Workload("cfg5", 2, (N, N), w, dt=dt, steps=steps, gaussians=[g], sources=src,
                    receivers=rec, seed=seed)


def cfg5_target(wl: Workload, seed=6):
    """Seeded 'true' model (U0*, a*) whose traces serve as the misfit target."""
    rng = np.random.default_rng(seed)
    n = len(wl.N)
    c = tuple(w_ + n_ / 2.0 + rng.uniform(-n_ / 8.0, n_ / 8.0) for w_, n_ in zip([wl.w] * n, wl.N))
    g = Gaussian(c, 8.0, rng.uniform(0.5, 1.5))
    amps = list(rng.uniform(-1.0, 1.0, size=len(wl.sources["amp"])))
    return [g], amps


def scaled(wl_fn, **kw):
    """Reduced-size variant of a workload (same layer, profile and sources recipe)."""
    return wl_fn(**kw)
