"""The paper's two printed 2D validation runs (Fig. HalfSpaceGauss and Fig. HalfSpaceRand,
Sec. 1.1.3), replayed on the FP64 oracle at the printed scale.

The setups come from the fixtures under ``tests/golden/`` (grid spacing, box, physical
window, damping, peak value or noise variance, end time, size of the reference box); the
paper reports that the reflection measured against an undamped run on the larger box is at
machine zero in double precision.  What the captions leave open is fixed here:

* dt = h/2 (the paper never states dt), so t = 1/2 is 80 steps;
* the layer sits on both sides of the 80-vertex physical window in a periodic 160-vertex
  box (the periodic image of the paper's [-1, 0] window with the layer on [0, 1]); the
  damping is carried by every layer edge except the two interface edges;
* the bump is a Gaussian of width 4h centred 0.2 and 0.45 from the two far interfaces, and
  the noise fills a disk of radius 10h at the window's centre; both are zero outside the
  physical window and both runs start from the same samples.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1804_01390_gb300 import workloads as wk

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            try:
                out[k] = Fraction(v)
            except ValueError:
                out[k] = v
    return out


def _setup(fx):
    h = fx["h"]
    T = int((fx["box_hi"] - fx["box_lo"]) / h)           # periodic box, vertices per axis
    N = int((fx["physical_hi"] - fx["physical_lo"]) / h)  # [lo, hi): the vertex at hi is the layer's first
    assert (T - N) % 2 == 0
    w = (T - N) // 2
    M = int((fx["reference_hi"] - fx["reference_lo"]) / h)
    dt = h / 2
    steps = int(fx["t_end"] / dt)
    assert steps * dt == fx["t_end"]
    return float(h), T, N, w, M, float(dt), steps


def _truncated_vs_reference(orc, h, N, w, M, sigmas, u0, steps, dt):
    """max |U - U_ref| over the physical window, max |U_ref| there and beyond it."""
    T = N + 2 * w
    g = orc.Grid((T, T), h, sigmas)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    yn, _ = orc.rk4(g, y, steps, dt)
    gb = orc.Grid((M, M), h, [np.zeros(M), np.zeros(M)])
    off = (M - N) // 2
    ub = np.zeros((M, M))
    ub[off:off + N, off:off + N] = u0[w:w + N, w:w + N]
    yb = gb.zeros_state()
    yb[0] = ub.reshape(-1)
    ybn, _ = orc.rk4(gb, yb, steps, dt, openmp=True)
    a = g.field(yn, 0)[w:w + N, w:w + N]
    big = gb.field(ybn, 0)
    b = big[off:off + N, off:off + N]
    outside = big.copy()
    outside[off:off + N, off:off + N] = 0.0
    return np.abs(a - b).max(), np.abs(b).max(), np.abs(outside).max()


def test_fixture_reads_as_printed():
    fx = _load("fig_halfspace_gauss.txt")
    h, T, N, w, M, dt, steps = _setup(fx)
    assert (T, N, w, M, steps) == (160, 80, 40, 800, 80)
    assert fx["sigma_times_h"] == 2 and fx["peak"] == 2 and fx["t_end"] == Fraction(1, 2)
    fr = _load("fig_halfspace_rand.txt")
    assert _setup(fr) == (h, T, N, w, M, dt, steps)
    assert fr["noise_variance"] == Fraction(1, 4) and fr["sigma_profile"] == "uniform_random"


def test_fig_halfspace_gauss(orc):
    fx = _load("fig_halfspace_gauss.txt")
    h, T, N, w, M, dt, steps = _setup(fx)
    smax = float(fx["sigma_times_h"]) / h
    sigmas = [orc.sigma_profile(N, w, orc.KIND_CONSTANT, smax) for _ in range(2)]
    # window x = -1 + (i - w) h; centre 0.2 from the interface at x = 0 and 0.45 from y = 0
    cx, cy = w + (0.8 / h), w + (0.55 / h)
    wl = wk.Workload("fig-gauss", 2, (N, N), w, h=h,
                     gaussians=[wk.Gaussian((cx, cy), 4.0, float(fx["peak"]))])
    u0 = wk.initial_field(wl)
    assert abs(u0.max() - float(fx["peak"])) < 1e-12
    err, ref, out = _truncated_vs_reference(orc, h, N, w, M, sigmas, u0, steps, dt)
    assert ref > 1e-2 and out > 1e-2      # waves have crossed the interface by t = 1/2
    print("max reflection", err, "peak", ref, "beyond window", out)
    assert err < 1e-14, err


def test_fig_halfspace_rand(orc):
    fx = _load("fig_halfspace_rand.txt")
    h, T, N, w, M, dt, steps = _setup(fx)
    smax = float(fx["sigma_times_h"]) / h
    rng = np.random.default_rng(1804)
    sigmas = [orc.sigma_profile(N, w, orc.KIND_RANDOM, smax, draws=rng.random(T)) for _ in range(2)]
    c = w + N / 2 - 0.5
    u0 = wk.white_noise_disk((T, T), (c, c), 10.0, float(fx["noise_variance"]), seed=1805,
                             window=((w, w), (w + N - 1, w + N - 1)))
    assert abs(u0[u0 != 0].var() - 0.25) < 0.05
    err, ref, out = _truncated_vs_reference(orc, h, N, w, M, sigmas, u0, steps, dt)
    assert ref > 1e-2 and out > 1e-3
    print("max reflection", err, "peak", ref, "beyond window", out)
    assert err < 1e-14, err
