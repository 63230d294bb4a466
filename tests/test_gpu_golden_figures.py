"""The CUDA path at the scale of the paper's printed 2D validation run (Fig. HalfSpaceGauss,
Sec. 1.1.3; setup in ``tests/golden/fig_halfspace_gauss.txt``): h = 1/80 on a periodic
[-1, 1]^2 box, constant sigma = 2/h, a bump of peak 2, t = 1/2 at dt = h/2.

Every other parity test runs at h = 1; here the 1/h, 1/h^2 and 1/(2h) factors of the
operator, the h-scaled coefficients of the closed-form interior step and sigma values of
order 1/h are all exercised.  Compared with the FP64 oracle on the same box (FP64 and FP32
modes, forward and transposed steps), and in FP64 with an undamped run on the printed
[-5, 5]^2 reference box: the reflection stays at machine zero.
"""
import numpy as np
import pytest

import oracle
from paper_1804_01390_gb300 import workloads as wk

from ._helpers import assert_close, TOL, rel_l2
from .test_golden_figures import _load, _setup

pytestmark = pytest.mark.gpu


def _case():
    fx = _load("fig_halfspace_gauss.txt")
    h, T, N, w, M, dt, steps = _setup(fx)
    smax = float(fx["sigma_times_h"]) / h
    wl = wk.Workload("fig-gauss", 2, (N, N), w, h=h,
                     gaussians=[wk.Gaussian((w + 0.8 / h, w + 0.55 / h), 4.0, float(fx["peak"]))])
    return h, T, N, w, M, dt, steps, smax, wk.initial_field(wl)


def _solver(N, w, h, dt, smax, prec, adjoint=False):
    import torch
    from paper_1804_01390_gb300.solver import PMLSolver
    return PMLSolver((N, N), w, h=h, dt=dt, sigma="constant", sigma_max=smax, precision=prec,
                     device=torch.device("cuda:0"), adjoint=adjoint)


def _oracle_grid(N, w, h, smax):
    sig = [oracle.sigma_profile(N, w, oracle.KIND_CONSTANT, smax) for _ in range(2)]
    return oracle.Grid((N + 2 * w, N + 2 * w), h, sig)


@pytest.mark.parametrize("prec", [64, 32])
def test_forward_at_printed_scale(prec):
    import torch
    h, T, N, w, M, dt, steps, smax, u0 = _case()
    rng = np.random.default_rng(80)
    v0 = rng.normal(scale=0.3, size=(T, T))     # nonzero velocity and a noisy start reach every term
    u0 = u0 + rng.normal(scale=0.3, size=(T, T))
    s = _solver(N, w, h, dt, smax, prec)
    s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
    s.step(steps)
    got = [s.read(f).double().cpu().numpy() for f in range(6)]
    s.close()
    g = _oracle_grid(N, w, h, smax)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    y[1] = v0.reshape(-1)
    want, _ = oracle.rk4(g, y, steps, dt)
    for f in range(6):
        assert_close(got[f], want[f], prec, repr((f,)))


def test_reflection_at_machine_zero_fp64():
    import torch
    h, T, N, w, M, dt, steps, smax, u0 = _case()
    s = _solver(N, w, h, dt, smax, 64)
    s.set_initial(torch.from_numpy(u0))
    s.step(steps)
    U = s.read(0).double().cpu().numpy()[w:w + N, w:w + N]
    s.close()
    off = (M - N) // 2
    ub = np.zeros((M, M))
    ub[off:off + N, off:off + N] = u0[w:w + N, w:w + N]
    gb = oracle.Grid((M, M), h, [np.zeros(M), np.zeros(M)])
    yb = gb.zeros_state()
    yb[0] = ub.reshape(-1)
    out, _ = oracle.rk4(gb, yb, steps, dt, openmp=True)
    big = out[0].reshape(M, M)
    ref = big[off:off + N, off:off + N]
    beyond = big.copy()
    beyond[off:off + N, off:off + N] = 0.0
    assert np.abs(ref).max() > 1e-2 and np.abs(beyond).max() > 1e-2
    assert np.abs(U - ref).max() <= 1e-13 * 2.0, np.abs(U - ref).max()


@pytest.mark.parametrize("prec", [64, 32])
def test_transposed_step_at_printed_scale(prec):
    """Reverse steps with a Ricker source (f = 20 per unit time) and receiver residuals
    injected in and outside the layer: the adjoint state, dJ/dU0 and dJ/da."""
    import torch
    h, T, N, w, M, dt, steps, smax, u0 = _case()
    n, f, t0 = 12, 20.0, 0.04
    rng = np.random.default_rng(81)
    src = [(w + 30, w + 50), (w + 31, w + 50)]
    amp = [0.7, -0.4]
    rec = [(w + 2, w + 3), (1, 2), (w + 31, w + 51), (150, 100)]
    residual = rng.normal(scale=0.1, size=(n, len(rec)))
    s = _solver(N, w, h, dt, smax, prec, adjoint=True)
    s.set_initial(torch.from_numpy(u0))
    s.set_sources(src, amp, f, t0)
    s.set_receivers(rec, n)
    s.step(n)
    s.adjoint_reset()
    gu, ga = s.adjoint_step(n, torch.from_numpy(residual))
    got = [s.adjoint_read(k).double().cpu().numpy() for k in range(6)]
    s.close()
    g = _oracle_grid(N, w, h, smax)
    srcd = {"idx": [g.flat(c) for c in src], "amp": amp, "f_peak": f, "t_delay": t0}
    yb, gamp = oracle.adjoint(g, g.zeros_state(), n, dt, n, sources=srcd,
                              receivers=[g.flat(c) for c in rec], residual=residual)
    assert_close(gu.double().cpu().numpy(), yb[0], prec)
    for k in range(6):
        assert_close(got[k], yb[k], prec, repr((k,)))
    assert np.abs(gamp).max() > 0
    assert rel_l2(ga, gamp) <= (1e-11 if prec == 64 else 1e-5)
