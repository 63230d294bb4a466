"""3D layer frame by level passes (variant 1 of a 3D context: one Horner level per launch
over scratch states, on the frame widened by 3, 2, 1, 0 vertices) against the FP64 oracle:
forward in FP64 and FP32 (with and without a layer, random damping, reflecting walls) and
the transposed step with sources and injected residuals.  Both 3D variants evaluate the same
operator expression per level, so they also agree with each other to rounding."""
import numpy as np
import pytest

import oracle

from ._helpers import assert_close, TOL, gaussian_u0, make_solver, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu

CASES = [((21, 18, 15), 5, "quadratic"), ((130, 14, 12), 6, "constant"), ((16, 27, 20), 4, "random"),
         ((20, 16, 24), 0, "quadratic"), ((9, 30, 10), 3, "constant")]


def _state(N, w, seed):
    rng = np.random.default_rng(seed)
    T = tuple(n + 2 * w for n in N)
    u0 = gaussian_u0(N, w, seed) + rng.normal(scale=0.3, size=T[::-1])
    v0 = rng.normal(scale=0.3, size=T[::-1])
    return rng, u0, v0


def _gpu(N, w, prec, sigma, draws, u0, v0, steps, variant, wall=False, dt=0.4):
    import torch
    from paper_1804_01390_gb300 import _lib
    from paper_1804_01390_gb300.solver import PMLSolver
    s = PMLSolver(N, w, dt=dt, sigma=sigma, sigma_max=2.0, draws=draws, precision=prec,
                  device=torch.device("cuda:0"), wall=wall)
    _lib.pml_set_variant(s.ctx, variant)
    assert _lib.pml_get_variant(s.ctx) == (variant, 3 if prec == 32 else 2)
    s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
    s.step(steps)
    got = [s.read(f).double().cpu().numpy() for f in range(8)]
    s.close()
    return got


@pytest.mark.parametrize("N,w,sigma", CASES)
@pytest.mark.parametrize("prec", [64, 32])
def test_level_passes_forward_parity(N, w, sigma, prec):
    rng, u0, v0 = _state(N, w, sum(N) + w)
    draws = [rng.random(n + 2 * w) for n in N] if sigma == "random" else None
    steps = 13
    got = _gpu(N, w, prec, sigma, draws, u0, v0, steps, 1)
    g = oracle_grid(N, w, sigma, 2.0, draws)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    y[1] = v0.reshape(-1)
    want, _ = oracle.rk4(g, y, steps, 0.4)
    for f in range(8):
        assert_close(got[f], want[f], prec, repr((f,)))
    ref = _gpu(N, w, prec, sigma, draws, u0, v0, steps, 0)
    for f in range(8):
        assert rel_l2(got[f], ref[f]) <= (1e-13 if prec == 64 else 1e-6), f


@pytest.mark.parametrize("prec", [64, 32])
def test_level_passes_wall(prec):
    N, w = (24, 19, 17), 4
    rng, u0, v0 = _state(N, w, 77)
    got = _gpu(N, w, prec, "quadratic", None, u0, v0, 15, 1, wall=True)
    g0 = oracle_grid(N, w)
    sig = [np.concatenate([s_[:-1], [0.0]]) for s_ in g0.sigmas]
    g = oracle.Grid(g0.T, 1.0, sig, wall=True)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    y[1] = v0.reshape(-1)
    want, _ = oracle.rk4(g, y, 15, 0.4)
    for f in range(8):
        assert_close(got[f], want[f], prec, repr((f,)))


@pytest.mark.parametrize("prec", [64, 32])
def test_level_passes_adjoint_with_points(prec):
    import torch
    from paper_1804_01390_gb300 import _lib
    N, w, steps, f, t0 = (18, 16, 14), 4, 12, 0.1, 8.0
    rng = np.random.default_rng(5)
    src = [(w + 8, w + 7, w + 6), (w + 9, w + 7, w + 6)]
    rec = [(w + 2, w + 3, w + 4), (1, 2, 3), (w + 10, w + 10, w + 9)]
    amp = [0.6, -0.4]
    residual = rng.normal(scale=0.1, size=(steps, len(rec)))
    s = make_solver(N, w, prec, adjoint=True, dt=0.4)
    _lib.pml_set_variant(s.ctx, 1)
    s.set_initial(torch.from_numpy(gaussian_u0(N, w, 2)))
    s.set_sources(src, amp, f, t0)
    s.set_receivers(rec, steps)
    s.step(steps)
    s.adjoint_reset()
    gu, ga = s.adjoint_step(steps, torch.from_numpy(residual))
    fields = [s.adjoint_read(k).double().cpu().numpy() for k in range(8)]
    s.close()
    g = oracle_grid(N, w)
    srcd = {"idx": [g.flat(c) for c in src], "amp": amp, "f_peak": f, "t_delay": t0}
    yb, gamp = oracle.adjoint(g, g.zeros_state(), steps, 0.4, steps, sources=srcd,
                              receivers=[g.flat(c) for c in rec], residual=residual)
    assert_close(gu.double().cpu().numpy(), yb[0], prec)
    for k, fk in enumerate(fields):
        assert_close(fk, yb[k], prec, repr((k,)))
    assert rel_l2(ga, gamp) <= (1e-11 if prec == 64 else 1e-5)
