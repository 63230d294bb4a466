"""Layer backed by a reflecting wall (PML_FLAG_WALL; Sec. 1.1.4's reflecting boundary):
every field is zero just beyond both ends of every axis.  Forward and transposed steps
against the oracle's wall mode, FP64 <= 1e-12 and FP32 <= 1e-5 relative L2 per field, on
shapes whose layer-free run is clamped by the walls (w = 0, 1, 2), several strips and a
ragged tail, and constant, quadratic and random damping.
"""
import numpy as np
import pytest

import oracle

from ._helpers import assert_close, TOL, gaussian_u0, rel_l2

pytestmark = pytest.mark.gpu

KIND = {"quadratic": oracle.KIND_POWER, "constant": oracle.KIND_CONSTANT, "random": oracle.KIND_RANDOM}


def _setup(N, w, sigma, seed):
    rng = np.random.default_rng(seed)
    T = tuple(n + 2 * w for n in N)
    draws = [rng.random(t) for t in T] if sigma == "random" else None
    sig = []
    for a, n in enumerate(N):
        s_ = oracle.sigma_profile(n, w, KIND[sigma], 2.0, 2.0, draws=None if draws is None else draws[a])
        s_[-1] = 0.0   # the wall replaces the wrap edge
        sig.append(s_)
    u0 = gaussian_u0(N, w, seed) + rng.normal(scale=0.3, size=T[::-1]) if min(N) > 8 else rng.normal(size=T[::-1])
    v0 = rng.normal(scale=0.3, size=T[::-1])
    return T, draws, sig, u0, v0


def _solver(N, w, sigma, draws, prec, adjoint=False):
    import torch
    from paper_1804_01390_gb300.solver import PMLSolver
    return PMLSolver(N, w, sigma=sigma, sigma_max=2.0, draws=draws, precision=prec, device=torch.device("cuda:0"),
                     adjoint=adjoint, wall=True)


CASES2 = [((37, 29), 6, "quadratic"), ((300, 70), 9, "constant"), ((40, 33), 0, "quadratic"),
          ((23, 41), 1, "constant"), ((30, 21), 2, "random"), ((64, 45), 12, "random")]


@pytest.mark.parametrize("N,w,sigma", CASES2)
@pytest.mark.parametrize("prec", [64, 32])
def test_wall_forward_parity_2d(N, w, sigma, prec):
    import torch
    T, draws, sig, u0, v0 = _setup(N, w, sigma, seed=sum(N) + w)
    s = _solver(N, w, sigma, draws, prec)
    s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
    s.step(23)
    got = [s.read(f).double().cpu().numpy() for f in range(6)]
    s.close()
    g = oracle.Grid(T, 1.0, sig, wall=True)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    y[1] = v0.reshape(-1)
    want, _ = oracle.rk4(g, y, 23, 0.5)
    for f in range(6):
        assert_close(got[f], want[f], prec, repr((f)))


CASES3 = [((21, 18, 15), 5, "quadratic"), ((30, 14, 12), 0, "constant"), ((16, 27, 20), 4, "random")]


@pytest.mark.parametrize("N,w,sigma", CASES3)
@pytest.mark.parametrize("prec", [64, 32])
def test_wall_forward_parity_3d(N, w, sigma, prec):
    import torch
    T, draws, sig, u0, v0 = _setup(N, w, sigma, seed=sum(N) + w)
    s = _solver(N, w, sigma, draws, prec)
    s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
    s.step(11)
    got = [s.read(f).double().cpu().numpy() for f in range(8)]
    s.close()
    g = oracle.Grid(T, 1.0, sig, wall=True)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    y[1] = v0.reshape(-1)
    want, _ = oracle.rk4(g, y, 11, 0.5)
    for f in range(8):
        assert_close(got[f], want[f], prec, repr((f)))


@pytest.mark.parametrize("N,w", [((40, 31), 6), ((18, 16, 14), 4)])
def test_wall_adjoint_parity(N, w):
    """The transposed step with walls: the adjoint state after injecting a receiver
    misfit and running back, against the oracle's transposed stage graph."""
    import torch
    T, draws, sig, u0, v0 = _setup(N, w, "quadratic", seed=7)
    g = oracle.Grid(T, 1.0, sig, wall=True)
    nf = 2 + 2 * len(N)
    rng = np.random.default_rng(8)
    rec = [tuple(w + n // 2 - 1 for n in N), tuple(w + 1 for n in N)]
    steps = 9
    tgt = rng.normal(size=(steps, len(rec)))
    s = _solver(N, w, "quadratic", None, 64, adjoint=True)
    s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
    tr = s.set_receivers(rec, steps)
    s.step(steps)
    res = tr.double().cpu().numpy() - tgt
    s.adjoint_reset()
    s.adjoint_step(steps, torch.from_numpy(res[::-1].copy()), want_grad_u=True)
    got = [s.adjoint_read(f).double().cpu().numpy() for f in range(nf)]
    s.close()
    yy = g.zeros_state()
    yy[0] = u0.reshape(-1)
    yy[1] = v0.reshape(-1)
    ridx = [g.flat(r) for r in rec]
    _, trace = oracle.rk4(g, yy, steps, 0.5, receivers=ridx)
    yb, _ = oracle.adjoint(g, g.zeros_state(), steps, 0.5, steps, receivers=ridx,
                           residual=(trace - tgt)[::-1].copy())
    for f in range(nf):
        err = rel_l2(got[f], yb[f])
        assert err <= 1e-12, (f, err)


@pytest.mark.parametrize("prec", [64, 32])
def test_wall_every_variant_2d(prec):
    """Every kernel shape of a 2D context (one-step shapes, including those with 3-row TMA
    boxes, and the two-step shapes) with reflecting walls against the oracle."""
    import torch
    from paper_1804_01390_gb300 import _lib
    N, w, steps = (70, 53), 3, 21
    T, draws, sig, u0, v0 = _setup(N, w, "quadratic", seed=404)
    g = oracle.Grid(T, 1.0, sig, wall=True)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    y[1] = v0.reshape(-1)
    want, _ = oracle.rk4(g, y, steps, 0.5)
    s = _solver(N, w, "quadratic", draws, prec)
    _, nv = _lib.pml_get_variant(s.ctx)
    for v in range(nv):
        _lib.pml_set_variant(s.ctx, v)
        s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
        s.step(steps)
        for f in range(6):
            assert_close(s.read(f).double().cpu().numpy(), want[f], prec, repr((v, f)))
    s.close()
