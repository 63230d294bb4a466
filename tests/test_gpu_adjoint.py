"""Discrete adjoint on the GPU: against the oracle's adjoint on seeded residuals,
against central differences of GPU forward runs (the misfit is quadratic, so central
differences are exact up to rounding), and through the torch.autograd.Function."""
import numpy as np
import pytest

import oracle

from ._helpers import assert_close, TOL, gaussian_u0, make_solver, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu


def _setup(N, w):
    rng = np.random.default_rng(40 + len(N))
    nd = len(N)
    src = [tuple(w + int(rng.integers(3, n - 3)) for n in N) for _ in range(3)]
    rec = [tuple(int(rng.integers(0, n + 2 * w)) for n in N) for _ in range(4)]
    rec += [tuple(w + int(rng.integers(1, n - 1)) for n in N) for _ in range(4)]
    amp = rng.uniform(-1, 1, len(src))
    return src, rec, amp, rng


@pytest.mark.parametrize("N,w", [((40, 34), 8), ((18, 16, 14), 4)])
@pytest.mark.parametrize("prec", [64, 32])
def test_adjoint_matches_oracle(N, w, prec):
    import torch
    src, rec, amp, rng = _setup(N, w)
    steps, dt, f, t0 = 30, 0.5, 0.1, 12.0
    residual = rng.normal(scale=0.1, size=(steps, len(rec)))
    s = make_solver(N, w, prec, adjoint=True)
    s.set_initial(torch.from_numpy(gaussian_u0(N, w, 1)))
    s.set_sources(src, amp, f, t0)
    s.set_receivers(rec, steps)
    s.step(steps)
    s.adjoint_reset()
    gu, ga = s.adjoint_step(steps, torch.from_numpy(residual))
    fields = [s.adjoint_read(k).double().cpu().numpy() for k in range(2 + 2 * len(N))]
    s.close()
    g = oracle_grid(N, w)
    srcd = {"idx": [g.flat(c) for c in src], "amp": amp, "f_peak": f, "t_delay": t0}
    yb, gamp = oracle.adjoint(g, g.zeros_state(), steps, dt, steps, sources=srcd,
                              receivers=[g.flat(c) for c in rec], residual=residual)
    assert_close(gu.double().cpu().numpy(), yb[0], prec)
    for k, fk in enumerate(fields):
        assert_close(fk, yb[k], prec, repr((k,)))
    assert rel_l2(ga, gamp) <= (1e-11 if prec == 64 else 1e-5), (ga, gamp)


def test_adjoint_vs_central_differences_fp64():
    """Gradients of J = 1/2 sum (U_m(x_r) - d)^2 w.r.t. source amplitudes and U0 agree with
    central differences of forward GPU runs to 1e-6 relative."""
    import torch
    N, w = (36, 30), 8
    src, rec, amp, rng = _setup(N, w)
    steps, f, t0 = 40, 0.1, 12.0
    u0 = gaussian_u0(N, w, 2)
    d = rng.normal(scale=0.05, size=(steps, len(rec)))
    s = make_solver(N, w, 64, adjoint=True)

    def J(u, a):
        s.set_initial(torch.from_numpy(u))
        s.set_sources(src, a, f, t0)
        tr = s.set_receivers(rec, steps)
        s.step(steps)
        t = tr.cpu().numpy()
        return 0.5 * float(np.sum((t - d) ** 2)), t

    J0, tr = J(u0, amp)
    s.adjoint_reset()
    gu, ga = s.adjoint_step(steps, torch.from_numpy((tr - d)[::-1].copy()))
    gu = gu.cpu().numpy()
    eps = 1e-3
    for k in range(len(amp)):
        ap, am = amp.copy(), amp.copy()
        ap[k] += eps
        am[k] -= eps
        fd = (J(u0, ap)[0] - J(u0, am)[0]) / (2 * eps)
        assert abs(fd - ga[k]) <= 1e-6 * max(abs(fd), 1e-8), (k, fd, ga[k])
    T = tuple(n + 2 * w for n in N)
    for (x, y) in [(w + 5, w + 6), (w + 20, w + 11), (w + 1, w + 28), (3, 4)]:
        up, um = u0.copy(), u0.copy()
        up[y, x] += eps
        um[y, x] -= eps
        fd = (J(up, amp)[0] - J(um, amp)[0]) / (2 * eps)
        assert abs(fd - gu[y, x]) <= 1e-6 * max(abs(fd), 1e-8), ((x, y), fd, gu[y, x])
    s.close()


def test_autograd_function_matches_adjoint_and_fd():
    import torch
    from paper_1804_01390_gb300.autograd import traces
    N, w = (30, 28), 6
    src, rec, amp, rng = _setup(N, w)
    steps, f, t0 = 25, 0.1, 12.0
    s = make_solver(N, w, 64, adjoint=True)
    u0 = torch.from_numpy(gaussian_u0(N, w, 3)).cuda().requires_grad_(True)
    a = torch.tensor(amp, dtype=torch.float64, requires_grad=True)
    d = torch.from_numpy(rng.normal(scale=0.05, size=(steps, len(rec)))).cuda()
    tr = traces(s, u0, a, steps, src, rec, f, t0)
    loss = 0.5 * ((tr - d) ** 2).sum()
    loss.backward()
    eps = 1e-4
    for k in range(len(amp)):
        ap = a.detach().clone()
        am = a.detach().clone()
        ap[k] += eps
        am[k] -= eps
        lp = 0.5 * ((traces(s, u0.detach(), ap, steps, src, rec, f, t0) - d) ** 2).sum()
        lm = 0.5 * ((traces(s, u0.detach(), am, steps, src, rec, f, t0) - d) ** 2).sum()
        fd = float((lp - lm) / (2 * eps))
        assert abs(fd - float(a.grad[k])) <= 1e-6 * max(abs(fd), 1e-8)
    assert u0.grad is not None and u0.grad.shape == u0.shape
    s.close()
