"""Point sources and receivers whose updates meet: sources with overlapping stencils (a
vertex and its neighbours) and several receivers at one vertex.  The point kernels run
one thread per point in levels that keep every vertex's additions in index order; the
forward state, the traces, the transposed step with injected residuals and the
source-amplitude gradient must match the FP64 oracle."""
import numpy as np
import pytest

import oracle

from ._helpers import assert_close, TOL, gaussian_u0, make_solver, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu


def _points(w):
    c = (w + 20, w + 18)
    src = [c, (c[0] + 1, c[1]), (c[0], c[1] + 2), (c[0] + 1, c[1] + 1), (c[0] + 9, c[1]), (c[0] - 2, c[1])]
    rec = [(w + 3, w + 4), (w + 3, w + 4), (w + 30, w + 7), (w + 3, w + 4), (2, 3), (w + 30, w + 7)]
    amp = [0.8, -0.5, 0.3, 1.1, -0.9, 0.4]
    return src, rec, amp


@pytest.mark.parametrize("prec", [64, 32])
def test_overlapping_points_forward_and_adjoint(prec):
    import torch
    N, w, steps, f, t0 = (48, 40), 8, 25, 0.1, 10.0
    src, rec, amp = _points(w)
    u0 = gaussian_u0(N, w, 4)
    s = make_solver(N, w, prec, adjoint=True)
    s.set_initial(torch.from_numpy(u0))
    s.set_sources(src, amp, f, t0)
    tr = s.set_receivers(rec, steps)
    s.step(steps)
    got = [s.read(k).double().cpu().numpy() for k in range(6)]
    tr_got = tr.double().cpu().numpy()
    rng = np.random.default_rng(3)
    residual = rng.normal(scale=0.1, size=(steps, len(rec)))
    s.adjoint_reset()
    gu, ga = s.adjoint_step(steps, torch.from_numpy(residual))
    gu = gu.double().cpu().numpy()
    s.close()

    g = oracle_grid(N, w)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    srcd = {"idx": [g.flat(c) for c in src], "amp": amp, "f_peak": f, "t_delay": t0}
    ridx = [g.flat(c) for c in rec]
    want, tr_want = oracle.rk4(g, y, steps, 0.5, sources=srcd, receivers=ridx)
    for k in range(6):
        assert_close(got[k], want[k], prec, repr((k,)))
    assert_close(tr_got, tr_want, prec)
    # duplicate receivers read the same value
    assert np.array_equal(tr_got[:, 0], tr_got[:, 1]) and np.array_equal(tr_got[:, 0], tr_got[:, 3])
    yb, gamp = oracle.adjoint(g, g.zeros_state(), steps, 0.5, steps, sources=srcd, receivers=ridx,
                              residual=residual)
    assert_close(gu, yb[0], prec)
    assert rel_l2(ga, gamp) <= (1e-11 if prec == 64 else 1e-5), (ga, gamp)
