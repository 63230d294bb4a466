"""Grid spacings other than h = 1 in the 3D kernels and in the batched mode, against the FP64
oracle run with the same h.

The operator carries 1/h^2 (Laplacian), 1/h (damping terms) and 1/(2h) (centred difference)
factors (eq:DiscretePML), and the closed-form interior step carries powers of dt/h; at h = 1
a factor taken from the wrong power of h goes unseen.  Here every run uses dt = h/2 and a
damping of order 2/h.  The batch mixes grids of different spacings, so each grid's own
coefficients must reach its tiles (one-step and two-step shapes, graph replays).
"""
import numpy as np
import pytest

import oracle

from ._helpers import assert_close, TOL, gaussian_u0, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu


def _solver(N, w, h, prec, sigma="quadratic"):
    import torch
    from paper_1804_01390_gb300.solver import PMLSolver
    return PMLSolver(N, w, h=h, dt=h / 2, sigma=sigma, sigma_max=2.0 / h, precision=prec,
                     device=torch.device("cuda:0"))


def _initial(N, w, seed):
    T = tuple(n + 2 * w for n in N)
    rng = np.random.default_rng(seed)
    u0 = gaussian_u0(N, w, seed) + rng.normal(scale=0.3, size=T[::-1])
    v0 = rng.normal(scale=0.3, size=T[::-1])
    return u0, v0


def _oracle(N, w, h, u0, v0, steps, sigma="quadratic"):
    g = oracle_grid(N, w, sigma, 2.0 / h, h=h)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    y[1] = v0.reshape(-1)
    out, _ = oracle.rk4(g, y, steps, h / 2)
    return out


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("prec", [64, 32])
def test_3d_spacing(variant, prec):
    import torch
    from paper_1804_01390_gb300 import _lib
    N, w, h, steps = (21, 18, 15), 5, 0.05, 11
    u0, v0 = _initial(N, w, 31)
    s = _solver(N, w, h, prec, "constant")
    _lib.pml_set_variant(s.ctx, variant)
    s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
    s.step(steps)
    got = [s.read(f).double().cpu().numpy() for f in range(8)]
    s.close()
    want = _oracle(N, w, h, u0, v0, steps, "constant")
    for f in range(8):
        assert_close(got[f], want[f], prec, repr((f,)))


GRIDS = [((150, 90), 12, 1.0 / 80), ((64, 45), 6, 0.37), ((40, 33), 0, 2.5), ((23, 47), 5, 1.0)]


@pytest.mark.parametrize("prec", [64, 32])
def test_batch_mixed_spacings(prec):
    import torch
    from paper_1804_01390_gb300.solver import PMLBatch
    solvers, inits = [], []
    for k, (N, w, h) in enumerate(GRIDS):
        s = _solver(N, w, h, prec)
        u0, v0 = _initial(N, w, 200 + k)
        s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
        solvers.append(s)
        inits.append((u0, v0))
    b = PMLBatch(solvers)
    b.step(35)          # one graph replay of 32 steps, then singles
    for (N, w, h), s, (u0, v0) in zip(GRIDS, solvers, inits):
        want = _oracle(N, w, h, u0, v0, 35)
        assert s.step_count == 35
        for f in range(6):
            assert_close(s.read(f).double().cpu().numpy(), want[f], prec, repr((N, h, f)))
    b.close()
    for s in solvers:
        s.close()
