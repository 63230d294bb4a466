"""3D layer frame by slab tiles (variant 2 of an FP32 3D context: per-class halos of 4
along axes with damping within reach and 2 along the others, two columns per thread)
against the FP64 oracle: forward steps with quadratic, constant and random damping, thin
and wide boxes, layers of 1 to 6 cells, z runs split into several work items, reflecting
walls, spacings other than 1, the transposed step with sources and injected residuals, and
the 560^3 workload in the benchmark's launch configuration on sampled vertices.  The slab
tiles evaluate the same Horner form as the other 3D variants, so all three agree to
rounding."""
import numpy as np
import pytest

import oracle
from paper_1804_01390_gb300 import workloads as wk

from ._helpers import assert_close, gaussian_u0, make_solver, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu

CASES = [((21, 18, 15), 5, "quadratic"), ((130, 14, 12), 6, "constant"), ((16, 27, 20), 4, "random"),
         ((14, 12, 150), 4, "quadratic"), ((9, 30, 10), 3, "constant"), ((40, 33, 29), 1, "quadratic"),
         ((26, 44, 18), 2, "random"), ((20, 16, 24), 0, "quadratic")]


def _state(N, w, seed):
    rng = np.random.default_rng(seed)
    T = tuple(n + 2 * w for n in N)
    u0 = gaussian_u0(N, w, seed) + rng.normal(scale=0.3, size=T[::-1])
    v0 = rng.normal(scale=0.3, size=T[::-1])
    return rng, u0, v0


def _gpu(N, w, sigma, draws, u0, v0, steps, variant, wall=False, dt=0.4, h=1.0):
    import torch
    from paper_1804_01390_gb300 import _lib
    from paper_1804_01390_gb300.solver import PMLSolver
    s = PMLSolver(N, w, h=h, dt=dt, sigma=sigma, sigma_max=2.0, draws=draws, precision=32,
                  device=torch.device("cuda:0"), wall=wall)
    _lib.pml_set_variant(s.ctx, variant)
    assert _lib.pml_get_variant(s.ctx) == (variant, 3)
    s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
    s.step(steps)
    s.sync()
    got = [s.read(f).double().cpu().numpy() for f in range(8)]
    s.close()
    return got


@pytest.mark.parametrize("N,w,sigma", CASES)
def test_slab_forward_parity(N, w, sigma):
    rng, u0, v0 = _state(N, w, 3 * sum(N) + w)
    draws = [rng.random(n + 2 * w) for n in N] if sigma == "random" else None
    steps = 13
    got = _gpu(N, w, sigma, draws, u0, v0, steps, 2)
    g = oracle_grid(N, w, sigma, 2.0, draws)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    y[1] = v0.reshape(-1)
    want, _ = oracle.rk4(g, y, steps, 0.4)
    for f in range(8):
        assert_close(got[f], want[f], 32, repr((f,)))
    ref = _gpu(N, w, sigma, draws, u0, v0, steps, 0)
    for f in range(8):
        assert rel_l2(got[f], ref[f]) <= 1e-6, f


@pytest.mark.parametrize("h", [0.05, 2.5])
def test_slab_other_spacing(h):
    N, w = (23, 19, 21), 5
    rng, u0, v0 = _state(N, w, 41)
    got = _gpu(N, w, "quadratic", None, u0, v0, 11, 2, dt=0.4 * h, h=h)
    g = oracle_grid(N, w, h=h)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    y[1] = v0.reshape(-1)
    want, _ = oracle.rk4(g, y, 11, 0.4 * h)
    for f in range(8):
        assert_close(got[f], want[f], 32, repr((h, f)))


def test_slab_wall():
    N, w = (24, 19, 17), 4
    rng, u0, v0 = _state(N, w, 78)
    got = _gpu(N, w, "quadratic", None, u0, v0, 15, 2, wall=True)
    g0 = oracle_grid(N, w)
    sig = [np.concatenate([s_[:-1], [0.0]]) for s_ in g0.sigmas]
    g = oracle.Grid(g0.T, 1.0, sig, wall=True)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    y[1] = v0.reshape(-1)
    want, _ = oracle.rk4(g, y, 15, 0.4)
    for f in range(8):
        assert_close(got[f], want[f], 32, repr((f,)))


def test_slab_adjoint_with_points():
    import torch
    from paper_1804_01390_gb300 import _lib
    N, w, steps, f, t0 = (18, 16, 14), 4, 12, 0.1, 8.0
    rng = np.random.default_rng(6)
    src = [(w + 8, w + 7, w + 6), (w + 9, w + 7, w + 6)]
    rec = [(w + 2, w + 3, w + 4), (1, 2, 3), (w + 10, w + 10, w + 9)]
    amp = [0.6, -0.4]
    residual = rng.normal(scale=0.1, size=(steps, len(rec)))
    s = make_solver(N, w, 32, adjoint=True, dt=0.4)
    _lib.pml_set_variant(s.ctx, 2)
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
    assert_close(gu.double().cpu().numpy(), yb[0], 32)
    for k, fk in enumerate(fields):
        assert_close(fk, yb[k], 32, repr((k,)))
    assert rel_l2(ga, gamp) <= 1e-5


def _patch3(u0, sig, c, k, Rp):
    """Oracle (U, V) at vertex c after k steps from a periodic patch of radius Rp >= 4k + 1."""
    Tz, Ty, Tx = u0.shape
    idx = [np.arange(c[a] - Rp, c[a] + Rp + 1) % (Tx, Ty, Tz)[a] for a in range(3)]
    g = oracle.Grid((2 * Rp + 1,) * 3, 1.0, [sig[a][idx[a]] for a in range(3)])
    st = g.zeros_state()
    st[0] = u0[np.ix_(idx[2], idx[1], idx[0])].reshape(-1)
    out, _ = oracle.rk4(g, st, k, 0.5)
    m = g.flat((Rp, Rp, Rp))
    return out[0][m], out[1][m]


def test_slab_full_size_cfg3_sampled():
    """The 512^3 + 24-cell workload in the benchmark's configuration (slab variant, 2
    steps), vertices sampled over every class of the frame (faces, edges, corners, the
    periodic seam) and the interior, each recomputed by the oracle on a local patch."""
    import torch
    from paper_1804_01390_gb300 import _lib
    wl = wk.cfg3()
    T = wl.T
    u0 = wk.initial_field(wl).astype(np.float32)
    rng = np.random.default_rng(19)
    u0[:30, :30, :30] += rng.normal(scale=0.2, size=(30, 30, 30)).astype(np.float32)        # a corner
    u0[-30:, 250:280, 520:550] += rng.normal(scale=0.2, size=(30, 30, 30)).astype(np.float32)   # z seam, x face
    u0[250:280, 530:560, 250:280] += rng.normal(scale=0.2, size=(30, 30, 30)).astype(np.float32)  # y face
    s = make_solver(wl.N, wl.w, 32)
    _lib.pml_set_variant(s.ctx, 2)
    s.set_initial(torch.from_numpy(u0))
    k = 2
    s.step(k)
    U = s.read(0).cpu().numpy()
    V = s.read(1).cpu().numpy()
    s.close()
    sig = [oracle.sigma_profile(n, wl.w, oracle.KIND_POWER, 2.0, 2.0) for n in wl.N]
    u64 = u0.astype(np.float64)
    pts = [(5, 7, 3), (555, 552, 2), (20, 20, 20), (540, 265, 10), (265, 545, 265), (265, 265, 548),
           (0, 0, 0), (559, 559, 559), (24, 300, 300), (300, 25, 300), (300, 300, 535), (26, 26, 300)]
    pts += [tuple(int(v) for v in rng.integers(0, T[0], 3)) for _ in range(20)]
    got, want = [], []
    for c in pts:
        wu, wv = _patch3(u64, sig, c, k, 4 * k + 2)
        got += [U[c[2], c[1], c[0]], V[c[2], c[1], c[0]]]
        want += [wu, wv]
    assert_close(got, want, 32, "sampled vertices (U and V)")
