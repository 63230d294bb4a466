"""Two forward steps per pass (temporal blocking depth 2, 2D FP32) against the oracle.

Every two-step kernel variant is compared with the FP64 oracle (1e-5 relative L2, the
FP32 bar) on boxes with and without a layer, with random damping, with reflecting walls,
on boxes too small for any layer-free vertex to remain after shrinking the run, and for
odd step counts (the last step then runs alone).  Where something has to happen between
the two steps (sources, receiver rows) the library steps one at a time: the results must
then be bit-identical to those of the one-step variant.  At the benchmark's full size
(8192^2 + 32-cell layer) sampled vertices are checked against oracle patches.
"""
import numpy as np
import pytest

import oracle
from paper_1804_01390_gb300 import workloads as wk

from ._helpers import assert_close, TOL, gaussian_u0, make_solver, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu


def _two_step_variants(s):
    from paper_1804_01390_gb300 import _lib
    _, n = _lib.pml_get_variant(s.ctx)
    out = []
    for v in range(n):
        _lib.pml_set_variant(s.ctx, v)
        if _lib.pml_get_time_block(s.ctx) == 2:
            out.append(v)
    return out


def _oracle_run(N, w, sigma, draws, u0, v0, steps, wall=False):
    g = oracle_grid(N, w, sigma, 2.0, draws)
    if wall:   # the wall replaces the wrap edge T-1 -> 0
        sig = [np.concatenate([s_[:-1], [0.0]]) for s_ in g.sigmas]
        g = oracle.Grid(g.T, 1.0, sig, wall=True)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    y[1] = v0.reshape(-1)
    out, _ = oracle.rk4(g, y, steps, 0.5)
    return out


CASES = [
    ((290, 61), 7, "quadratic", False, 14),
    ((96, 130), 16, "random", False, 9),     # odd: four pairs, then one single step
    ((64, 72), 0, "quadratic", False, 10),   # no layer: the run is the whole periodic box
    ((120, 90), 12, "constant", True, 12),   # reflecting walls
    ((5, 7), 3, "quadratic", False, 8),      # run shrunk to nothing: layer passes only
    ((200, 4), 20, "quadratic", False, 6),   # run empty on one axis
]


@pytest.mark.parametrize("N,w,sigma,wall,steps", CASES)
def test_two_step_variants_match_oracle(N, w, sigma, wall, steps):
    import torch
    from paper_1804_01390_gb300 import _lib
    from paper_1804_01390_gb300.solver import PMLSolver
    rng = np.random.default_rng(sum(N) + w)
    T = tuple(n + 2 * w for n in N)
    draws = [rng.random(t) for t in T] if sigma == "random" else None
    u0 = gaussian_u0(N, w, 5) + rng.normal(scale=0.1, size=T[::-1])
    v0 = 0.2 * rng.normal(size=T[::-1])
    want = _oracle_run(N, w, sigma, draws, u0, v0, steps, wall=wall)
    s = PMLSolver(N, w, sigma=sigma, sigma_max=2.0, draws=draws, precision=32, device=torch.device("cuda:0"),
                  wall=wall)
    vs = _two_step_variants(s)
    assert len(vs) >= 1
    for v in vs:
        _lib.pml_set_variant(s.ctx, v)
        s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
        s.step(steps)
        assert s.step_count == steps
        for f in range(6):
            got = s.read(f).double().cpu().numpy()
            assert_close(got, want[f].reshape(got.shape), 32, repr((v, f)))
    s.close()


def test_two_steps_as_accurate_as_single_steps():
    """Two-step pairs against single steps of the same FP32 library over 40 steps: the
    pairs only change the rounding of the first step's values where the layer passes take
    over from the closed form, so per field their error against the FP64 oracle stays at
    the level of the single steps' own error (both far inside the FP32 bar)."""
    import torch
    from paper_1804_01390_gb300 import _lib
    N, w, steps = (300, 260), 16, 40
    rng = np.random.default_rng(8)
    T = tuple(n + 2 * w for n in N)
    u0 = gaussian_u0(N, w, 9) + rng.normal(scale=0.1, size=T[::-1])
    g = oracle_grid(N, w)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    want, _ = oracle.rk4(g, y, steps, 0.5)
    s = make_solver(N, w, 32)
    vs = _two_step_variants(s)
    runs = []
    for v in (0, vs[0]):
        _lib.pml_set_variant(s.ctx, v)
        s.set_initial(torch.from_numpy(u0))
        s.step(steps)
        runs.append([s.read(f).double().cpu().numpy() for f in range(6)])
    s.close()
    for f in range(6):
        e1 = rel_l2(runs[0][f], want[f].reshape(runs[0][f].shape))
        e2 = rel_l2(runs[1][f], want[f].reshape(runs[1][f].shape))
        assert e2 <= 2.0 * e1 + 1e-7, (f, e1, e2)
        assert e2 <= TOL[32] / 4, (f, e2)


def test_sources_and_receivers_step_singly_bit_exact():
    """With sources or receiver rows the two-step variant steps one at a time: the state
    and the traces are bit-identical to those of the one-step variant."""
    import torch
    from paper_1804_01390_gb300 import _lib
    N, w, steps = (140, 120), 12, 11
    u0 = gaussian_u0(N, w, 3)
    src = [(w + 70, w + 60), (w + 30, w + 90)]
    rec = [(w + 10, w + 10), (w + 100, w + 50), (2, 3)]
    out = []
    for which in ("one", "two"):
        s = make_solver(N, w, 32)
        vs = _two_step_variants(s)
        _lib.pml_set_variant(s.ctx, 0 if which == "one" else vs[0])
        s.set_initial(torch.from_numpy(u0))
        s.set_sources(src, [0.5, -0.7], 0.1, 10.0)
        s.set_receivers(rec, steps)
        s.step(steps)
        tr = s.traces.clone()
        st = [s.read(f).clone() for f in range(6)]
        out.append((st, tr))
        s.close()
    for a, b in zip(out[0][0], out[1][0]):
        assert torch.equal(a, b)
    assert torch.equal(out[0][1], out[1][1])


def test_trace_buffer_full_allows_pairs():
    """Once the receiver buffer is full no row is recorded, so steps pair up again; the
    state still matches the oracle."""
    import torch
    from paper_1804_01390_gb300 import _lib
    N, w = (100, 80), 10
    u0 = gaussian_u0(N, w, 4)
    s = make_solver(N, w, 32)
    vs = _two_step_variants(s)
    _lib.pml_set_variant(s.ctx, vs[0])
    s.set_initial(torch.from_numpy(u0))
    s.set_receivers([(w + 5, w + 5)], 3)
    s.step(12)
    g = oracle_grid(N, w)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    want, _ = oracle.rk4(g, y, 12, 0.5)
    for f in range(6):
        got = s.read(f).double().cpu().numpy()
        assert_close(got, want[f].reshape(got.shape), 32)
    s.close()


def _patch_oracle(u0, sig, x, y, k, Rp):
    Ty, Tx = u0.shape
    xs = (np.arange(x - Rp, x + Rp + 1)) % Tx
    ys = (np.arange(y - Rp, y + Rp + 1)) % Ty
    g = oracle.Grid((2 * Rp + 1, 2 * Rp + 1), 1.0, [sig[0][xs], sig[1][ys]])
    st = g.zeros_state()
    st[0] = u0[np.ix_(ys, xs)].reshape(-1)
    out, _ = oracle.rk4(g, st, k, 0.5)
    c = g.flat((Rp, Rp))
    return out[0][c], out[1][c]


@pytest.mark.parametrize("variant_pos", [0, -1])
def test_full_size_cfg2_two_step_sampled(variant_pos):
    """8192^2 + 32-cell layer with a two-step variant (as the benchmark may select it):
    four steps (two pairs), then vertices sampled over the interior, the band where the
    layer passes take over, the layer, corners and the periodic seam, each recomputed by
    the oracle on a local patch."""
    import torch
    from paper_1804_01390_gb300 import _lib
    wl = wk.cfg2()
    T = wl.T
    u0 = wk.initial_field(wl)
    rng = np.random.default_rng(13)
    u0[:40, :40] += rng.normal(scale=0.2, size=(40, 40))
    u0[-40:, 4000:4040] += rng.normal(scale=0.2, size=(40, 40))
    u0[4000:4060, 20:80] += rng.normal(scale=0.2, size=(60, 60))   # across the x interface
    s = make_solver(wl.N, wl.w, 32)
    vs = _two_step_variants(s)
    _lib.pml_set_variant(s.ctx, vs[variant_pos])
    s.set_initial(torch.from_numpy(u0))
    k = 4
    s.step(k)
    U = s.read(0).double().cpu().numpy()
    V = s.read(1).double().cpu().numpy()
    s.close()
    sig = [oracle.sigma_profile(n, wl.w, oracle.KIND_POWER, 2.0, 2.0) for n in wl.N]
    w = wl.w
    pts = [(0, 0), (T[0] - 1, T[1] - 1), (5, 17), (33, 33), (32, 4000), (4100, 8255), (8230, 10),
           (4020, 8240), (64, 64), (4000, 4000)]
    # the band of the run where the second layer pass writes (run shrunk by 2) and where
    # the first pass's values feed it (shrunk by 6)
    for d in range(0, 9):
        pts += [(w + 1 + d, 4030), (T[0] - w - 2 - d, 4030), (4030, w + 1 + d), (40 + d, T[1] - w - 2 - d)]
    pts += [(int(a), int(b)) for a, b in zip(rng.integers(0, T[0], 60), rng.integers(0, T[1], 60))]
    got, want = [], []
    for (x, y) in pts:
        wu, wv = _patch_oracle(u0, sig, x, y, k, 4 * k + 2)
        got += [U[y, x], V[y, x]]
        want += [wu, wv]
    assert_close(got, want, 32, "sampled vertices (U and V)")


# ------------------------------------------------------------------------------------
# batched mode
# ------------------------------------------------------------------------------------
BGRIDS = [((150, 90), 12), ((40, 33), 0), ((2, 2), 4), ((64, 201), 6), ((23, 47), 5), ((300, 70), 9)]


def _batch_make(grids=BGRIDS, seed0=300):
    import torch
    solvers, inits = [], []
    for k, (N, w) in enumerate(grids):
        s = make_solver(N, w, 32)
        T = tuple(n + 2 * w for n in N)
        rng = np.random.default_rng(seed0 + k)
        u0 = gaussian_u0(N, w, seed0 + k) + rng.normal(scale=0.3, size=T[::-1])
        v0 = rng.normal(scale=0.3, size=T[::-1])
        s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
        solvers.append(s)
        inits.append((u0, v0))
    return solvers, inits


def _batch_two_step_variants(b):
    out = []
    for v in range(b.variant_count):
        b.set_variant(v)
        if b.time_block() == 2:
            out.append(v)
    return out


def test_batch_two_step_odd_parities_match_oracle():
    """Two-step batch variants from the odd ping-pong half, with a second-pass counter parity
    that must be realigned before the graph replay (1 + 2 + 35 + 5 steps)."""
    from paper_1804_01390_gb300.solver import PMLBatch
    probe, _ = _batch_make(BGRIDS[:1])
    vs = _batch_two_step_variants(PMLBatch(probe))
    assert vs
    for v in vs:
        solvers, inits = _batch_make()
        b = PMLBatch(solvers)
        b.set_variant(v)
        assert b.time_block() == 2
        for n in (1, 2, 35, 5):
            b.step(n)
        for k, ((N, w), s, (u0, v0)) in enumerate(zip(BGRIDS, solvers, inits)):
            want = _oracle_run(N, w, "quadratic", None, u0, v0, 43)
            assert s.step_count == 43
            for f in range(6):
                got = s.read(f).double().cpu().numpy()
                assert_close(got, want[f].reshape(got.shape), 32, repr((v, k, f)))
        b.close()
        for s in solvers:
            s.close()


def test_batch_two_step_equals_single_context_two_step():
    """Same arithmetic per vertex (4 columns per lane, the same frame tables): the batched
    two-step launches reproduce the per-context two-step launches bit for bit."""
    import torch
    from paper_1804_01390_gb300 import _lib
    from paper_1804_01390_gb300.solver import PMLBatch
    a, _ = _batch_make()
    c, _ = _batch_make()
    for s in a:
        vs = _two_step_variants(s)
        _lib.pml_set_variant(s.ctx, vs[1])   # 4 columns per lane, 3-row boxes
        s.step(40)
    batch = PMLBatch(c)
    bv = _batch_two_step_variants(batch)
    batch.set_variant(bv[0])
    batch.step(40)
    for x, y in zip(a, c):
        for f in range(6):
            assert torch.equal(x.read(f), y.read(f)), f


# ------------------------------------------------------------------------------------
# transposed steps
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("N,w,wall", [((290, 61), 7, False), ((96, 130), 16, False), ((120, 90), 12, True),
                                      ((64, 72), 0, False), ((5, 7), 3, False)])
def test_two_step_transposed_matches_oracle(N, w, wall):
    """One transposed step with receiver residuals (a nonzero adjoint state), then 12 more
    with nothing injected: those pair up.  Against the oracle's adjoint with the same residual
    rows (the first one nonzero)."""
    import torch
    from paper_1804_01390_gb300 import _lib
    from paper_1804_01390_gb300.solver import PMLSolver
    rng = np.random.default_rng(sum(N) + w + 7)
    T = tuple(n + 2 * w for n in N)
    rec = [tuple(int(rng.integers(0, t)) for t in T) for _ in range(5)]
    steps = 13
    residual = np.zeros((steps, len(rec)))
    residual[0] = rng.normal(size=len(rec))
    s = PMLSolver(N, w, sigma="quadratic", sigma_max=2.0, precision=32, device=torch.device("cuda:0"),
                  adjoint=True, wall=wall)
    vs = _two_step_variants(s)
    _lib.pml_set_variant(s.ctx, vs[0])
    s.set_initial(torch.from_numpy(gaussian_u0(N, w, 3)))
    s.set_receivers(rec, steps)
    s.step(steps)
    s.adjoint_reset()
    s.adjoint_step(1, torch.from_numpy(residual[:1].copy()))
    gu, _ = s.adjoint_step(steps - 1)
    fields = [s.adjoint_read(k).double().cpu().numpy() for k in range(6)]
    s.close()
    g0 = oracle_grid(N, w)
    if wall:
        g0 = oracle.Grid(g0.T, 1.0, [np.concatenate([s_[:-1], [0.0]]) for s_ in g0.sigmas], wall=True)
    yb, _ = oracle.adjoint(g0, g0.zeros_state(), steps, 0.5, steps, receivers=[g0.flat(c) for c in rec],
                           residual=residual)
    assert_close(gu.double().cpu().numpy(), yb[0], 32)
    for k, fk in enumerate(fields):
        assert_close(fk, yb[k], 32, repr((k,)))
