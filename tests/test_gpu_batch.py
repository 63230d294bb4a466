"""Batched stepping of many independent 2D grids (pml_batch_*) against the FP64 oracle.

Every grid of a batch is stepped by the oracle on its own; the batch must reproduce each
grid's fields to the precision's tolerance (FP64 <= 1e-12 relative L2 per field, FP32
<= 1e-5).  Step counts of at least 32 run through the captured CUDA graph.
"""
import numpy as np
import pytest

import oracle
from paper_1804_01390_gb300 import workloads as wk

from ._helpers import assert_close, TOL, gaussian_u0, make_solver, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu

# uneven sizes and widths: several strips and row blocks, ragged tails, a grid without a
# layer (w = 0) and one whose layer-free run is empty (N = 2, w = 4)
GRIDS = [((150, 90), 12), ((40, 33), 0), ((2, 2), 4), ((64, 201), 6), ((23, 47), 5), ((300, 70), 9)]


def _initial(N, w, seed):
    T = tuple(n + 2 * w for n in N)
    rng = np.random.default_rng(seed)
    u0 = gaussian_u0(N, w, seed) + rng.normal(scale=0.3, size=T[::-1])
    v0 = rng.normal(scale=0.3, size=T[::-1])
    return u0, v0


def _oracle_fields(N, w, u0, v0, steps):
    g = oracle_grid(N, w)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    y[1] = v0.reshape(-1)
    out, _ = oracle.rk4(g, y, steps, 0.5)
    T = tuple(n + 2 * w for n in N)
    return [out[f].reshape(T[::-1]) for f in range(6)]


def _make(prec, grids=GRIDS, seed0=100):
    import torch
    solvers, inits = [], []
    for k, (N, w) in enumerate(grids):
        s = make_solver(N, w, prec)
        u0, v0 = _initial(N, w, seed0 + k)
        s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
        solvers.append(s)
        inits.append((u0, v0))
    return solvers, inits


def _check(solvers, inits, steps, prec, grids=GRIDS):
    for k, ((N, w), s, (u0, v0)) in enumerate(zip(grids, solvers, inits)):
        want = _oracle_fields(N, w, u0, v0, steps)
        assert s.step_count == steps
        for f in range(6):
            assert_close(s.read(f).double().cpu().numpy(), want[f], prec, repr((k, N, w, f)))


@pytest.mark.parametrize("prec", [64, 32])
def test_batch_every_variant_matches_oracle(prec):
    from paper_1804_01390_gb300.solver import PMLBatch
    probe, _ = _make(prec, GRIDS[:1])
    nvar = PMLBatch(probe).variant_count
    for v in range(nvar):
        solvers, inits = _make(prec)
        b = PMLBatch(solvers)
        b.set_variant(v)
        b.step(35)   # one graph replay of 32 steps, then 3 single steps
        _check(solvers, inits, 35, prec)
        b.close()
        for s in solvers:
            s.close()


def test_batch_info_counts():
    from paper_1804_01390_gb300.solver import PMLBatch
    solvers, _ = _make(32)
    b = PMLBatch(solvers)
    ngrid, items, tiles, ctas = b.info()
    assert ngrid == len(GRIDS)
    assert items > 0 and tiles > 0 and ctas > 0
    # the grid with an empty layer-free run and the layer-free grid still step correctly
    b.close()


def test_batch_equals_single_context_kernels():
    """Same kernel shape, same arithmetic: the batched launch reproduces the per-context
    launch bit for bit (a consistency check of the batching; the oracle checks above are
    the parity claim)."""
    import torch
    from paper_1804_01390_gb300 import _lib
    from paper_1804_01390_gb300.solver import PMLBatch
    a, _ = _make(32)
    b, _ = _make(32)
    for s in a:
        _lib.pml_set_variant(s.ctx, 0)   # interior shape (4 columns per lane, 6-row boxes, 3 stages)
        s.step(40)
    batch = PMLBatch(b)
    batch.set_variant(0)                 # the same shape, 64 rows per work item
    batch.step(40)
    for x, y in zip(a, b):
        for f in range(6):
            assert torch.equal(x.read(f), y.read(f)), f


def test_batch_odd_parity_and_interleaving():
    """Batch steps starting from the odd ping-pong half, mixed with single-context steps."""
    from paper_1804_01390_gb300.solver import PMLBatch
    solvers, inits = _make(64)
    for s in solvers:
        s.step(1)
    b = PMLBatch(solvers)
    b.step(40)       # odd start: one single step, then a graph replay, then singles
    for s in solvers:
        s.step(3)
    b.step(33)
    b.step(0)
    _check(solvers, inits, 77, 64)


def test_batch_rejects_invalid_sets():
    from paper_1804_01390_gb300 import _lib
    from paper_1804_01390_gb300.solver import PMLBatch
    a = make_solver((40, 40), 4, 32)
    d = make_solver((40, 40), 4, 64)
    t = make_solver((16, 16, 16), 4, 32)
    with pytest.raises(_lib.PMLError) as e:
        PMLBatch([a, d])
    assert e.value.status == _lib.PML_EINVAL
    with pytest.raises(_lib.PMLError) as e:
        PMLBatch([a, t])
    assert e.value.status == _lib.PML_EINVAL
    with pytest.raises(_lib.PMLError) as e:
        PMLBatch([a, a])
    assert e.value.status == _lib.PML_EINVAL
    b2 = make_solver((50, 30), 5, 32)
    b = PMLBatch([a, b2])
    a.step(1)                                  # parities now differ
    with pytest.raises(_lib.PMLError) as e:
        b.step(4)
    assert e.value.status == _lib.PML_ESTATE
    b2.step(1)
    a.set_sources([[24, 24]], [1.0], 0.1, 15.0)
    with pytest.raises(_lib.PMLError) as e:
        b.step(4)
    assert e.value.status == _lib.PML_ESTATE
    a.set_sources([], [], 0.1, 15.0)
    b.step(4)
    assert a.step_count == 5 and b2.step_count == 5
    with pytest.raises(_lib.PMLError):
        b.set_variant(99)


def _patch_oracle(u0, v0, sig, x, y, k, Rp):
    """Oracle (U, V) at vertex (x, y) after k steps from a periodic patch of radius
    Rp >= 4k + 1 around it (the patch wrap never reaches the centre)."""
    Ty, Tx = u0.shape
    xs = (np.arange(x - Rp, x + Rp + 1)) % Tx
    ys = (np.arange(y - Rp, y + Rp + 1)) % Ty
    g = oracle.Grid((2 * Rp + 1, 2 * Rp + 1), 1.0, [sig[0][xs], sig[1][ys]])
    st = g.zeros_state()
    st[0] = u0[np.ix_(ys, xs)].reshape(-1)
    st[1] = v0[np.ix_(ys, xs)].reshape(-1)
    out, _ = oracle.rk4(g, st, k, 0.5)
    c = g.flat((Rp, Rp))
    return out[0][c], out[1][c]


def test_full_size_batched_96_grids_sampled():
    """The 96-grid workload (sides 256..2048, layers 16..32, FP32) in the benchmark's
    launch configuration (autotuned variant, graph replay): 32 steps, then vertices of
    four grids sampled over the interior, the layer, the corners and the periodic seam,
    each recomputed by the oracle on a local patch."""
    import torch
    from paper_1804_01390_gb300.solver import PMLBatch
    wls = wk.cfg4()
    rng = np.random.default_rng(44)
    sizes = [wl.N[0] * wl.N[1] for wl in wls]
    check = sorted({0, int(np.argmin(sizes)), int(np.argmax(sizes)), 57})
    solvers, inits = [], {}
    for k, wl in enumerate(wls):
        s = make_solver(wl.N, wl.w, 32)
        u0 = wk.initial_field(wl)
        if k in check:   # structure in the layer, a corner and across the seam
            T = wl.T
            u0[:40, :40] += rng.normal(scale=0.2, size=(40, 40))
            u0[-40:, T[0] // 2:T[0] // 2 + 40] += rng.normal(scale=0.2, size=(40, 40))
            u0[T[1] // 2:T[1] // 2 + 40, -20:] += rng.normal(scale=0.2, size=(40, 20))
            inits[k] = u0.copy()
        s.set_initial(torch.from_numpy(u0))
        solvers.append(s)
    b = PMLBatch(solvers)
    b.autotune(4)
    for k, wl in enumerate(wls):   # autotuning advanced the state: start again
        u0 = inits[k] if k in check else wk.initial_field(wl)
        solvers[k].set_initial(torch.from_numpy(u0))
    steps = 32
    b.step(steps)
    for k in check:
        wl = wls[k]
        T = wl.T
        U = solvers[k].read(0).double().cpu().numpy()
        V = solvers[k].read(1).double().cpu().numpy()
        u0 = inits[k]
        v0 = np.zeros_like(u0)
        sig = [oracle.sigma_profile(n, wl.w, oracle.KIND_POWER, 2.0, 2.0) for n in wl.N]
        pts = [(0, 0), (T[0] - 1, T[1] - 1), (5, 17), (T[0] // 2 + 10, T[1] - 3), (T[0] - 8, T[1] // 2 + 20),
               (wl.w, wl.w), (T[0] // 2, T[1] // 2)]
        pts += [(int(x), int(y)) for x, y in zip(rng.integers(0, T[0], 8), rng.integers(0, T[1], 8))]
        got, want = [], []
        for (x, y) in pts:
            wu, wv = _patch_oracle(u0, v0, sig, x, y, steps, 4 * steps + 2)
            got += [U[y, x], V[y, x]]
            want += [wu, wv]
        assert_close(got, want, 32, repr((k)))
    b.close()


def test_batch_of_wall_boxes_every_variant():
    """A batch of contexts backed by reflecting walls (one-step and two-step shapes) against
    the oracle's wall mode, per grid."""
    import torch
    from paper_1804_01390_gb300.solver import PMLBatch, PMLSolver
    grids = [((60, 44), 6), ((23, 41), 1), ((90, 37), 9)]

    def make():
        solvers, inits = [], []
        for k, (N, w) in enumerate(grids):
            s = PMLSolver(N, w, sigma="quadratic", sigma_max=2.0, precision=32, device=torch.device("cuda:0"),
                          wall=True)
            u0, v0 = _initial(N, w, 500 + k)
            s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
            solvers.append(s)
            inits.append((u0, v0))
        return solvers, inits

    probe, _ = make()
    nvar = PMLBatch(probe).variant_count
    for v in range(nvar):
        solvers, inits = make()
        b = PMLBatch(solvers)
        b.set_variant(v)
        b.step(35)
        for k, ((N, w), s, (u0, v0)) in enumerate(zip(grids, solvers, inits)):
            g0 = oracle_grid(N, w)
            g = oracle.Grid(g0.T, 1.0, [np.concatenate([s_[:-1], [0.0]]) for s_ in g0.sigmas], wall=True)
            y = g.zeros_state()
            y[0] = u0.reshape(-1)
            y[1] = v0.reshape(-1)
            want, _ = oracle.rk4(g, y, 35, 0.5)
            for f in range(6):
                got = s.read(f).double().cpu().numpy()
                assert_close(got, want[f].reshape(got.shape), 32, repr((v, k, f)))
        b.close()
        for s in solvers:
            s.close()
