"""3D parity of the CUDA path (through the C ABI) against the FP64 CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1804_01390_gb300 import workloads as wk

from ._helpers import assert_close, TOL, gaussian_u0, make_solver, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu

CASES3 = [
    ((21, 18, 15), 5, "quadratic"),
    ((130, 14, 12), 6, "constant"),    # two 120-column strips, ragged tail
    ((16, 27, 20), 4, "random"),
    ((20, 16, 24), 0, "quadratic"),    # no layer
    ((12, 13, 11), 2, "quadratic"),
    ((9, 30, 10), 3, "constant"),
]


@pytest.mark.parametrize("N,w,sigma", CASES3)
@pytest.mark.parametrize("prec", [64, 32])
def test_forward_parity_3d(N, w, sigma, prec):
    got, want = _run_3d_dt(N, w, prec, 17, sigma, seed=sum(N) + w)
    for f, (a, b) in enumerate(zip(got, want)):
        assert_close(a, b, prec, repr((f)))


def _run_3d_dt(N, w, prec, steps, sigma, seed, dt=0.4):
    import torch
    rng = np.random.default_rng(seed)
    draws = [rng.random(n + 2 * w) for n in N] if sigma == "random" else None
    T = tuple(n + 2 * w for n in N)
    u0 = gaussian_u0(N, w, seed) + rng.normal(scale=0.3, size=T[::-1])
    v0 = rng.normal(scale=0.3, size=T[::-1])
    s = make_solver(N, w, prec, sigma=sigma, draws=draws, dt=dt)
    s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
    s.step(steps)
    got = [s.read(f).double().cpu().numpy() for f in range(8)]
    s.close()
    g = oracle_grid(N, w, sigma, 2.0, draws)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    y[1] = v0.reshape(-1)
    want, _ = oracle.rk4(g, y, steps, dt)
    return got, want


def test_layout_tables_bit_exact_3d():
    N, w = (21, 18, 15), 5
    s = make_solver(N, w, 32)
    g = oracle_grid(N, w)
    for a in range(3):
        phi, psi, inner = s.layout(a)
        ophi, opsi, oin = oracle.layout_axis(g.sigmas[a], w + N[a] // 2)
        assert np.array_equal(phi, ophi) and np.array_equal(psi, opsi) and np.array_equal(inner, oin)
    s.close()


def test_sources_receivers_3d():
    import torch
    N, w = (30, 26, 22), 6
    coords = [(w + 5, w + 6, w + 7), (w + 20, w + 12, w + 15), (w + 14, w + 20, w + 3)]
    amp = [0.7, -0.4, 1.1]
    f, t0 = 0.1, 15.0
    rec = [(w + 2, w + 3, w + 4), (1, 2, 3), (w + 20, w + 12, w + 15)]
    steps = 40
    for prec in (64, 32):
        s = make_solver(N, w, prec)
        s.set_initial(torch.from_numpy(gaussian_u0(N, w, 3, 1)))
        s.set_sources(coords, amp, f, t0)
        tr = s.set_receivers(rec, steps)
        s.step(steps)
        got = s.read(0).double().cpu().numpy()
        gtr = tr.double().cpu().numpy()
        s.close()
        g = oracle_grid(N, w)
        y = g.zeros_state()
        y[0] = gaussian_u0(N, w, 3, 1).reshape(-1)
        src = {"idx": [g.flat(c) for c in coords], "amp": amp, "f_peak": f, "t_delay": t0}
        want, wtr = oracle.rk4(g, y, steps, 0.5, sources=src, receivers=[g.flat(c) for c in rec])
        assert_close(got, want[0], prec)
        assert_close(gtr, wtr, prec)


def test_norms_3d():
    import torch
    N, w = (24, 20, 18), 5
    s = make_solver(N, w, 64)
    u0 = gaussian_u0(N, w, 4)
    s.set_initial(torch.from_numpy(u0))
    s.step(11)
    g = oracle_grid(N, w)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    want, _ = oracle.rk4(g, y, 11, 0.5)
    lo = (w, w, w)
    hi = tuple(w + n - 1 for n in N)
    E = oracle.energy(g, want, lo, hi)
    nr = s.norms()
    s.close()
    assert abs(nr["energy"] - E) <= 1e-12 * E


def _patch3(u0, sig, x, y, z, k, Rp):
    Tz, Ty, Tx = u0.shape
    xs = np.arange(x - Rp, x + Rp + 1) % Tx
    ys = np.arange(y - Rp, y + Rp + 1) % Ty
    zs = np.arange(z - Rp, z + Rp + 1) % Tz
    n = 2 * Rp + 1
    g = oracle.Grid((n, n, n), 1.0, [sig[0][xs], sig[1][ys], sig[2][zs]])
    st = g.zeros_state()
    st[0] = u0[np.ix_(zs, ys, xs)].reshape(-1)
    out, _ = oracle.rk4(g, st, k, 0.5)
    c = g.flat((Rp, Rp, Rp))
    return out[0][c], out[1][c]


def test_full_size_cfg3_sampled():
    """Config 3 size (512^3 + 24-cell layer, FP32) with the z-streaming tile kernel of the
    frame (variant 0; the slab tiles that FP32 3D contexts use by default have their own
    full-size check): two steps, sampled vertices recomputed by the oracle on local
    patches."""
    import torch
    from paper_1804_01390_gb300 import _lib
    wl = wk.cfg3()
    T = wl.T
    u0 = wk.initial_field(wl)
    rng = np.random.default_rng(5)
    u0[:30, :30, :30] += rng.normal(scale=0.2, size=(30, 30, 30))     # corner, across the seams
    u0[-20:, 200:230, -25:] += rng.normal(scale=0.2, size=(20, 30, 25))
    s = make_solver(wl.N, wl.w, 32)
    _lib.pml_set_variant(s.ctx, 0)
    s.set_initial(torch.from_numpy(u0.astype(np.float32)))
    k = 2
    s.step(k)
    U = s.read(0).double().cpu().numpy()
    V = s.read(1).double().cpu().numpy()
    s.close()
    sig = [oracle.sigma_profile(n, wl.w, oracle.KIND_POWER, 2.0, 2.0) for n in wl.N]
    pts = [(0, 0, 0), (T[0] - 1, T[1] - 1, T[2] - 1), (5, 17, 9), (24, 24, 24), (25, 25, 25),
           (280, 280, 280), (535, 300, 559), (210, 3, 548), (12, 500, 556)]
    pts += [tuple(int(v) for v in rng.integers(0, 560, 3)) for _ in range(30)]
    got, want = [], []
    for (x, y, z) in pts:
        wu, wv = _patch3(u0, sig, x, y, z, k, 4 * k + 2)
        got += [U[z, y, x], V[z, y, x]]
        want += [wu, wv]
    assert_close(got, want, 32)
