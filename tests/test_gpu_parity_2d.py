"""2D parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 mode <= 1e-12 relative L2 on every field, FP32 mode <= 1e-5; integer
layout tables bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_1804_01390_gb300 import workloads as wk

from ._helpers import assert_close, TOL, gaussian_u0, make_solver, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu


def _noise(T, seed, scale=1.0):
    return np.random.default_rng(seed).normal(scale=scale, size=T[::-1])


def _run_both(N, w, prec, steps, sigma="quadratic", sigma_max=2.0, seed=0, noise=True):
    import torch
    rng = np.random.default_rng(seed)
    draws = None
    if sigma == "random":
        draws = [rng.random(n + 2 * w) for n in N]
    T = tuple(n + 2 * w for n in N)
    u0 = gaussian_u0(N, w, seed)
    v0 = np.zeros(T[::-1])
    if noise:
        u0 = u0 + _noise(T, seed + 1, 0.3)
        v0 = _noise(T, seed + 2, 0.3)
    s = make_solver(N, w, prec, sigma=sigma, sigma_max=sigma_max, draws=draws)
    s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
    s.step(steps)
    got = [s.read(f).double().cpu().numpy() for f in range(2 + 2 * len(N))]
    s.close()
    g = oracle_grid(N, w, sigma, sigma_max, draws)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    y[1] = v0.reshape(-1)
    want, _ = oracle.rk4(g, y, steps, 0.5)
    return got, want


CASES = [
    ((37, 29), 6, "quadratic"),
    ((300, 70), 9, "quadratic"),     # several 120-column strips and a ragged tail
    ((131, 97), 16, "constant"),
    ((64, 45), 12, "random"),
    ((40, 33), 0, "quadratic"),      # no layer: plain periodic wave equation
    ((23, 41), 1, "constant"),
    ((30, 21), 2, "quadratic"),
    ((17, 26), 3, "random"),
    ((9, 250), 5, "quadratic"),      # tall and narrow
]


@pytest.mark.parametrize("N,w,sigma", CASES)
@pytest.mark.parametrize("prec", [64, 32])
def test_forward_parity(N, w, sigma, prec):
    got, want = _run_both(N, w, prec, 23, sigma, seed=hash((N, w)) % 1000)
    for f, (a, b) in enumerate(zip(got, want)):
        assert_close(a, b, prec, repr((f)))


def test_every_interior_variant_matches_oracle():
    """Each shape of the layer-free kernel the autotuner may pick, forward and adjoint."""
    import torch
    from paper_1804_01390_gb300 import _lib
    N, w = (290, 61), 7
    T = tuple(n + 2 * w for n in N)
    rng = np.random.default_rng(31)
    u0 = gaussian_u0(N, w, 4) + rng.normal(scale=0.2, size=T[::-1])
    g = oracle_grid(N, w)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    want, _ = oracle.rk4(g, y, 13, 0.5)
    for prec in (64, 32):
        s = make_solver(N, w, prec, adjoint=True)
        _, nv = _lib.pml_get_variant(s.ctx)
        assert nv >= 2
        for v in range(nv):
            _lib.pml_set_variant(s.ctx, v)
            s.set_initial(torch.from_numpy(u0))
            s.step(13)
            for f in range(6):
                assert_close(s.read(f).double().cpu().numpy(), want[f], prec, repr((prec, v, f)))
        s.close()


@pytest.mark.parametrize("N,w,sigma", CASES[:4])
def test_layout_tables_bit_exact(N, w, sigma):
    rng = np.random.default_rng(3)
    draws = [rng.random(n + 2 * w) for n in N] if sigma == "random" else None
    s = make_solver(N, w, 64, sigma=sigma, draws=draws)
    g = oracle_grid(N, w, sigma, 2.0, draws)
    for a in range(len(N)):
        phi, psi, inner = s.layout(a)
        ophi, opsi, oin = oracle.layout_axis(g.sigmas[a], w + N[a] // 2)
        assert np.array_equal(phi, ophi)
        assert np.array_equal(psi, opsi)
        assert np.array_equal(inner, oin)
        np.testing.assert_allclose(s.sigma(a), g.sigmas[a], rtol=1e-15, atol=0)
    s.close()


def test_cfg1_full_fp64_and_fp32():
    """Config 1 (128^2 + 16-cell quadratic layer, 1000 steps), both precisions.

    Per-field relative L2 at step 60 (the pulse is crossing the layer, every field is
    large) and at step 200; by step 1000 the pulse has left the box and the remaining
    field is ~1e-10 of the initial one, so the late-time error is measured against the
    initial state's norm (FP64) and as a state-vector relative L2 (FP32)."""
    import torch
    wl = wk.cfg1()
    u0 = wk.initial_field(wl)
    g = oracle_grid(wl.N, wl.w)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    want60, _ = oracle.rk4(g, y, 60, wl.dt)
    want200, _ = oracle.rk4(g, want60, 140, wl.dt, step0=60)
    want, _ = oracle.rk4(g, want200, 800, wl.dt, step0=200)
    n0 = np.linalg.norm(u0)
    for prec in (64, 32):
        s = make_solver(wl.N, wl.w, prec)
        s.set_initial(torch.from_numpy(u0))
        s.step(60)
        got60 = [s.read(f).double().cpu().numpy() for f in range(6)]
        s.step(140)
        got200 = [s.read(f).double().cpu().numpy() for f in range(6)]
        s.step(800)
        got = [s.read(f).double().cpu().numpy() for f in range(6)]
        s.close()
        for f in range(6):
            assert_close(got60[f], want60[f], prec, repr((prec, f,)))
        if prec == 64:
            for f in range(6):
                assert_close(got200[f], want200[f], 64, repr((f,)))
                diff = np.linalg.norm(got[f].reshape(-1) - want[f].reshape(-1))
                assert diff <= TOL[64] * n0, (f, diff / n0)
        else:
            assert_close(np.stack(got200), want200, 32)
            for f in range(6):
                diff = np.linalg.norm(got[f].reshape(-1) - want[f].reshape(-1))
                assert diff <= TOL[32] * n0, (f, diff / n0)


def test_truncation_vs_big_domain_fp64():
    """Sec. 1.1.4 / Fig. Roundtrip: a thick layer (the 64-cell reference mode) agrees with a
    box whose boundary is never reached to machine precision after 1000 steps; thinner
    layers leave residual waves that shrink exponentially with the thickness (the 16-cell
    layer of config 1: ~1e-7, physics shared with the oracle)."""
    import torch
    errs = {}
    for w in (16, 32, 64):
        wl = wk.cfg1(w=w)
        u0 = wk.initial_field(wl)
        s = make_solver(wl.N, wl.w, 64)
        s.set_initial(torch.from_numpy(u0))
        big, offs = wk.reference_box(wl, 1024)
        ub = wk.reference_initial_field(wl, 1024)
        r = make_solver(big.N, 0, 64)
        r.set_initial(torch.from_numpy(ub))
        s.step(1000)
        r.step(1000)
        a = s.read(0).cpu().numpy()[wl.w:wl.w + 128, wl.w:wl.w + 128]
        b = r.read(0).cpu().numpy()[offs[1]:offs[1] + 128, offs[0]:offs[0] + 128]
        ref = torch.from_numpy(np.ascontiguousarray(b))
        nrm = s.norms(ref)
        errs[w] = float(np.abs(a - b).max())
        assert abs(nrm["diff_max"] - errs[w]) <= 1e-15 + 1e-12 * errs[w]
        s.close()
        r.close()
    assert errs[64] <= 1e-12, errs
    assert errs[16] > 100 * errs[32] > 100 * errs[64], errs
    assert 1e-9 < errs[16] < 1e-5, errs


def test_sources_and_receivers_fp64():
    import torch
    N, w = (60, 52), 10
    T = tuple(n + 2 * w for n in N)
    rng = np.random.default_rng(7)
    coords = [(w + 10, w + 12), (w + 30, w + 40), (w + 45, w + 8)]
    amp = rng.uniform(-1, 1, 3)
    f, t0 = 0.1, 15.0
    rec = [(w + 2, w + 3), (w + 20, w + 25), (3, 4), (T[0] - 1, T[1] - 1), (w + 30, w + 40)]
    steps = 60
    for prec in (64, 32):
        s = make_solver(N, w, prec)
        u0 = gaussian_u0(N, w, 11, 1)
        s.set_initial(torch.from_numpy(u0))
        s.set_sources(coords, amp, f, t0)
        tr = s.set_receivers(rec, steps)
        s.step(steps)
        got = s.read(0).double().cpu().numpy()
        gtr = tr.double().cpu().numpy()
        s.close()
        g = oracle_grid(N, w)
        y = g.zeros_state()
        y[0] = u0.reshape(-1)
        src = {"idx": [g.flat(c) for c in coords], "amp": amp, "f_peak": f, "t_delay": t0}
        want, wtr = oracle.rk4(g, y, steps, 0.5, sources=src, receivers=[g.flat(c) for c in rec])
        assert_close(got, want[0], prec)
        assert_close(gtr, wtr, prec)


def test_sources_must_avoid_layer():
    from paper_1804_01390_gb300 import _lib
    s = make_solver((40, 40), 8, 64)
    with pytest.raises(_lib.PMLError) as e:
        s.set_sources([(8, 20)], [1.0], 0.1, 15.0)     # first physical vertex: next to the layer
    assert e.value.status == _lib.PML_EINVAL
    s.set_sources([(9, 20)], [1.0], 0.1, 15.0)
    s.close()


def test_norms_match_oracle():
    import torch
    N, w = (80, 66), 12
    s = make_solver(N, w, 64)
    u0 = gaussian_u0(N, w, 5)
    s.set_initial(torch.from_numpy(u0))
    s.step(37)
    g = oracle_grid(N, w)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    want, _ = oracle.rk4(g, y, 37, 0.5)
    lo = (w, w)
    hi = (w + N[0] - 1, w + N[1] - 1)
    nr = s.norms()
    E = oracle.energy(g, want, lo, hi)
    mx, l2, _ = oracle.norms(g, want[0], None, lo, hi)
    assert abs(nr["energy"] - E) <= 1e-12 * E
    assert abs(nr["max"] - mx) <= 1e-12 * mx
    assert abs(nr["l2"] - l2) <= 1e-12 * l2
    s.close()


def test_energy_without_layer_matches_oracle():
    """sigma = 0: eq:Energy over the whole periodic box only decreases (RK4 multiplies each
    mode's energy by |R(i omega dt)|^2 <= 1) and equals the oracle's after 1000 steps."""
    import torch
    N = (96, 80)
    u0 = gaussian_u0(N, 0, 9)
    s = make_solver(N, 0, 64)
    s.set_initial(torch.from_numpy(u0))
    e = [s.norms()["energy"]]
    for _ in range(10):
        s.step(100)
        e.append(s.norms()["energy"])
    s.close()
    assert all(b <= a * (1 + 1e-14) for a, b in zip(e, e[1:]))
    g = oracle_grid(N, 0)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    want, _ = oracle.rk4(g, y, 1000, 0.5)
    E = oracle.energy(g, want)
    assert abs(e[-1] - E) <= 1e-12 * E


def test_checkpoint_roundtrip_bit_exact():
    import torch
    N, w = (70, 50), 10
    s = make_solver(N, w, 32)
    s.set_initial(torch.from_numpy(gaussian_u0(N, w, 2)))
    s.step(15)
    ck = s.save_state()
    ck_host = s.save_state(torch.empty(s.state_bytes(), dtype=torch.uint8))
    s.step(20)
    a = [s.read(f).clone() for f in range(6)]
    s.load_state(ck)
    assert s.step_count == 15
    s.step(20)
    b = [s.read(f).clone() for f in range(6)]
    s.load_state(ck_host)
    s.step(20)
    c = [s.read(f).clone() for f in range(6)]
    s.close()
    for x, y, z in zip(a, b, c):
        assert torch.equal(x, y) and torch.equal(x, z)


def _patch_oracle(u0, v0, sig, x, y, k, Rp):
    """Oracle value of (U, V) at vertex (x, y) after k steps, from a periodic patch of
    radius Rp >= 4k + 1 around it (the patch wrap never reaches the centre)."""
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


@pytest.mark.parametrize("prec", [32, 64])
def test_full_size_cfg2_sampled(prec):
    """Config 2 size (8192^2 + 32-cell layer) in the benchmark's launch configuration:
    two steps, then vertices sampled over interior, layer, corners and the periodic
    seam, each recomputed by the oracle on a local patch."""
    import torch
    wl = wk.cfg2()
    T = wl.T
    u0 = wk.initial_field(wl)
    rng = np.random.default_rng(12)
    # add structured noise near the seam and in a corner so the layer path is exercised
    u0[:40, :40] += rng.normal(scale=0.2, size=(40, 40))
    u0[-40:, 4000:4040] += rng.normal(scale=0.2, size=(40, 40))
    v0 = np.zeros_like(u0)
    s = make_solver(wl.N, wl.w, prec)
    s.set_initial(torch.from_numpy(u0))
    k = 2
    s.step(k)
    U = s.read(0).double().cpu().numpy()
    V = s.read(1).double().cpu().numpy()
    s.close()
    sig = [oracle.sigma_profile(n, wl.w, oracle.KIND_POWER, 2.0, 2.0) for n in wl.N]
    pts = [(0, 0), (T[0] - 1, T[1] - 1), (5, 17), (33, 33), (32, 4000), (4100, 8255), (8230, 10),
           (4020, 8240), (64, 64), (4000, 4000)]
    pts += [(int(a), int(b)) for a, b in zip(rng.integers(0, T[0], 60), rng.integers(0, T[1], 60))]
    got, want = [], []
    for (x, y) in pts:
        wu, wv = _patch_oracle(u0, v0, sig, x, y, k, 4 * k + 2)
        got += [U[y, x], V[y, x]]
        want += [wu, wv]
    assert_close(got, want, prec, "sampled vertices (U and V)")
