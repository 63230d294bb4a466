"""The paper's stress experiments on the GPU (Sec. 1.1.4 random damping with white noise,
Sec. 1.1.5 long-time energy), through the user-sigma path of the C ABI.

* Random sigma_a[e] ~ U[0, 2/h) on every layer edge (zero on the physical edges) and
  Gaussian white noise of variance 1/4 in a disk: the PML box must reproduce a large
  sigma = 0 box on the physical window to machine precision (the discrete layer does not
  reflect, and what crosses it is damped away before it can return).
* Long runs with constant sigma = 2/h and with random sigma: the FP64 energy of the
  physical window (eq:Energy) stays below its initial value and decays by more than eight
  orders of magnitude; the state at an intermediate step matches the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1804_01390_gb300 import workloads as wk

from ._helpers import TOL

pytestmark = pytest.mark.gpu


def _random_sigma(n, w, seed, smax=2.0):
    """sigma_max * u_e on the layer edges, zero on the physical edges w-1 .. w+n-1."""
    T = n + 2 * w
    u = np.random.default_rng(seed).random(T)
    e = np.arange(T)
    layer = (e <= w - 2) | (e >= w + n)
    return np.where(layer, smax * u, 0.0)


def _const_sigma(n, w, smax=2.0):
    T = n + 2 * w
    e = np.arange(T)
    return np.where((e <= w - 2) | (e >= w + n), smax, 0.0)


def _solver(N, w, sigmas, prec):
    import torch
    from paper_1804_01390_gb300.solver import PMLSolver
    return PMLSolver(N, w, sigma="user", user_sigma=sigmas, precision=prec, device=torch.device("cuda:0"))


def _noise(N, w, centre, radius, seed):
    T = tuple(n + 2 * w for n in N)
    lo = tuple(w for _ in N)
    hi = tuple(w + n - 1 for n in N)
    return wk.white_noise_disk(T, centre, radius, 0.25, seed, window=(lo, hi))


def test_random_sigma_white_noise_matches_large_box():
    """E2: 96^2 window, 32-cell random layer, noise disk 4 cells from one interface, 60
    steps (30 time units: nothing that entered the layer can cross the 64 layer cells to
    the far side and come back); compared on the window with a 256^2 box without layer
    (its edges are never reached)."""
    import torch
    N, w, steps = (96, 96), 32, 60
    sig = [_random_sigma(N[0], w, 71), _random_sigma(N[1], w, 72)]
    u0 = _noise(N, w, (w + 14.0, w + 48.0), 10.0, seed=73)
    s = _solver(N, w, sig, 64)
    s.set_initial(torch.from_numpy(u0))
    s.step(steps)
    U = s.read(0).double().cpu().numpy()[w:w + N[1], w:w + N[0]]
    s.close()
    B = 256
    off = (B - N[0]) // 2
    big = np.zeros((B, B))
    big[off:off + N[1], off:off + N[0]] = u0[w:w + N[1], w:w + N[0]]
    g = oracle.Grid((B, B), 1.0, [np.zeros(B), np.zeros(B)])
    y = g.zeros_state()
    y[0] = big.reshape(-1)
    out, _ = oracle.rk4(g, y, steps, 0.5, openmp=True)
    ref = out[0].reshape(B, B)[off:off + N[1], off:off + N[0]]
    scale = np.abs(u0).max()
    assert np.abs(ref).max() > 1e-2 * scale
    assert np.abs(U - ref).max() <= 1e-13 * scale, np.abs(U - ref).max() / scale


@pytest.mark.parametrize("kind", ["constant", "random"])
def test_long_run_energy_decays(kind):
    """E4: 64^2 window, 20-cell layer, noise disk in the middle, 20000 FP64 steps."""
    import torch
    N, w = (64, 64), 20
    if kind == "constant":
        sig = [_const_sigma(N[0], w), _const_sigma(N[1], w)]
    else:
        sig = [_random_sigma(N[0], w, 81), _random_sigma(N[1], w, 82)]
    u0 = _noise(N, w, (w + 32.0, w + 32.0), 12.0, seed=83)
    s = _solver(N, w, sig, 64)
    s.set_initial(torch.from_numpy(u0))
    e0 = s.norms()["energy"]
    # parity with the oracle after 2000 steps
    s.step(2000)
    g = oracle.Grid(tuple(n + 2 * w for n in N), 1.0, sig)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    want, _ = oracle.rk4(g, y, 2000, 0.5, openmp=True)
    got = np.concatenate([s.read(f).double().cpu().numpy().reshape(-1) for f in range(6)])
    ref_norm = np.linalg.norm(u0)
    err = np.linalg.norm(got - want.reshape(-1)) / ref_norm
    assert err <= TOL[64], err
    e_or = oracle.energy(g, want, [w, w], [w + N[0] - 1, w + N[1] - 1])
    energies = [s.norms()["energy"]]
    assert abs(energies[0] - e_or) <= 1e-12 * e0
    for _ in range(9):
        s.step(2000)
        energies.append(s.norms()["energy"])
    s.close()
    assert np.all(np.isfinite(energies))
    assert max(energies) <= e0, (max(energies), e0)
    assert energies[-1] <= 1e-8 * e0, energies[-1] / e0
