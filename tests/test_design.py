"""Layer design calls (pml_residual_factor, pml_design_width): host logic of the library,
no device work.

The residual factor is pinned by the oracle: a narrow-band 1D wave packet makes one
round of the periodic box, crossing every layer edge once (Sec. 1.1.4's residual wave);
its amplitude relative to the same run without a layer must match the product of the
one-edge decay rates at the packet's wave number (within the few percent that the
packet's bandwidth and dispersion allow).  The bounds of Thm 1.1 (|rho| < 1 and the
reflected-wave ratio < 1) and the width search are checked as properties.
"""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def lib():
    from paper_1804_01390_gb300 import _lib
    _lib.load()
    return _lib


def _packet_ratio(N, w, kind, smax, kh, env):
    T = N + 2 * w
    sig = oracle.sigma_profile(N, w, kind, smax, 2.0)
    j = np.arange(T)
    x0 = w + 0.3 * N
    G = np.exp(-0.5 * ((j - x0) / env) ** 2)
    wh = 2.0 * np.sin(kh / 2.0)                     # 1D discrete dispersion relation
    U = G * np.cos(kh * (j - x0))
    V = wh * G * np.sin(kh * (j - x0))              # right-travelling
    steps = int(round(T / np.cos(kh / 2.0) / 0.5))  # one round at the group velocity
    amp = []
    for s_ in (sig, np.zeros(T)):
        g = oracle.Grid((T,), 1.0, [s_])
        y = g.zeros_state()
        y[0] = U
        y[1] = V
        yn, _ = oracle.rk4(g, y, steps, 0.5)
        amp.append(np.abs(yn[0][w:w + N]).max())
    return amp[0] / amp[1], sig[sig != 0.0], wh


@pytest.mark.parametrize("kind,smax,kh", [(oracle.KIND_CONSTANT, 0.05, 0.3), (oracle.KIND_CONSTANT, 0.05, 0.6),
                                          (oracle.KIND_POWER, 0.2, 0.6)])
def test_residual_factor_matches_packet_through_layer(lib, kind, smax, kh):
    measured, sig, wh = _packet_ratio(300, 12, kind, smax, kh, 25.0)
    pred = lib.pml_residual_factor(sig, kh, wh)
    assert 0.05 < measured < 0.9
    assert abs(measured - pred) <= 0.03 * pred, (measured, pred)


def test_decay_bounds_of_the_theorem(lib):
    rng = np.random.default_rng(3)
    for _ in range(200):
        s = rng.uniform(1e-3, 4.0)
        wh = rng.uniform(1e-3, 2.0)
        kh = rng.uniform(1e-3, np.pi - 1e-3)
        one = lib.pml_residual_factor([s], kh, wh)   # travelling waves: real k, Re(k) in (0, pi/h)
        ratio = lib.pml_residual_factor([s], kh, wh, backed=True)
        assert one < 1.0 and ratio < 1.0
    assert lib.pml_residual_factor([0.0, 0.0], 0.5, 0.49) == pytest.approx(1.0, abs=1e-15)


def test_design_width_is_the_smallest_that_meets_the_target(lib):
    from paper_1804_01390_gb300 import _lib
    for kind, order in ((_lib.PML_SIGMA_CONSTANT, 2.0), (_lib.PML_SIGMA_POWER, 2.0)):
        w, worst = lib.pml_design_width(kind, 1.0, order, 0.5, 1.0, 1e-12)
        assert w > 1 and worst <= 1e-12
        w2, worst2 = lib.pml_design_width(kind, 1.0, order, 0.5, 1.0, 1e-12, w_max=w - 1)
        assert w2 == -1 and worst2 > 1e-12
        # a backed layer is crossed twice: it needs about half the width
        wb, _ = lib.pml_design_width(kind, 1.0, order, 0.5, 1.0, 1e-12, backed=True)
        assert wb < w
    with pytest.raises(_lib.PMLError):
        lib.pml_design_width(_lib.PML_SIGMA_RANDOM, 1.0, 2.0, 0.5, 1.0, 1e-12)
