"""Accuracy statement of the FP32 path (max-abs and relative L2 beside each other):

* truncation against a box whose boundary is never reached (the paper's check of the layer,
  Sec. 1.1.4), in FP32 as in FP64: the FP32 layer adds nothing above FP32 rounding;
* the full-length 8192^2 + 32-cell run (5000 steps) in FP32 against the same run in FP64
  (the FP64 path is the one the oracle pins element by element in the parity tests);
* repeat runs at full size are bit-identical (no race between work items).
"""
import numpy as np
import pytest

from paper_1804_01390_gb300 import workloads as wk

from ._helpers import errors, make_solver

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


def _window_run(wl, prec, M=None, steps=1000):
    """U over the physical window after `steps` steps: the layer run of `wl` (M None) or the
    sigma = 0 run of the M^2 box holding the same masked initial data."""
    import torch
    if M is None:
        s = make_solver(wl.N, wl.w, prec)
        s.set_initial(torch.from_numpy(wk.initial_field(wl)))
        lo = (wl.w, wl.w)
    else:
        big, offs = wk.reference_box(wl, M)
        s = make_solver(big.N, 0, prec)
        s.set_initial(torch.from_numpy(wk.reference_initial_field(wl, M)))
        lo = offs
    s.step(steps)
    u = s.read(0).double().cpu().numpy()[lo[1]:lo[1] + wl.N[1], lo[0]:lo[0] + wl.N[0]]
    s.close()
    return u


def test_truncation_vs_big_domain_fp32():
    """Config 1 geometry (128^2, quadratic layer, 1000 steps) with 32- and 64-cell layers
    in FP32 and FP64 against the FP64 run of a 1024^2 box without layer.  In FP64 the
    layer's truncation error falls by orders of magnitude from 32 to 64 cells (Sec. 1.1.4:
    it shrinks exponentially with the thickness); in FP32 both widths leave an error of one
    size, set by FP32 rounding rather than by the layer, and within the FP32 target of
    1e-5 of the initial field.  The FP32 run of the big box itself (no layer) gives the
    rounding floor, reported beside them.  Errors are stated against the initial field (by
    step 1000 the pulse has left the window)."""
    wl64 = wk.cfg1(w=64)
    b64 = _window_run(wl64, 64, M=1024)
    b32 = _window_run(wl64, 32, M=1024)
    u0 = wk.initial_field(wl64)
    peak0 = float(np.abs(u0).max())
    n0 = float(np.linalg.norm(u0))
    floor = float(np.abs(b32 - b64).max())
    report = {"fp32_floor_max_abs": floor / peak0}
    t32, t64 = {}, {}
    for w in (32, 64):
        wl = wk.cfg1(w=w)
        a32 = _window_run(wl, 32)
        a64 = _window_run(wl, 64)
        t64[w] = float(np.abs(a64 - b64).max())
        t32[w] = float(np.abs(a32 - b64).max())
        l2_32 = float(np.linalg.norm(a32 - b64)) / n0
        report[w] = {"fp32_max_abs": t32[w] / peak0, "fp32_rel_l2": l2_32, "fp64_max_abs": t64[w] / peak0}
        assert t32[w] <= 1e-5 * peak0 and l2_32 <= 1e-5, report
    print("FP32 truncation vs the 1024^2 box (relative to the initial peak / norm):", report)
    assert t64[32] > 1e3 * t64[64], report              # FP64: the layer's truncation error
    assert 0.1 <= t32[32] / t32[64] <= 10.0, report      # FP32: rounding, the same at both widths
    assert t32[64] > 1e3 * t64[64], report
    assert floor <= 1e-5 * peak0, report


@pytest.fixture(scope="module")
def cfg2_fp64():
    """U and V of the 8192^2 + 32-cell workload after its 5000 steps in FP64 (host copies)."""
    import torch
    wl = wk.cfg2()
    s = make_solver(wl.N, wl.w, 64)
    s.set_initial(torch.from_numpy(wk.initial_field(wl)))
    s.step(wl.steps)
    out = [s.read(f).cpu().numpy() for f in (0, 1)]
    s.close()
    torch.cuda.empty_cache()
    return out


@pytest.mark.parametrize("two_step", [False, True])
def test_full_length_cfg2_fp32_vs_fp64(cfg2_fp64, two_step):
    """The 8192^2 + 32-cell workload over its full 5000 steps: FP32 against FP64.  RK4 with
    dt = 0.5 h is non-expansive on every mode (|R(i omega dt)| <= 1), so the rounding errors
    of the n steps add at most linearly: the bound is n x 4 x 2^-24 of the field's peak,
    relative L2 alike.  A race or a wrong vertex would show as an error of the order of the
    field itself."""
    import torch
    from paper_1804_01390_gb300 import _lib
    wl = wk.cfg2()
    n = wl.steps
    s = make_solver(wl.N, wl.w, 32)
    _, nv = _lib.pml_get_variant(s.ctx)
    want_tb = 2 if two_step else 1
    for v in range(nv):
        _lib.pml_set_variant(s.ctx, v)
        if _lib.pml_get_time_block(s.ctx) == want_tb:
            break
    assert _lib.pml_get_time_block(s.ctx) == want_tb
    s.set_initial(torch.from_numpy(wk.initial_field(wl)))
    s.step(n)
    got = [s.read(f).cpu().numpy() for f in (0, 1)]
    s.close()
    bound = n * 4.0 * EPS32
    for f in (0, 1):
        r, mx, mr = errors(got[f], cfg2_fp64[f])
        print("field %d after %d steps (%s): FP32 vs FP64 rel-L2 %.3e, max-abs %.3e (%.3e of peak)"
              % (f, n, "two steps per pass" if two_step else "one step per pass", r, mx, mr))
        assert r <= bound and mr <= bound, (f, r, mx, mr, bound)


def test_repeat_runs_bit_identical_full_size():
    """Two runs of 24 steps from the same state, with the one-step and the two-step
    kernels, give bit-identical fields (every vertex is written by exactly one item)."""
    import torch
    from paper_1804_01390_gb300 import _lib
    wl = wk.cfg2()
    u0 = torch.from_numpy(wk.initial_field(wl, dtype=np.float32))
    rng = np.random.default_rng(5)
    v0 = torch.from_numpy(rng.normal(scale=0.1, size=u0.shape).astype(np.float32))
    s = make_solver(wl.N, wl.w, 32)
    _, nv = _lib.pml_get_variant(s.ctx)
    tbs = {}
    for v in range(nv):
        _lib.pml_set_variant(s.ctx, v)
        tbs.setdefault(_lib.pml_get_time_block(s.ctx), v)
    for tb, v in sorted(tbs.items()):
        _lib.pml_set_variant(s.ctx, v)
        runs = []
        for _ in range(2):
            s.set_initial(u0, v0)
            s.step(24)
            runs.append([s.read(f).clone() for f in range(6)])
        for f in range(6):
            assert torch.equal(runs[0][f], runs[1][f]), (tb, v, f)
    s.close()
