"""Shared helpers of the GPU parity tests: run the same seeded problem through the
CUDA library (via the C ABI) and through the CPU oracle, and compare."""
import numpy as np

import oracle
from paper_1804_01390_gb300 import workloads as wk

KIND = {"quadratic": oracle.KIND_POWER, "constant": oracle.KIND_CONSTANT,
        "random": oracle.KIND_RANDOM}

# Tolerances: FP64 mode 1e-12 relative L2, FP32 mode 1e-5 relative L2.
TOL = {64: 1e-12, 32: 1e-5}


# Elementwise bound beside the relative L2 one: max |got - want| <= MAXABS_TOL * max |want|.
# The largest elementwise error, measured against the field's peak, may exceed the relative
# L2 error by up to the ratio of the field's peak to its RMS over the error's support, so the
# bound is ten times the L2 tolerance; a wrong or raced vertex (an error of the order of the
# field itself) fails it whatever the size of the box.
MAXABS_TOL = {64: 1e-11, 32: 1e-4}


def errors(got, want):
    """(relative L2 error, max-abs error, max-abs error relative to max |want|)."""
    got = np.asarray(got, dtype=np.float64).reshape(-1)
    want = np.asarray(want, dtype=np.float64).reshape(-1)
    d = np.abs(got - want)
    mx = float(d.max()) if d.size else 0.0
    peak = float(np.abs(want).max()) if want.size else 0.0
    return rel_l2(got, want), mx, (mx / peak if peak > 0 else mx)


def assert_close(got, want, prec, what="", tol=None, tol_max=None):
    """Assert rel-L2 <= tol (TOL[prec]) and max-abs <= tol_max (MAXABS_TOL[prec]) x peak;
    the message states both errors."""
    tol = TOL[prec] if tol is None else tol
    tol_max = MAXABS_TOL[prec] if tol_max is None else tol_max
    r, mx, mr = errors(got, want)
    msg = "%s: rel-L2 %.3e (tol %.0e), max-abs %.3e = %.3e of peak (tol %.0e)" % (what, r, tol, mx, mr, tol_max)
    assert r <= tol and mr <= tol_max, msg
    return r, mx


def rel_l2(got, want):
    got = np.asarray(got, dtype=np.float64).reshape(-1)
    want = np.asarray(want, dtype=np.float64).reshape(-1)
    den = np.linalg.norm(want)
    if den == 0.0:
        return float(np.linalg.norm(got))
    return float(np.linalg.norm(got - want) / den)


def oracle_grid(N, w, sigma="quadratic", sigma_max=2.0, draws=None, h=1.0):
    sigs = []
    for a, n in enumerate(N):
        d = None if draws is None else draws[a]
        sigs.append(oracle.sigma_profile(n, w, KIND[sigma], sigma_max, 2.0, draws=d))
    return oracle.Grid(tuple(n + 2 * w for n in N), h, sigs)


def make_solver(N, w, precision, sigma="quadratic", sigma_max=2.0, draws=None, dt=0.5, h=1.0,
                adjoint=False):
    import torch
    from paper_1804_01390_gb300.solver import PMLSolver
    return PMLSolver(N, w, h=h, dt=dt, sigma=sigma, sigma_max=sigma_max, draws=draws,
                     precision=precision, device=torch.device("cuda:0"), adjoint=adjoint)


def gaussian_u0(N, w, seed, ngauss=3):
    rng = np.random.default_rng(seed)
    gs = []
    for _ in range(ngauss):
        s = rng.uniform(2.0, 5.0)
        c = tuple(w + rng.uniform(0.1 * n, 0.9 * n) for n in N)
        gs.append(wk.Gaussian(c, s, rng.uniform(-1, 1)))
    T = tuple(n + 2 * w for n in N)
    lo = tuple(w for _ in N)
    hi = tuple(w + n - 1 for n in N)
    return wk.gaussian_field(T, gs, (lo, hi))


def random_state(grid, rng):
    """Random U, V and random Phi/Psi on their supports (zero elsewhere)."""
    y = rng.normal(size=(grid.nfields, grid.n))
    nd = grid.ndim
    idx = np.indices(grid.T[::-1])
    for a in range(nd):
        c = idx[nd - 1 - a].reshape(-1)
        s = grid.sigmas[a]
        y[2 + 2 * a, s[c] == 0] = 0.0
        y[3 + 2 * a, np.roll(s, 1)[c] == 0] = 0.0
    return y
