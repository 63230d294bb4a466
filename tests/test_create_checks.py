"""Argument validation of pml_create, run without a GPU: every rejected call returns before
the library touches a device, with the status the header documents and a message.

The time-step limit is the RK4 stability bound of the undamped operator: RK4 is stable on
the imaginary axis up to |z| = 2 sqrt(2), and the discrete Laplacian's largest frequency is
2 sqrt(d) / h, so dt <= sqrt(2/d) h (dt is never stated in the paper; dt = h/2 is used
throughout).  Damping profiles must be non-negative, finite and zero on the physical edges
(sigma_a(i) = 0 for i < 0 in Sec. 1.1.2; both interface edges here), random draws in [0, 1].
"""

import numpy as np
import pytest

from paper_1804_01390_gb300 import _lib


@pytest.fixture(scope="module")
def L():
    from paper_1804_01390_gb300 import build as b
    b.build()
    return _lib.load()


def _create(ndim=2, n=(32, 24), h=1.0, dt=0.5, w=4, kind=_lib.PML_SIGMA_POWER, smax=2.0, order=2.0, user=None,
            prec=32, workspace=None, workspace_bytes=0, flags=0):
    return _lib.pml_create(ndim, n, h, dt, w, kind, smax, order, user, prec, None, workspace, workspace_bytes, flags)


def _status(**kw):
    with pytest.raises(_lib.PMLError) as e:
        _create(**kw)
    assert _lib.pml_last_error(None)
    return e.value.status


@pytest.mark.parametrize("ndim,n", [(2, (32, 24)), (3, (12, 10, 9))])
def test_time_step_beyond_the_rk4_limit(L, ndim, n):
    for h in (1.0, 0.0125, 3.0):
        limit = np.sqrt(2.0 / ndim) * h
        assert _status(ndim=ndim, n=n, h=h, dt=limit * (1 + 1e-9)) == _lib.PML_EUNSTABLE
        assert _status(ndim=ndim, n=n, h=h, dt=2.0 * h) == _lib.PML_EUNSTABLE


@pytest.mark.parametrize("kw", [dict(h=0.0), dict(h=-1.0), dict(h=float("nan")), dict(dt=0.0),
                                dict(dt=float("inf")), dict(ndim=4, n=(8, 8, 8)), dict(w=-1),
                                dict(n=(0, 24)), dict(n=(2, 24), w=1), dict(prec=16),
                                dict(kind=7), dict(kind=_lib.PML_SIGMA_POWER, order=0.0),
                                dict(smax=-1.0), dict(smax=float("nan"))])
def test_invalid_arguments(L, kw):
    assert _status(**kw) == _lib.PML_EINVAL


def test_workspace_too_small_or_misaligned(L):
    need = _lib.pml_workspace_bytes(2, (32, 24), 4, 32)
    # the pointer is only compared and checked for alignment before the size test fails
    assert _status(workspace=0x10000, workspace_bytes=need - 1) == _lib.PML_ENOMEM
    assert _status(workspace=0x10000 + 64, workspace_bytes=need) == _lib.PML_EINVAL


def _user(arrs):
    keep = [np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
    return keep, [a.ctypes.data for a in keep]


def test_user_and_random_profiles_are_checked(L):
    n, w = (20, 16), 3
    T = [x + 2 * w for x in n]
    base = [np.zeros(t) for t in T]
    for a in range(2):
        base[a][: w - 1] = 1.0          # layer edges 0 .. w-2
        base[a][w + n[a]:] = 1.0        # layer edges w+N .. T-1
    keep, ptr = _user(base)              # a valid profile (only its first axis is used below)
    bad = [b.copy() for b in base]
    bad[1][w + 5] = 0.5                  # damping on a physical edge
    k2, p2 = _user(bad)
    assert _status(n=n, w=w, kind=_lib.PML_SIGMA_USER, user=p2) == _lib.PML_EINVAL
    assert "physical" in _lib.pml_last_error(None)
    for v in (-0.1, float("nan"), float("inf")):
        bad = [b.copy() for b in base]
        bad[0][0] = v
        k3, p3 = _user(bad)
        assert _status(n=n, w=w, kind=_lib.PML_SIGMA_USER, user=p3) == _lib.PML_EINVAL
    draws = [np.full(t, 0.5) for t in T]
    draws[0][2] = 1.5
    k4, p4 = _user(draws)
    assert _status(n=n, w=w, kind=_lib.PML_SIGMA_RANDOM, user=p4) == _lib.PML_EINVAL
    assert _status(n=n, w=w, kind=_lib.PML_SIGMA_RANDOM, user=None) == _lib.PML_EINVAL
    assert _status(n=n, w=w, kind=_lib.PML_SIGMA_USER, user=[ptr[0], None]) == _lib.PML_EINVAL


@pytest.mark.parametrize("ndim", [2, 3])
def test_limit_is_where_the_oracle_starts_to_grow(L, orc, ndim):
    """The same bound seen from the oracle: the checkerboard mode (the discrete Laplacian's
    largest frequency) stays bounded just below sqrt(2/d) h and grows just above it."""
    T, h = (8,) * ndim, 0.7
    g = orc.Grid(T, h, [np.zeros(t) for t in T])
    idx = np.indices(T[::-1]).sum(axis=0)
    y0 = g.zeros_state()
    y0[0] = ((-1.0) ** idx).reshape(-1)
    limit = np.sqrt(2.0 / ndim) * h
    grow = []
    for f in (0.99, 1.01):
        y, _ = orc.rk4(g, y0.copy(), 3000, f * limit)
        grow.append(np.abs(y).max())
    assert grow[0] < 2.0 and grow[1] > 10.0, grow
