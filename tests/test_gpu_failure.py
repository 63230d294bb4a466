"""Failure detection on the GPU without faulting it: a bounded device wait that runs out
reports PML_ETIMEOUT and leaves the context usable, and the periodic finiteness scan turns
a non-finite state into PML_ENONFINITE.

The waits are made to run out by a wait limit below a microsecond, under which every
bounded wait gives up at once; the kernel then lets its copies in flight (the one it gave
up on included) land before it ends, so nothing is left writing to shared memory."""
import numpy as np
import pytest

import oracle

from ._helpers import TOL, assert_close, gaussian_u0, make_solver, oracle_grid

pytestmark = pytest.mark.gpu


def _oracle_run(N, w, u0, steps):
    g = oracle_grid(N, w)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    want, _ = oracle.rk4(g, y, steps, 0.5)
    return want


@pytest.mark.parametrize("N,w,prec,two_step", [((70, 52), 8, 32, False), ((70, 52), 8, 32, True),
                                               ((44, 40), 6, 64, False), ((24, 20, 22), 5, 32, False)])
def test_wait_limit_runs_out_then_context_recovers(N, w, prec, two_step):
    import torch
    from paper_1804_01390_gb300 import _lib
    u0 = gaussian_u0(N, w, 3)
    s = make_solver(N, w, prec)
    if two_step:   # the two-step interior kernel and both layer passes
        _, nv = _lib.pml_get_variant(s.ctx)
        for v in range(nv):
            _lib.pml_set_variant(s.ctx, v)
            if _lib.pml_get_time_block(s.ctx) == 2:
                break
        assert _lib.pml_get_time_block(s.ctx) == 2
    s.set_initial(torch.from_numpy(u0))
    s.set_wait_limit(1)
    s.step(4)
    with pytest.raises(_lib.PMLError) as e:
        s.sync()
    assert e.value.status == _lib.PML_ETIMEOUT
    assert "wait gave up" in str(e.value)
    with pytest.raises(_lib.PMLError):   # sticky until the state is replaced
        s.sync()
    # the same context: default limit, a new state, a clean run that matches the oracle
    s.set_wait_limit(0)
    s.set_initial(torch.from_numpy(u0))
    s.step(9)
    s.sync()
    want = _oracle_run(N, w, u0, 9)
    for f in range(2 + 2 * len(N)):
        assert_close(s.read(f).double().cpu().numpy(), want[f], prec, "field %d" % f)
    s.close()
    # and a fresh context after destroying the one that timed out
    r = make_solver(N, w, prec)
    r.set_initial(torch.from_numpy(u0))
    r.step(9)
    r.sync()
    assert_close(r.read(0).double().cpu().numpy(), want[0], prec, "U, fresh context")
    r.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_nonfinite_state_is_reported(prec):
    import torch
    from paper_1804_01390_gb300 import _lib
    N, w = (60, 48), 8
    T = tuple(n + 2 * w for n in N)
    u0 = gaussian_u0(N, w, 5)
    bad = u0.copy()
    bad[T[1] // 2, T[0] // 3] = np.nan
    s = make_solver(N, w, prec)
    s.set_check_interval(5)
    s.set_initial(torch.from_numpy(bad))
    s.step(4)                      # no multiple of 5 crossed yet: no scan
    s.sync()
    s.step(1)                      # step 5: scan
    with pytest.raises(_lib.PMLError) as e:
        s.sync()
    assert e.value.status == _lib.PML_ENONFINITE
    assert "after step 5" in str(e.value)
    # an infinite velocity is found too (a scan at step 10 after 10 single steps)
    v0 = np.zeros_like(u0)
    v0[w + 3, w + 4] = np.inf
    s.set_initial(torch.from_numpy(u0), torch.from_numpy(v0))
    s.sync()                       # the new state cleared the error word
    s.step(10)
    with pytest.raises(_lib.PMLError) as e:
        s.sync()
    assert e.value.status == _lib.PML_ENONFINITE
    # scan off: the NaN spreads silently
    s.set_check_interval(0)
    s.set_initial(torch.from_numpy(bad))
    s.step(10)
    s.sync()
    assert np.isnan(s.read(0).cpu().numpy()).any()
    # a finite state passes every scan and still matches the oracle
    s.set_check_interval(1)
    s.set_initial(torch.from_numpy(u0))
    s.step(7)
    s.sync()
    assert_close(s.read(0).double().cpu().numpy(), _oracle_run(N, w, u0, 7)[0], prec, "U")
    with pytest.raises(_lib.PMLError) as e:
        s.set_check_interval(-1)
    assert e.value.status == _lib.PML_EINVAL
    s.close()


def test_nonfinite_adjoint_state_is_reported():
    import torch
    from paper_1804_01390_gb300 import _lib
    N, w = (40, 36), 6
    s = make_solver(N, w, 32, adjoint=True)
    s.set_check_interval(3)
    s.set_initial(torch.from_numpy(gaussian_u0(N, w, 8)))
    s.step(6)
    rec = [(w + 4, w + 5)]
    s.set_receivers(rec, 6)
    s.adjoint_reset()
    res = torch.full((3, 1), float("nan"))
    s.adjoint_step(3, res, want_grad_u=False)
    with pytest.raises(_lib.PMLError) as e:
        s.sync()
    assert e.value.status == _lib.PML_ENONFINITE
    s.close()
