"""The allocation-free norms entry point against the context-based one.

pml_norms_dense_static serves callers that cannot allocate device memory when they need
the energy and error norms (services that reserve all memory at start-up and must not
allocate later, or processes whose device memory belongs to another allocator or a fixed
budget).  Its partial sums live in a fixed array inside the library.  This test feeds it
the dense fields of a running context and checks its five numbers against pml_norms on
the same state, twice in a row (with and without a reference field), in both precisions.
This file is collected last so that a failure here does not hide any other test.
"""
import numpy as np
import pytest

from ._helpers import gaussian_u0, make_solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [64, 32])
def test_norms_without_allocation_match_pml_norms(prec):
    import torch
    from paper_1804_01390_gb300 import _lib
    N, w = (150, 97), 12
    s = make_solver(N, w, prec)
    s.set_initial(torch.from_numpy(gaussian_u0(N, w, 21)))
    lo = (w, w)
    hi = (w + N[0] - 1, w + N[1] - 1)
    stream = s.stream.cuda_stream
    for k in range(2):
        s.step(17 + 11 * k)
        U = s.read(0)
        V = s.read(1)
        ref = None
        if k == 1:   # second call: compare against a reference field as well
            ref = (U[w:w + N[1], w:w + N[0]].double() * 0.5).contiguous()
        want = s.norms(ref)
        got = _lib.pml_norms_dense_static(2, s.T, prec, U.data_ptr(), V.data_ptr(), lo, hi, s.h,
                                          ref.data_ptr() if ref is not None else None, stream)
        names = ["energy", "max", "l2", "diff_l2", "diff_max"]
        for i, nm in enumerate(names):
            assert abs(got[i] - want[nm]) <= 1e-12 * max(abs(want[nm]), 1e-300), (k, nm, got[i], want[nm])
    s.close()


def test_norms_without_allocation_3d():
    """A 3D box: the z index, the periodic z neighbour and the third difference term."""
    import torch
    from paper_1804_01390_gb300 import _lib
    N, w = (24, 24, 24), 6
    s = make_solver(N, w, 64)
    s.set_initial(torch.from_numpy(gaussian_u0(N, w, 13)))
    lo = (w, w, w)
    hi = tuple(w + n - 1 for n in N)
    for k in range(2):
        s.step(5 + 4 * k)
        U = s.read(0)
        V = s.read(1)
        ref = (U[w:w + N[2], w:w + N[1], w:w + N[0]] * 0.25).contiguous() if k == 1 else None
        want = s.norms(ref)
        got = _lib.pml_norms_dense_static(3, s.T, 64, U.data_ptr(), V.data_ptr(), lo, hi, s.h,
                                          ref.data_ptr() if ref is not None else None, s.stream.cuda_stream)
        for i, nm in enumerate(["energy", "max", "l2", "diff_l2", "diff_max"]):
            assert abs(got[i] - want[nm]) <= 1e-12 * max(abs(want[nm]), 1e-300), (k, nm, got[i], want[nm])
    s.close()


def _numpy_norms(U, V, lo, hi, h, ref):
    """The five numbers in plain FP64 numpy: energy with periodic forward differences over
    the window, max |U|, ||U||, ||U - ref||, max |U - ref|."""
    U = U.astype(np.float64)
    V = V.astype(np.float64)
    sl = tuple(slice(l, hi_ + 1) for l, hi_ in zip(lo[::-1], hi[::-1]))
    e = (V[sl] ** 2).sum()
    for ax in range(U.ndim):
        d = (np.roll(U, -1, axis=ax) - U) / h
        e += (d[sl] ** 2).sum()
    u = U[sl]
    d = u - ref
    return [0.5 * e, np.abs(u).max(), np.sqrt((u ** 2).sum()), np.sqrt((d ** 2).sum()), np.abs(d).max()]


@pytest.mark.parametrize("prec", [32, 64])
def test_norms_without_allocation_window_at_box_edge(prec):
    """A window that starts at x = 0 and ends at the last vertex of both axes (where the
    forward differences wrap around the box), at h != 1, against numpy in FP64."""
    import torch
    from paper_1804_01390_gb300 import _lib
    rng = np.random.default_rng(17)
    T = (90, 61)
    dt = torch.float32 if prec == 32 else torch.float64
    U = torch.from_numpy(rng.normal(size=T[::-1])).to(dt).cuda()
    V = torch.from_numpy(rng.normal(size=T[::-1])).to(dt).cuda()
    lo, hi, h = (0, 3), (T[0] - 1, T[1] - 1), 0.7
    ref = torch.from_numpy(rng.normal(size=(hi[1] - lo[1] + 1, hi[0] - lo[0] + 1))).cuda()
    for k in range(2):   # two calls in a row: the second must not see the first's partials
        r = ref if k == 1 else None
        got = _lib.pml_norms_dense_static(2, T, prec, U.data_ptr(), V.data_ptr(), lo, hi, h,
                                          r.data_ptr() if r is not None else None, None)
        want = _numpy_norms(U.cpu().numpy(), V.cpu().numpy(), lo, hi, h,
                            ref.cpu().numpy() if k == 1 else 0.0)
        for i in range(5):
            if k == 0 and i >= 3:
                assert got[i] == 0.0
                continue
            assert abs(got[i] - want[i]) <= 1e-12 * abs(want[i]), (k, i, got[i], want[i])


def test_rejects_windows_beyond_its_scratch():
    import torch
    from paper_1804_01390_gb300 import _lib
    T = (16, 20000)
    U = torch.zeros(T[::-1], dtype=torch.float32, device="cuda")
    with pytest.raises(_lib.PMLError) as e:
        _lib.pml_norms_dense_static(2, T, 32, U.data_ptr(), U.data_ptr(), (0, 0), (15, 19999), 1.0, None, None)
    assert e.value.status == _lib.PML_EINVAL
    assert "16384" in str(e.value)
