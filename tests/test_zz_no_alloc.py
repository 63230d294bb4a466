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


def test_rejects_windows_beyond_its_scratch():
    import torch
    from paper_1804_01390_gb300 import _lib
    T = (16, 20000)
    U = torch.zeros(T[::-1], dtype=torch.float32, device="cuda")
    with pytest.raises(_lib.PMLError) as e:
        _lib.pml_norms_dense_static(2, T, 32, U.data_ptr(), U.data_ptr(), (0, 0), (15, 19999), 1.0, None, None)
    assert e.value.status == _lib.PML_EINVAL
    assert "16384" in str(e.value)
