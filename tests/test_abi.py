"""The C-ABI library loads on a machine without a GPU and exports every symbol that
include/pml.h declares (no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "pml.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pml_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1804_01390_gb300 import build as b
    return ctypes.CDLL(b.build())


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("pml_create", "pml_set_initial", "pml_step", "pml_read_field", "pml_adjoint_step",
                 "pml_norms", "pml_set_sources", "pml_set_receivers", "pml_save_state",
                 "pml_load_state", "pml_destroy", "pml_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1804_01390_gb300 import _lib
    assert sorted(_lib.EXPORTED) == _declared()


def test_host_only_calls_without_gpu(lib):
    """pml_workspace_bytes and pml_status_string need no device."""
    from paper_1804_01390_gb300 import _lib
    _lib.load()
    b32 = _lib.pml_workspace_bytes(2, (128, 128), 16, 32)
    b64 = _lib.pml_workspace_bytes(2, (128, 128), 16, 64)
    assert b64 > b32 > 0
    with pytest.raises(_lib.PMLError) as e:
        _lib.pml_workspace_bytes(4, (1, 1), 1, 32)
    assert e.value.status == _lib.PML_EINVAL
    with pytest.raises(_lib.PMLError):
        _lib.pml_workspace_bytes(2, (2, 2), 1, 32)       # n + 2w < 8
    assert _lib.pml_status_string(_lib.PML_EUNSTABLE).startswith("time step")


def test_batch_argument_checks_without_gpu(lib):
    """pml_batch_* reject empty and NULL arguments before touching a device."""
    import ctypes
    from paper_1804_01390_gb300 import _lib
    L = _lib.load()
    out = ctypes.c_void_p(0)
    assert L.pml_batch_create(0, None, ctypes.byref(out)) == _lib.PML_EINVAL
    assert "count >= 1" in _lib.pml_last_error(None)
    arr = (ctypes.c_void_p * 2)(None, None)
    assert L.pml_batch_create(2, arr, ctypes.byref(out)) == _lib.PML_EINVAL
    assert L.pml_batch_step(None, 1) == _lib.PML_EINVAL
    assert L.pml_batch_set_variant(None, 0) == _lib.PML_EINVAL
    assert L.pml_batch_info(None, None) == _lib.PML_EINVAL
    L.pml_batch_destroy(None)


def test_variant_and_time_block_queries_reject_null_without_gpu(lib):
    """The variant and temporal-block queries check their arguments before any device
    work; the two-step scratch state enlarges the 2D FP32 workspace only."""
    import ctypes
    from paper_1804_01390_gb300 import _lib
    L = _lib.load()
    d = ctypes.c_int(0)
    assert L.pml_get_time_block(None, ctypes.byref(d)) == _lib.PML_EINVAL
    assert L.pml_batch_get_time_block(None, ctypes.byref(d)) == _lib.PML_EINVAL
    assert L.pml_get_variant(None, None, None) == _lib.PML_EINVAL
    assert L.pml_set_variant(None, 0) == _lib.PML_EINVAL
    # 2D FP32 holds a third state (the two-step blocks' first-step values): 3 states x 6
    # fields x 4 B per vertex against FP64's 2 x 6 x 8 B, a ratio near 4/3 (2 without it)
    b32 = _lib.pml_workspace_bytes(2, (2000, 2000), 16, 32)
    b64 = _lib.pml_workspace_bytes(2, (2000, 2000), 16, 64)
    field32 = (2032 + 8 + 31) // 32 * 32 * (2032 + 8) * 4
    assert b32 >= 3 * 6 * field32
    assert 1.25 < b64 / b32 < 1.45


def test_no_cpu_fallback(tmp_path):
    """The product path has no CPU fallback: a missing library is an error on first use, and
    a solver refuses any device but CUDA (the oracle is never called in its place)."""
    import torch
    from paper_1804_01390_gb300 import _lib
    from paper_1804_01390_gb300.solver import PMLSolver
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            _lib.load(str(tmp_path / "libpml.so"))
    finally:
        _lib._lib = saved
    with pytest.raises(ValueError, match="CUDA"):
        PMLSolver((16, 16), 4, precision=64, device=torch.device("cpu"))
    # no module of the package imports the oracle
    import re
    pkg = os.path.join(ROOT, "paper_1804_01390_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
