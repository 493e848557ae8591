"""The C-ABI library loads and exports every entry point include/rxr.h
declares; argument errors come back as negative codes without touching a GPU;
without a GPU the library fails loudly (no CPU fallback)."""
import ctypes
import os
import re

import pytest

from paper_2111_11148_gb300 import rxr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rxr.h")


def declared_symbols():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"RXR_API\s+(?:const\s+)?\w+\s*\*?\s*(rxr_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(rxr.LIB_PATH):
        from paper_2111_11148_gb300 import build

        build.build()
    return rxr.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("rxr_create", "rxr_destroy", "rxr_cholqr", "rxr_cholqr_async", "rxr_cholqr_host",
              "rxr_cholqr_batched", "rxr_omega", "rxr_sketch", "rxr_xr_factor", "rxr_precond_gram",
              "rxr_cholesky", "rxr_workspace_bytes", "rxr_status_string"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert sorted(declared_symbols()) == sorted(rxr.exported_symbols())


def test_status_strings(lib):
    for code in range(0, 9):
        assert rxr.status_string(code) != "unknown status"
    assert "invalid" in rxr.status_string(-3)


def test_argument_errors_are_negative_codes(lib):
    # rxr_omega validates before launching anything
    assert lib.rxr_omega(0, 0, 0, 10, None, None) == -2
    assert lib.rxr_omega(0, 8, -1, 10, None, None) == -3
    assert lib.rxr_omega(0, 8, 0, -1, None, None) == -4
    assert lib.rxr_omega(0, 8, 0, 10, None, None) == -5
    assert lib.rxr_omega(0, 8, 0, 0, None, None) == 0
    assert lib.rxr_create(None, 0) == -1
    v = ctypes.c_size_t()
    assert lib.rxr_workspace_bytes(10, 20, 40, 0, ctypes.byref(v)) == -1     # m < n


def test_no_gpu_fails_loudly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.rxr_create(ctypes.byref(h), 0) == rxr.CUDA_ERROR
    with pytest.raises(rxr.RxrError):
        rxr.Handle(0)
