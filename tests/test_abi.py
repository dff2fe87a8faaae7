"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/fmm.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1602_02244_gb300 import build
    return ctypes.CDLL(build.build())


def declared():
    src = open(os.path.join(ROOT, "include", "fmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for f in ("fmm_plan_create", "fmm_eval", "fmm_adjoint", "fmm_plan_destroy", "fmm_plan_export"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_status_strings_without_gpu(lib):
    lib.fmm_status_string.restype = ctypes.c_char_p
    assert lib.fmm_status_string(0) == b"FMM_OK"
    assert lib.fmm_status_string(4) == b"FMM_ERR_TIMEOUT"


def test_invalid_arguments_rejected_before_any_cuda_call(lib):
    lib.fmm_plan_create.restype = ctypes.c_int
    lib.fmm_last_error_message.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    # negative n, bad leaf size, bad order, NULL out: all rejected on the host
    assert lib.fmm_plan_create(None, ctypes.c_int64(-1), 8, 4, None, None, ctypes.byref(out)) == 1
    assert lib.fmm_plan_create(None, ctypes.c_int64(10), 0, 4, None, None, ctypes.byref(out)) == 1
    assert lib.fmm_plan_create(None, ctypes.c_int64(10), 8, 21, None, None, ctypes.byref(out)) == 1
    assert lib.fmm_plan_create(None, ctypes.c_int64(10), 8, 4, None, None, None) == 1
    assert b"out" in lib.fmm_last_error_message()
    lib.fmm_eval.restype = ctypes.c_int
    assert lib.fmm_eval(None, None, None, None, None) == 1


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1602_02244_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(binding.FMMError):
        binding.library()
