"""The C-ABI library builds, loads and exports every symbol the public header
declares (CPU only: no compute call is made)."""
import ctypes
import re
import os

import pytest

from paper_2109_00661_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "aem_rjsmc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(aem_\w+|smc_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    try:
        build.nvcc_path()
    except RuntimeError:
        pytest.skip("nvcc not available")
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_entry_points():
    names = header_functions()
    assert "aem_forward_f32" in names and "aem_loglik_f32" in names and "aem_system_create" in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_every_declared_symbol():
    missing = [n for n in header_functions() if n not in _lib.SIGNATURES]
    assert not missing, f"binding lacks: {missing}"


def test_last_error_is_callable_without_gpu(lib):
    lib.aem_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.aem_last_error(), bytes)


def test_system_create_rejects_bad_descriptor_without_gpu(lib):
    # argument validation happens before any CUDA call
    desc = _lib.SystemDesc(13.0, -1.0, 1.0, 40, 1.0, 1e7, 0, None, 120, 0)
    h = ctypes.c_void_p()
    lib.aem_system_create.argtypes = [ctypes.POINTER(_lib.SystemDesc), ctypes.POINTER(ctypes.c_void_p)]
    assert lib.aem_system_create(ctypes.byref(desc), ctypes.byref(h)) == -1
    lib.aem_last_error.restype = ctypes.c_char_p
    assert b"height" in lib.aem_last_error()
