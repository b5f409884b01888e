"""ctypes loader for libaemrjsmc.so.  Fails loudly when the library is missing:
there is no CPU fallback anywhere in this package."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_int = ctypes.c_int
c_double = ctypes.c_double
c_void_p = ctypes.c_void_p


class SystemDesc(ctypes.Structure):
    _fields_ = [
        ("loop_radius", c_double),
        ("height", c_double),
        ("current", c_double),
        ("n_freq", c_int),
        ("f_min_hz", c_double),
        ("f_max_hz", c_double),
        ("n_gates", c_int),
        ("gate_times", ctypes.POINTER(c_double)),
        ("n_hankel", c_int),
        ("cc_form", c_int),
    ]


class Models(ctypes.Structure):
    """Layout shared by aem_models_f32 and aem_models_f64 (pointers only)."""
    _fields_ = [
        ("n_models", c_int),
        ("lmax", c_int),
        ("nlayers", c_void_p),
        ("logsig", c_void_p),
        ("logh", c_void_p),
        ("m", c_void_p),
        ("logtau", c_void_p),
        ("c", c_void_p),
    ]


# Every symbol include/aem_rjsmc.h declares, with its ctypes signature.
SIGNATURES = {
    "aem_last_error": ([], ctypes.c_char_p),
    "aem_system_create": ([ctypes.POINTER(SystemDesc), ctypes.POINTER(c_void_p)], c_int),
    "aem_system_destroy": ([c_void_p], c_int),
    "aem_system_tables": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p], c_int),
    "aem_forward_f32": ([c_void_p, ctypes.POINTER(Models), c_void_p, c_void_p, c_void_p], c_int),
    "aem_forward_f64": ([c_void_p, ctypes.POINTER(Models), c_void_p, c_void_p, c_void_p], c_int),
    "aem_loglik_f32": ([c_void_p, ctypes.POINTER(Models), c_void_p, c_void_p, c_double, c_void_p, c_void_p,
                        c_void_p], c_int),
    "aem_loglik_f64": ([c_void_p, ctypes.POINTER(Models), c_void_p, c_void_p, c_double, c_void_p, c_void_p,
                        c_void_p], c_int),
    "aem_probe_peaks": ([c_void_p, c_void_p, c_void_p, c_void_p], c_int),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the library (building it first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libaemrjsmc.so not found at {path}; run paper_2109_00661_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


class AEMError(RuntimeError):
    pass


def check(rc: int, what: str):
    if rc != 0:
        msg = load().aem_last_error()
        raise AEMError(f"{what} failed ({rc}): {msg.decode() if msg else ''}")
