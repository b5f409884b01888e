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


class SMCDesc(ctypes.Structure):
    _fields_ = [
        ("n_particles", c_int),
        ("n_soundings", c_int),
        ("kappa_max", c_int),
        ("lambda_max", c_int),
        ("zmax", c_double),
        ("alpha", c_double),
        ("c_mut", c_double),
        ("r_max", c_int),
        ("step_phi", c_double),
        ("step_m", c_double),
        ("step_tau", c_double),
        ("step_c", c_double),
        ("step_z", c_double),
        ("phi_lo", c_double),
        ("phi_hi", c_double),
        ("tau_log_prior", c_int),
        ("logtau_lo", c_double),
        ("logtau_hi", c_double),
        ("seed", ctypes.c_ulonglong),
        ("bisect_iters", c_int),
        ("n_langevin", c_int),
        ("langevin_h", c_double),
        ("langevin_adapt", c_int),
        ("adaptive", c_int),
        ("pca_target", c_double),
        ("pca_bisect_iters", c_int),
        ("pca_ridge", c_double),
        ("recycle_stages", c_int),
        ("zca", c_double),
        ("precision", c_int),
    ]


class ParticlesHost(ctypes.Structure):
    _fields_ = [(n, c_void_p) for n in ("kappa", "lam", "phib", "tau", "c", "zc", "phic", "zm", "mv", "ll", "move",
                                          "valid")]


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
    "aem_autotune_forward": ([c_void_p, ctypes.POINTER(Models), c_int, c_void_p, c_void_p, c_void_p], c_int),
    "aem_forward_shape": ([c_void_p, c_int, c_int], c_int),
    "aem_system_set_depth_cutoff": ([c_void_p, ctypes.c_double], c_int),
    "aem_forward_f32_count": ([c_void_p, ctypes.POINTER(Models), c_void_p, c_void_p, c_void_p, c_void_p], c_int),
    "aem_gates_from_spectrum": ([c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p, c_double, c_void_p, c_void_p,
                                 c_void_p], c_int),
    "aem_loglik_f32_tc": ([c_void_p, ctypes.POINTER(Models), c_void_p, c_void_p, c_double, c_int, c_void_p, c_void_p,
                           c_void_p, c_void_p], c_int),
    "aem_system_status": ([c_void_p, c_void_p], c_int),
    "aem_debug_bounded_wait": ([c_void_p, ctypes.c_uint, c_int], c_int),
    "aem_loglik_grad_f32": ([c_void_p, ctypes.POINTER(Models), c_void_p, c_void_p, c_double, c_void_p, c_void_p,
                             c_void_p], c_int),
    "smc_desc_defaults": ([ctypes.POINTER(SMCDesc)], c_int),
    "smc_create": ([c_void_p, ctypes.POINTER(SMCDesc), c_void_p, c_void_p, c_double, c_void_p,
                    ctypes.POINTER(c_void_p)], c_int),
    "smc_destroy": ([c_void_p], c_int),
    "smc_init": ([c_void_p], c_int),
    "smc_reweight": ([c_void_p, c_void_p], c_int),
    "smc_resample": ([c_void_p], c_int),
    "smc_mutate": ([c_void_p, c_int], c_int),
    "smc_propose": ([c_void_p, c_int, c_int], c_int),
    "smc_loglik_current": ([c_void_p], c_int),
    "smc_grad_current": ([c_void_p, c_void_p], c_int),
    "smc_langevin_propose": ([c_void_p, c_int, c_int], c_int),
    "smc_langevin": ([c_void_p, c_int], c_int),
    "smc_ppd": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p], c_int),
    "smc_adapt": ([c_void_p], c_int),
    "smc_get_log_factors": ([c_void_p, c_void_p], c_int),
    "smc_run_graph": ([c_void_p, c_int, c_int, c_void_p], c_int),
    "smc_get_adaptation": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p], c_int),
    "smc_checkpoint": ([c_void_p, c_void_p, ctypes.POINTER(ctypes.c_size_t)], c_int),
    "smc_restore": ([c_void_p, c_void_p, ctypes.c_size_t], c_int),
    "smc_langevin_stats": ([c_void_p, c_void_p, c_void_p, c_void_p], c_int),
    "smc_run": ([c_void_p, c_int, c_int, c_void_p], c_int),
    "smc_model_odds": ([c_void_p, c_void_p, c_void_p, c_void_p], c_int),
    "smc_status": ([c_void_p, c_void_p, c_void_p], c_int),
    "smc_stats": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p], c_int),
    "smc_get_particles": ([c_void_p, c_int, ctypes.POINTER(ParticlesHost)], c_int),
    "smc_set_particles": ([c_void_p, ctypes.POINTER(ParticlesHost), c_void_p, c_void_p, c_int], c_int),
    "aem_smc_workspace_bytes": ([c_int, c_int], ctypes.c_size_t),
    "aem_reweight": ([c_void_p, c_void_p, c_int, c_int, c_double, c_double, c_int, c_void_p, c_void_p, c_void_p,
                      c_void_p, c_void_p, ctypes.c_size_t, c_void_p], c_int),
    "aem_resample_systematic": ([c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, ctypes.c_size_t,
                                 c_void_p], c_int),
    "aem_philox4x32": ([c_void_p, ctypes.c_uint, ctypes.c_uint, c_void_p, c_int, c_void_p], c_int),
    "aem_resample_systematic_noalloc": ([c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p], c_int),
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
        err = AEMError(f"{what} failed ({rc}): {msg.decode() if msg else ''}")
        err.code = rc
        raise err
