"""GB300-native hot path of RJSMC for airborne-EM IP detectability
(Davies et al., arXiv 2109.00661).

Thin Python binding over the C ABI in ``include/aem_rjsmc.h``: argument
marshalling only.  Every step of the forward model, likelihood and SMC stage
runs in the CUDA kernels of ``libaemrjsmc.so``; PyTorch provides device memory
and streams.  Calls fail loudly if the library or a CUDA device is missing.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import AEMError, check

__all__ = ["System", "forward_f32", "forward_f64", "spectrum_f32", "loglik_f32", "loglik_f64", "loglik_f32_tc",
           "gates_from_spectrum", "loglik_grad_f32", "loglik", "system_status", "debug_bounded_wait", "probe_peaks",
           "AEMError",
           "CC_PAPER", "CC_PELTON", "GATES_FP32", "GATES_TF32_SPLIT", "GATES_BF16_SPLIT"]

CC_PAPER = 0
CC_PELTON = 1
CC_LITERAL = 2
GATES_FP32 = 0
GATES_TF32_SPLIT = 1
GATES_BF16_SPLIT = 2
F32_SHAPES = 10  # AEM_F32_SHAPES: launch shapes of the FP32 forward kernel


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise AEMError("paper_2109_00661_gb300 needs a CUDA device; there is no CPU path")
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class System:
    """aem_system: loop geometry plus the precomputed Hankel rule and transform matrix."""

    def __init__(self, loop_radius=13.0, height=30.0, current=1.0, n_freq=60, f_min_hz=1.0, f_max_hz=1e7,
                 gate_times=None, n_hankel=200, cc_form=CC_PAPER):
        _torch()
        lib = _lib.load()
        if gate_times is None:
            gate_times = np.logspace(-5, -2, 30)
        self._times = np.ascontiguousarray(gate_times, dtype=np.float64)
        desc = _lib.SystemDesc(float(loop_radius), float(height), float(current), int(n_freq), float(f_min_hz),
                               float(f_max_hz), len(self._times),
                               self._times.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(n_hankel),
                               int(cc_form))
        h = ctypes.c_void_p()
        check(lib.aem_system_create(ctypes.byref(desc), ctypes.byref(h)), "aem_system_create")
        self._h = h
        self.F, self.G, self.K = int(n_freq), len(self._times), int(n_hankel)
        self.loop_radius, self.height, self.current, self.cc_form = loop_radius, height, current, cc_form
        self.times = self._times.copy()

    @property
    def handle(self):
        return self._h

    def tables(self):
        """Host copies of (freqs_hz [F], lambda [K], hankel_w [K], T [G, F])."""
        f = np.zeros(self.F)
        lam = np.zeros(self.K)
        hw = np.zeros(self.K)
        T = np.zeros((self.G, self.F))
        check(_lib.load().aem_system_tables(self._h, f.ctypes.data, lam.ctypes.data, hw.ctypes.data, T.ctypes.data),
              "aem_system_tables")
        return f, lam, hw, T

    def autotune(self, models, repeats=3, stream=None):
        """aem_autotune_forward on a sample batch (float32 CUDA model tensors):
        records the fastest launch shape of the FP32 forward kernel for the
        batch's lmax; returns (shape, per-shape ms, -1 where a shape does not fit)."""
        torch = _torch()
        ms = _models_struct(models, torch.float32)
        shape = ctypes.c_int()
        times = (ctypes.c_float * F32_SHAPES)()
        check(_lib.load().aem_autotune_forward(self._h, ctypes.byref(ms), int(repeats), _stream_ptr(stream),
                                               ctypes.byref(shape), times), "aem_autotune_forward")
        return shape.value, [float(t) for t in times]

    def set_forward_shape(self, lmax, shape):
        """aem_forward_shape: the FP32 forward kernel's launch shape for lmax."""
        check(_lib.load().aem_forward_shape(self._h, int(lmax), int(shape)), "aem_forward_shape")

    def set_depth_cutoff(self, attenuation):
        """aem_system_set_depth_cutoff: the FP32 forward kernel drops the layers
        below the depth where the round-trip attenuation exceeds
        exp(-attenuation) (times the model's conductivity contrast); 0 keeps
        every layer.  Default 20."""
        check(_lib.load().aem_system_set_depth_cutoff(self._h, float(attenuation)), "aem_system_set_depth_cutoff")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().aem_system_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _models_struct(models, dtype):
    torch = _torch()
    nl = models["nlayers"]
    arrs = [models[k] for k in ("logsig", "logh", "m", "logtau", "c")]
    for a in arrs:
        if a.dtype != dtype or not a.is_cuda or not a.is_contiguous() or a.dim() != 2:
            raise AEMError(f"model arrays must be contiguous 2-D CUDA tensors of {dtype}")
    if nl.dtype != torch.int8 or not nl.is_cuda:
        raise AEMError("nlayers must be a CUDA int8 tensor")
    P, lmax = arrs[0].shape
    return _lib.Models(P, lmax, nl.data_ptr(), *[a.data_ptr() for a in arrs])


def _forward(fn, models, dtype, want_gates, want_imh, system, stream):
    torch = _torch()
    ms = _models_struct(models, dtype)
    P = ms.n_models
    dev = models["logsig"].device
    gates = torch.empty((P, system.G), dtype=dtype, device=dev) if want_gates else None
    imh = torch.empty((P, system.F), dtype=dtype, device=dev) if want_imh else None
    check(fn(system.handle, ctypes.byref(ms), _dptr(gates), _dptr(imh), _stream_ptr(stream)), fn.__name__)
    return gates, imh


def forward_f32(system, models, want_imh=False, stream=None):
    """aem_forward_f32: gates [P, G] (float32), and Im Hz_s [P, F] when want_imh."""
    g, i = _forward(_lib.load().aem_forward_f32, models, _torch().float32, True, want_imh, system, stream)
    return (g, i) if want_imh else g


def forward_f64(system, models, want_imh=False, stream=None):
    """aem_forward_f64: the plain double-precision form of the same kernel."""
    g, i = _forward(_lib.load().aem_forward_f64, models, _torch().float64, True, want_imh, system, stream)
    return (g, i) if want_imh else g


def spectrum_f32(system, models, stream=None, out=None):
    """aem_forward_f32 with the spectrum only: Im Hz_s [P, F] (float32), into
    out (a contiguous [P, F] CUDA float32 tensor) when given."""
    if out is None:
        return _forward(_lib.load().aem_forward_f32, models, _torch().float32, False, True, system, stream)[1]
    torch = _torch()
    ms = _models_struct(models, torch.float32)
    if out.dtype != torch.float32 or not out.is_contiguous() or tuple(out.shape) != (ms.n_models, system.F):
        raise AEMError("out must be a contiguous [P, F] float32 CUDA tensor")
    check(_lib.load().aem_forward_f32(system.handle, ctypes.byref(ms), None, _dptr(out), _stream_ptr(stream)),
          "aem_forward_f32")
    return out


def forward_layer_steps(system, models, stream=None):
    """aem_forward_f32_count: the (layer, abscissa pair) steps the FP32
    recursion runs on this batch (an int), and the fraction of the whole
    stack, P F ceil(K/2) sum(L) / P, that it is (the depth cutoff's share)."""
    torch = _torch()
    ms = _models_struct(models, torch.float32)
    dev = models["logsig"].device
    steps = torch.zeros(1, dtype=torch.int64, device=dev)
    scratch = torch.empty((max(ms.n_models, 1), system.F), dtype=torch.float32, device=dev)
    check(_lib.load().aem_forward_f32_count(system.handle, ctypes.byref(ms), None, _dptr(scratch), _dptr(steps),
                                            _stream_ptr(stream)), "aem_forward_f32_count")
    n = int(steps.item())
    full = int(models["nlayers"].to(torch.int64).sum().item()) * system.F * ((system.K + 1) // 2)
    return n, (n / full if full else 1.0)


def _obs(y_obs, eps_an, system, dev):
    torch = _torch()
    y = torch.as_tensor(y_obs, dtype=torch.float64, device=dev).contiguous()
    e = torch.as_tensor(eps_an, dtype=torch.float64, device=dev).expand(system.G).contiguous()
    return y, e


def gates_from_spectrum(system, imh, mode=GATES_TF32_SPLIT, y_obs=None, eps_an=None, eps_mn=0.0, want_gates=True,
                        stream=None, ll_out=None):
    """aem_gates_from_spectrum: gates [P, G] (float32, or None) and, when y_obs
    is given, ll [P] (float64, else None; into ll_out when given) from spectra
    imh [P, F] (float32)."""
    torch = _torch()
    if imh.dtype != torch.float32 or not imh.is_cuda or not imh.is_contiguous() or imh.dim() != 2:
        raise AEMError("imh must be a contiguous 2-D CUDA float32 tensor")
    P = imh.shape[0]
    gates = torch.empty((P, system.G), dtype=torch.float32, device=imh.device) if want_gates else None
    ll = y = e = None
    if y_obs is not None:
        y, e = _obs(y_obs, eps_an, system, imh.device)
        ll = ll_out if ll_out is not None else torch.empty(P, dtype=torch.float64, device=imh.device)
        if ll.dtype != torch.float64 or not ll.is_contiguous() or ll.numel() != P:
            raise AEMError("ll_out must be a contiguous float64 CUDA tensor of P elements")
    check(_lib.load().aem_gates_from_spectrum(system.handle, _dptr(imh), P, int(mode), _dptr(y), _dptr(e),
                                              float(eps_mn), _dptr(gates), _dptr(ll), _stream_ptr(stream)),
          "aem_gates_from_spectrum")
    return gates, ll


def loglik_f32_tc(system, models, y_obs, eps_an, eps_mn, mode=GATES_TF32_SPLIT, want_gates=False, stream=None):
    """aem_loglik_f32_tc: the FP32 forward model with the gate transform of
    `mode` (tensor-core TF32 / BF16 split, or FP32); ll [P] (and gates)."""
    torch = _torch()
    ms = _models_struct(models, torch.float32)
    P = ms.n_models
    dev = models["logsig"].device
    y, e = _obs(y_obs, eps_an, system, dev)
    work = torch.empty((P, system.F), dtype=torch.float32, device=dev)
    ll = torch.empty(P, dtype=torch.float64, device=dev)
    gates = torch.empty((P, system.G), dtype=torch.float32, device=dev) if want_gates else None
    check(_lib.load().aem_loglik_f32_tc(system.handle, ctypes.byref(ms), _dptr(y), _dptr(e), float(eps_mn),
                                        int(mode), _dptr(work), _dptr(ll), _dptr(gates), _stream_ptr(stream)),
          "aem_loglik_f32_tc")
    return (ll, gates) if want_gates else ll


def debug_bounded_wait(system, spins=0, skip_first_mma=False):
    """aem_debug_bounded_wait: the tensor-core transform's completion-wait limit
    (0: the default) and whether its CTAs skip the first tile's MMAs (tests)."""
    check(_lib.load().aem_debug_bounded_wait(system.handle, int(spins), int(skip_first_mma)),
          "aem_debug_bounded_wait")


def system_status(system):
    """aem_system_status: 0, or the error a kernel recorded (cleared on read)."""
    v = ctypes.c_int()
    check(_lib.load().aem_system_status(system.handle, ctypes.byref(v)), "aem_system_status")
    return v.value


def _loglik(fn, models, dtype, y_obs, eps_an, eps_mn, system, want_gates, stream):
    torch = _torch()
    ms = _models_struct(models, dtype)
    P = ms.n_models
    dev = models["logsig"].device
    y_obs = torch.as_tensor(y_obs, dtype=torch.float64, device=dev).contiguous()
    eps_an = torch.as_tensor(eps_an, dtype=torch.float64, device=dev).expand(system.G).contiguous()
    ll = torch.empty(P, dtype=torch.float64, device=dev)
    gates = torch.empty((P, system.G), dtype=dtype, device=dev) if want_gates else None
    check(fn(system.handle, ctypes.byref(ms), _dptr(y_obs), _dptr(eps_an), float(eps_mn), _dptr(ll), _dptr(gates),
             _stream_ptr(stream)), fn.__name__)
    return (ll, gates) if want_gates else ll


def loglik_f32(system, models, y_obs, eps_an, eps_mn, want_gates=False, stream=None):
    """aem_loglik_f32: Gaussian log-likelihood [P] (float64 sums of FP32 predictions)."""
    return _loglik(_lib.load().aem_loglik_f32, models, _torch().float32, y_obs, eps_an, eps_mn, system,
                   want_gates, stream)


def loglik_f64(system, models, y_obs, eps_an, eps_mn, want_gates=False, stream=None):
    """aem_loglik_f64: the same likelihood on the double-precision forward model."""
    return _loglik(_lib.load().aem_loglik_f64, models, _torch().float64, y_obs, eps_an, eps_mn, system,
                   want_gates, stream)


def loglik_grad_f32(system, models, y_obs, eps_an, eps_mn, stream=None):
    """aem_loglik_grad_f32: (ll [P] float64, grad [P, lmax, 5] float32) with the
    gradient taken with respect to (log10 sigma, log10 h, m, log10 tau, c)."""
    torch = _torch()
    ms = _models_struct(models, torch.float32)
    P, lmax = ms.n_models, ms.lmax
    dev = models["logsig"].device
    y_obs = torch.as_tensor(y_obs, dtype=torch.float64, device=dev).contiguous()
    eps_an = torch.as_tensor(eps_an, dtype=torch.float64, device=dev).expand(system.G).contiguous()
    ll = torch.empty(P, dtype=torch.float64, device=dev)
    grad = torch.empty((P, lmax, 5), dtype=torch.float32, device=dev)
    check(_lib.load().aem_loglik_grad_f32(system.handle, ctypes.byref(ms), _dptr(y_obs), _dptr(eps_an),
                                          float(eps_mn), _dptr(ll), _dptr(grad), _stream_ptr(stream)),
          "aem_loglik_grad_f32")
    return ll, grad


PARAMS = ("logsig", "logh", "m", "logtau", "c")


def _autograd_function():
    torch = _torch()

    class _LogLik(torch.autograd.Function):
        """ll(models) with the adjoint kernel's gradient as its backward: the
        forward call runs aem_loglik_grad_f32 once (likelihood and gradient in
        one launch) and backward only scales the stored gradient."""

        @staticmethod
        def forward(ctx, system, nlayers, y_obs, eps_an, eps_mn, logsig, logh, m, logtau, c):
            models = dict(nlayers=nlayers, logsig=logsig.detach(), logh=logh.detach(), m=m.detach(),
                          logtau=logtau.detach(), c=c.detach())
            ll, grad = loglik_grad_f32(system, models, y_obs, eps_an, eps_mn)
            ctx.save_for_backward(grad)
            return ll

        @staticmethod
        def backward(ctx, g_ll):
            (grad,) = ctx.saved_tensors
            scale = g_ll.to(grad.dtype)[:, None]
            return (None, None, None, None, None, *[scale * grad[:, :, i] for i in range(5)])

    return _LogLik


_LOGLIK_FN = None


def loglik(system, models, y_obs, eps_an, eps_mn):
    """Differentiable FP32 log-likelihood: a torch.autograd.Function whose
    backward is the reverse-mode adjoint kernel.  models holds float32 CUDA
    tensors (logsig, logh, m, logtau, c) of shape [P, lmax] (any of which may
    require grad) and int8 nlayers [P]; returns ll [P] float64.  When no
    gradient can be needed (grad mode off, or no parameter tensor requires
    grad) it is the plain aem_loglik_f32 launch, without the adjoint."""
    global _LOGLIK_FN
    torch = _torch()
    if not (torch.is_grad_enabled() and any(models[k].requires_grad for k in PARAMS)):
        plain = {k: (models[k].detach() if k in PARAMS else models[k]) for k in ("nlayers",) + PARAMS}
        return loglik_f32(system, plain, y_obs, eps_an, eps_mn)
    if _LOGLIK_FN is None:
        _LOGLIK_FN = _autograd_function()
    return _LOGLIK_FN.apply(system, models["nlayers"], y_obs, eps_an, eps_mn, *[models[k] for k in PARAMS])


def probe_peaks():
    """aem_probe_peaks: measured FP32 FMA/s, MUFU ex2/s, FP64 FMA/s and the
    forward recursion's MUFU mix (ops/s)."""
    _torch()
    out = [ctypes.c_double() for _ in range(4)]
    check(_lib.load().aem_probe_peaks(*[ctypes.byref(o) for o in out]), "aem_probe_peaks")
    return dict(fp32_fma_per_s=out[0].value, mufu_ex2_per_s=out[1].value, fp64_fma_per_s=out[2].value,
                mufu_mix_per_s=out[3].value)
