"""FP64 CPU oracle for the RJSMC airborne-EM hot path (arXiv 2109.00661).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2109_00661_gb300``) never imports it and
shares no code with it: the forward model here is ``aem_oracle.cpp`` (adaptive
quadrature Hankel integrals, its own transform matrix) and the sampler is the
plain serial code in ``oracle/rjsmc.py``.

Parity status of each function (what pins it, see tests/test_oracle_*.py):
  colecole      -- DC / high-frequency limits, m = 0 reduction, paper <-> Pelton
                   bijection (Section 2).
  r0            -- reflection recursion vs the independent tanh-admittance
                   recursion; split-layer and uniform-stack invariants.
  hz            -- closed-form central-loop field over a half-space (Ward &
                   Hohmann 1988, the reference the paper cites in Section 2).
  tmatrix       -- closed-form step-off transient over a half-space; exact
                   sine transform of w / (1 + (w tau)^2).
  forward       -- the above plus the late-time t^(-5/2) law at h = 30 m.
  loglik        -- hand-computed two-gate example (Section 2.3.2).
  loglik_grad_fd -- central differences of loglik; step-convergence pin.
  forward_jacobian_fd -- central differences of the gates; the chain rule
                   sum_g dl/dy_g J_g reproduces loglik_grad_fd.
  rjsmc.*       -- see oracle/rjsmc.py: toy closed-form evidence and model
                   probabilities, bisection / resampling definitions; the
                   Langevin move by invariance of a Gaussian target and the
                   particle-space gradient against the chain rule of the
                   merged-layer gradient.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aem_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with the host C++ compiler."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            d = ctypes.c_double
            i = ctypes.c_int
            p = ctypes.c_void_p
            _lib.orc_forward.argtypes = [i, i, p, p, p, p, p, p, i, d, d, d, i, p, i, p, i, i, d, p, p, i, p]
            _lib.orc_forward.restype = i
            _lib.orc_tmatrix.argtypes = [i, p, i, p, p]
            _lib.orc_colecole.argtypes = [i, d, d, d, d, d, p]
            _lib.orc_r0.argtypes = [i, p, p, p, d, d, i, p]
            _lib.orc_hz.argtypes = [i, p, p, p, d, d, d, d, i, i, d, p]
            _lib.orc_hankel_rule.argtypes = [i, d, d, d, p, p]
            _lib.orc_loglik.argtypes = [i, i, p, p, p, d, p]
            _lib.orc_merge.argtypes = [i, p, p, i, p, p, p, p, p]
            _lib.orc_merge.restype = i
        return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


MU0 = 4e-7 * np.pi

# Quadrature modes of the forward model.
QUAD_REFLECTION = 0
QUAD_ADMITTANCE = 1
HANKEL_RULE = 2


def colecole(form, sig, m, tau, c, w):
    """Complex conductivity (Section 2).  form 0: paper, 1: Pelton resistivity,
    2: Pelton's expression taken as a conductivity."""
    out = np.zeros(2)
    lib().orc_colecole(int(form), float(sig), float(m), float(tau), float(c), float(w), _ptr(out))
    return complex(out[0], out[1])


def r0(sig, thick, lam, w, method=0):
    """TE reflection coefficient at the surface.  sig: complex per layer."""
    sig = np.asarray(sig, dtype=np.complex128)
    L = len(sig)
    th = _f64(np.concatenate([np.asarray(thick, dtype=np.float64), np.zeros(max(0, L - len(thick)))]))
    sr, si = _f64(sig.real), _f64(sig.imag)
    out = np.zeros(2)
    lib().orc_r0(L, _ptr(sr), _ptr(si), _ptr(th), float(lam), float(w), int(method), _ptr(out))
    return complex(out[0], out[1])


def hz(sig, thick, a, h, w, mode=QUAD_REFLECTION, K=200, current=1.0, rtol=1e-11):
    """Secondary Hz (A/m) at the loop centre for complex layer conductivities."""
    sig = np.asarray(sig, dtype=np.complex128)
    L = len(sig)
    th = _f64(np.concatenate([np.asarray(thick, dtype=np.float64), np.zeros(max(0, L - len(thick)))]))
    sr, si = _f64(sig.real), _f64(sig.imag)
    out = np.zeros(2)
    lib().orc_hz(L, _ptr(sr), _ptr(si), _ptr(th), float(a), float(h), float(current), float(w), int(mode),
                 int(K), float(rtol), _ptr(out))
    return complex(out[0], out[1])


def hankel_rule(K, a, h, current=1.0):
    lam = np.zeros(K)
    c = np.zeros(K)
    lib().orc_hankel_rule(int(K), float(a), float(h), float(current), _ptr(lam), _ptr(c))
    return lam, c


def tmatrix(freqs, times):
    """G x F matrix taking Im Hz_s at the frequency nodes (Hz) to -dBz/dt at the gates."""
    freqs = _f64(freqs)
    times = _f64(times)
    T = np.zeros((len(times), len(freqs)))
    lib().orc_tmatrix(len(freqs), _ptr(freqs), len(times), _ptr(times), _ptr(T))
    return T


def forward(models, system, mode=QUAD_REFLECTION, rtol=1e-11, nthreads=None, want_imh=False, want_absh=False):
    """Gates -dBz/dt (T/s per the system current) for a batch of merged-layer models.

    models: dict with int 'nlayers' [P] and float arrays 'logsig', 'logh', 'm',
    'logtau', 'c' of shape [P, LMAX] (log10 of sigma_inf in S/m, thickness in
    m and tau in s).  system: dict with 'a', 'h', 'freqs', 'times', 'K',
    'cc_form', 'current' and optionally a precomputed 'T'.  With the Hankel
    rule, want_absh also returns sum_k |w_k| |R_0(lambda_k, w_f)| per node,
    the magnitude scale of the rule's sum.
    """
    nl = np.ascontiguousarray(models["nlayers"], dtype=np.int32)
    P = len(nl)
    arrs = [_f64(models[k]) for k in ("logsig", "logh", "m", "logtau", "c")]
    LMAX = arrs[0].shape[1]
    freqs = _f64(system["freqs"])
    times = _f64(system["times"])
    T = system.get("T")
    if T is None:
        T = tmatrix(freqs, times)
    T = _f64(T)
    F, G = len(freqs), len(times)
    y = np.zeros((P, G))
    imh = np.zeros((P, F)) if want_imh else None
    absh = np.zeros((P, F)) if want_absh else None
    if want_absh and mode != HANKEL_RULE:
        raise ValueError("want_absh needs the Hankel rule mode")
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    rc = lib().orc_forward(P, LMAX, _ptr(nl), *[_ptr(a) for a in arrs], int(system.get("cc_form", 0)),
                           float(system["a"]), float(system["h"]), float(system.get("current", 1.0)), F,
                           _ptr(freqs), G, _ptr(T), int(mode), int(system.get("K", 200)), float(rtol),
                           _ptr(imh), _ptr(y), int(nthreads), _ptr(absh))
    if rc != 0:
        raise ValueError("oracle forward: layer count out of range")
    out = (y,) + ((imh,) if want_imh else ()) + ((absh,) if want_absh else ())
    return out if len(out) > 1 else y


def loglik(y_model, y_obs, eps_an, eps_mn):
    """Gaussian log-likelihood per model (Section 2.3.2)."""
    y_model = _f64(np.atleast_2d(y_model))
    P, G = y_model.shape
    y_obs = _f64(y_obs)
    eps_an = _f64(np.broadcast_to(eps_an, (G,)))
    ll = np.zeros(P)
    lib().orc_loglik(P, G, _ptr(y_model), _ptr(y_obs), _ptr(eps_an), float(eps_mn), _ptr(ll))
    return ll


def merge(zc, logsig, zm, mval):
    """Direct-sum merge of the decoupled profiles (Section 2.1, Fig. 2).

    zc: conductive interface depths (kappa), logsig: kappa+1 values (background
    first); zm: chargeable interface depths (lambda), mval: lambda values.
    Returns (thickness, logsig, m) per merged layer, top to bottom.
    """
    zc = _f64(zc)
    logsig = _f64(logsig)
    zm = _f64(zm)
    mval = _f64(mval)
    n = len(zc) + len(zm) + 1
    th, ls, mm = np.zeros(n), np.zeros(n), np.zeros(n)
    L = lib().orc_merge(len(zc), _ptr(zc), _ptr(logsig), len(zm), _ptr(zm), _ptr(mval), _ptr(th), _ptr(ls),
                        _ptr(mm))
    return th[:L], ls[:L], mm[:L]


PARAMS = ("logsig", "logh", "m", "logtau", "c")


def loglik_grad_fd(models, system, y_obs, eps_an, eps_mn, step=1e-5, mode=HANKEL_RULE):
    """FP64 gradient of the log-likelihood by central differences with respect
    to every layer's (log10 sigma, log10 h, m, log10 tau, c): returns
    (ll [P], grad [P, LMAX, 5]); entries past each model's layer count and the
    basement thickness are 0."""
    base = {k: np.array(models[k], dtype=np.float64, copy=True) for k in PARAMS}
    nl = np.asarray(models["nlayers"])
    P, LMAX = base["logsig"].shape
    ll0 = loglik(forward(dict(base, nlayers=nl), system, mode=mode), y_obs, eps_an, eps_mn)
    grad = np.zeros((P, LMAX, 5))
    for pi, name in enumerate(PARAMS):
        for n in range(LMAX):
            active = (n < nl) & ~((name == "logh") & (n == nl - 1))
            if not np.any(active):
                continue
            lp = {k: v.copy() for k, v in base.items()}
            lm = {k: v.copy() for k, v in base.items()}
            lp[name][:, n] += step
            lm[name][:, n] -= step
            fp = loglik(forward(dict(lp, nlayers=nl), system, mode=mode), y_obs, eps_an, eps_mn)
            fm = loglik(forward(dict(lm, nlayers=nl), system, mode=mode), y_obs, eps_an, eps_mn)
            grad[:, n, pi] = np.where(active, (fp - fm) / (2 * step), 0.0)
    return ll0, grad


def forward_jacobian_fd(models, system, step=1e-5, mode=HANKEL_RULE):
    """FP64 Jacobian of the gates with respect to every layer's (log10 sigma,
    log10 h, m, log10 tau, c) by central differences: returns (y [P, G],
    jac [P, G, LMAX, 5]), zero past each model's layer count and for the
    basement thickness."""
    base = {k: np.array(models[k], dtype=np.float64, copy=True) for k in PARAMS}
    nl = np.asarray(models["nlayers"])
    P, LMAX = base["logsig"].shape
    y0 = forward(dict(base, nlayers=nl), system, mode=mode)
    jac = np.zeros((P, y0.shape[1], LMAX, 5))
    for pi, name in enumerate(PARAMS):
        for n in range(LMAX):
            active = (n < nl) & ~((name == "logh") & (n == nl - 1))
            if not np.any(active):
                continue
            lp = {k: v.copy() for k, v in base.items()}
            lm = {k: v.copy() for k, v in base.items()}
            lp[name][:, n] += step
            lm[name][:, n] -= step
            d = (forward(dict(lp, nlayers=nl), system, mode=mode) - forward(dict(lm, nlayers=nl), system, mode=mode))
            jac[:, :, n, pi] = np.where(active[:, None], d / (2 * step), 0.0)
    return y0, jac
