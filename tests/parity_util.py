"""Shared parity helpers: per-gate condition numbers of the step-off
transform and the error bounds the forward-model tests derive from them."""
import numpy as np

import oracle as O
from paper_2109_00661_gb300 import inputs as I

EPS_AN = I.EPS_AN

_T_cache = {}


def oracle_system(name, cc_form=0):
    s = I.oracle_system(name, cc_form)
    if name not in _T_cache:
        _T_cache[name] = O.tmatrix(s["freqs"], s["times"])
    s["T"] = _T_cache[name]
    return s


def rel_err(gpu, ref):
    return np.abs(gpu - ref) / np.maximum(np.abs(ref), EPS_AN)


def kappa(imh, T, y):
    """Condition numbers of each gate of y = T imh: elementwise (kappa) and
    against a perturbation of T bounded by its row maximum (kappa_T)."""
    den = np.maximum(np.abs(y), EPS_AN)
    k = (np.abs(imh) @ np.abs(T).T) / den
    kT = np.sum(np.abs(imh), axis=1, keepdims=True) * np.max(np.abs(T), axis=1)[None, :] / den
    return np.stack([k, kT])


def bound64(kap):
    return 1e-7 + kap[0] * 1e-9 + kap[1] * 1e-8


def bound32(kap, F):
    return 1e-4 + kap[0] * (1e-5 + (F + 1) * 2.0 ** -24) + kap[1] * 1e-8


def loglik_bound(y_model, y_obs, gate_bound, eps_an=EPS_AN, eps_mn=I.EPS_MN):
    """First-order bound on |d ll| from per-gate relative errors gate_bound
    (relative to max(|y|, eps_an)): 2 sum_g |d ll / d yhat_g| |d yhat_g|."""
    dy = gate_bound * np.maximum(np.abs(y_model), eps_an)
    v = eps_an ** 2 + (eps_mn * y_model) ** 2
    r = y_obs - y_model
    dll = np.abs(r / v + (eps_mn ** 2 * y_model / v) * (r ** 2 / v - 1.0))
    return 2.0 * np.sum(dll * dy, axis=1)
