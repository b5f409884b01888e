"""Binding of the RJSMC stage entry points (smc_* and the standalone a7/a8
kernels of include/aem_rjsmc.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import AEMError, check

SLOTS = 10
GRAD_DIM = 3 + 4 * SLOTS  # AEM_SMC_GRAD_DIM: phi_b, phi_c[10], z_c[10], z_m[10], m[10], tau coordinate, c
MOVES = ("sigma_birth", "sigma_death", "m_birth", "m_death", "depth", "perturb")


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise AEMError("paper_2109_00661_gb300 needs a CUDA device; there is no CPU path")
    return torch


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def desc_defaults(**kw):
    d = _lib.SMCDesc()
    check(_lib.load().smc_desc_defaults(ctypes.byref(d)), "smc_desc_defaults")
    for k, v in kw.items():
        if not hasattr(d, k):
            raise AEMError(f"unknown smc_desc field {k}")
        setattr(d, k, v)
    return d


class Particles:
    """Host copy of a particle set (numpy arrays)."""

    FIELDS = (("kappa", np.int32, 1), ("lam", np.int32, 1), ("phib", np.float32, 1), ("tau", np.float32, 1),
              ("c", np.float32, 1), ("zc", np.float32, SLOTS), ("phic", np.float32, SLOTS),
              ("zm", np.float32, SLOTS), ("mv", np.float32, SLOTS), ("ll", np.float64, 1))

    def __init__(self, P):
        for name, dt, w in self.FIELDS:
            setattr(self, name, np.zeros((P, w) if w > 1 else P, dtype=dt))
        self.move = np.zeros(P, dtype=np.int8)
        self.valid = np.zeros(P, dtype=np.int8)

    def struct(self):
        return _lib.ParticlesHost(*[getattr(self, n).ctypes.data for n, _, _ in self.FIELDS],
                                  self.move.ctypes.data, self.valid.ctypes.data)


class SMC:
    """smc_state: RJSMC over S independent soundings of N particles each."""

    def __init__(self, system, y_obs, eps_an, eps_mn, stream=None, **desc):
        torch = _torch()
        lib = _lib.load()
        self.desc = desc_defaults(**desc)
        self.S, self.N = self.desc.n_soundings, self.desc.n_particles
        self.P = self.S * self.N
        self.M = (self.desc.kappa_max + 1) * (self.desc.lambda_max + 1)
        y = np.ascontiguousarray(np.broadcast_to(np.asarray(y_obs, dtype=np.float64), (self.S, system.G)))
        ea = np.ascontiguousarray(np.broadcast_to(np.asarray(eps_an, dtype=np.float64), (system.G,)))
        self._stream_obj = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        check(lib.smc_create(system.handle, ctypes.byref(self.desc), y.ctypes.data, ea.ctypes.data, float(eps_mn),
                             ctypes.c_void_p(self._stream_obj.cuda_stream), ctypes.byref(h)), "smc_create")
        self._h = h
        self.system = system

    def init(self):
        check(_lib.load().smc_init(self._h), "smc_init")

    def reweight(self):
        g = np.zeros(self.S)
        check(_lib.load().smc_reweight(self._h, g.ctypes.data), "smc_reweight")
        return g

    def resample(self):
        check(_lib.load().smc_resample(self._h), "smc_resample")

    def mutate(self, n_sweeps=0):
        check(_lib.load().smc_mutate(self._h, int(n_sweeps)), "smc_mutate")

    def propose(self, stage, sweep):
        check(_lib.load().smc_propose(self._h, int(stage), int(sweep)), "smc_propose")

    def loglik_current(self):
        check(_lib.load().smc_loglik_current(self._h), "smc_loglik_current")

    def grad_current(self):
        """smc_grad_current: [P, GRAD_DIM] float32 gradient of the log-likelihood
        with respect to each current particle's parameters (slot layout of
        AEM_SMC_GRAD_DIM); also refreshes the current particles' ll."""
        g = np.zeros((self.P, GRAD_DIM), dtype=np.float32)
        check(_lib.load().smc_grad_current(self._h, g.ctypes.data), "smc_grad_current")
        return g

    def langevin_propose(self, stage, sweep):
        check(_lib.load().smc_langevin_propose(self._h, int(stage), int(sweep)), "smc_langevin_propose")

    def langevin(self, n_sweeps):
        check(_lib.load().smc_langevin(self._h, int(n_sweeps)), "smc_langevin")

    def langevin_stats(self):
        """(accepted [S], proposed [S], h [S]) of the last mutate / langevin call."""
        acc = np.zeros(self.S, dtype=np.int32)
        prop = np.zeros(self.S, dtype=np.int32)
        h = np.zeros(self.S)
        check(_lib.load().smc_langevin_stats(self._h, acc.ctypes.data, prop.ctypes.data, h.ctypes.data),
              "smc_langevin_stats")
        return acc, prop, h

    def run(self, max_stages=1000, n_sweeps=0):
        t = ctypes.c_int()
        check(_lib.load().smc_run(self._h, int(max_stages), int(n_sweeps), ctypes.byref(t)), "smc_run")
        return t.value

    def run_graph(self, max_stages=1000, n_sweeps=10):
        """smc_run_graph: the stage loop captured as a CUDA graph with a device-side
        loop condition (n_sweeps random-walk sweeps per stage, or App. B's R_t
        decided on the device when n_sweeps <= 0, plus the descriptor's adaptive,
        recycling and Langevin steps)."""
        t = ctypes.c_int()
        check(_lib.load().smc_run_graph(self._h, int(max_stages), int(n_sweeps), ctypes.byref(t)), "smc_run_graph")
        return t.value

    def status(self):
        """smc_status: (status, nonfinite [S]): the failure a reweight step
        recorded since the last call (0 for none; cleared on read) and the per
        sounding count of non-finite log-likelihoods set to -inf since init."""
        v = ctypes.c_int()
        nf = np.zeros(self.S, dtype=np.int32)
        check(_lib.load().smc_status(self._h, ctypes.byref(v), nf.ctypes.data), "smc_status")
        return v.value, nf

    def model_odds(self):
        post = np.zeros((self.S, self.M))
        lb = np.zeros(self.S)
        lz = np.zeros((self.S, self.M))
        check(_lib.load().smc_model_odds(self._h, post.ctypes.data, lb.ctypes.data, lz.ctypes.data), "smc_model_odds")
        return post, lb, lz

    def stats(self):
        g = np.zeros(self.S)
        st = ctypes.c_int()
        acc = np.zeros((self.S, 6), dtype=np.int32)
        prop = np.zeros((self.S, 6), dtype=np.int32)
        check(_lib.load().smc_stats(self._h, g.ctypes.data, ctypes.byref(st), acc.ctypes.data, prop.ctypes.data),
              "smc_stats")
        return dict(gamma=g, stage=st.value, accepted=acc, proposed=prop)

    def get_particles(self, which=0):
        p = Particles(self.P)
        s = p.struct()
        check(_lib.load().smc_get_particles(self._h, int(which), ctypes.byref(s)), "smc_get_particles")
        return p

    def set_particles(self, p, gamma=None, log_z=None, stage=-1):
        s = p.struct()
        g = None if gamma is None else np.ascontiguousarray(gamma, dtype=np.float64)
        lz = None if log_z is None else np.ascontiguousarray(log_z, dtype=np.float64)
        check(_lib.load().smc_set_particles(self._h, ctypes.byref(s), None if g is None else g.ctypes.data,
                                            None if lz is None else lz.ctypes.data, int(stage)), "smc_set_particles")

    def log_factors(self):
        """smc_get_log_factors: [P] log factor of each particle's last proposal."""
        lf = np.zeros(self.P)
        check(_lib.load().smc_get_log_factors(self._h, lf.ctypes.data), "smc_get_log_factors")
        return lf

    def adapt(self):
        check(_lib.load().smc_adapt(self._h), "smc_adapt")

    def adaptation(self):
        """smc_get_adaptation: dict of mu [S, M, D], U [S, M, D, D], lam [S, M, D],
        scale [S, M], ok [S, M] with D = 3 + 2 kappa_max + 2 lambda_max."""
        D = 3 + 2 * self.desc.kappa_max + 2 * self.desc.lambda_max
        mu, lam = np.zeros((self.S, self.M, D)), np.zeros((self.S, self.M, D))
        U = np.zeros((self.S, self.M, D, D))
        scale = np.zeros((self.S, self.M))
        ok = np.zeros((self.S, self.M), dtype=np.int32)
        check(_lib.load().smc_get_adaptation(self._h, mu.ctypes.data, U.ctypes.data, lam.ctypes.data,
                                             scale.ctypes.data, ok.ctypes.data), "smc_get_adaptation")
        return dict(mu=mu, U=U, lam=lam, scale=scale, ok=ok)

    def ppd(self, want_gates=False):
        """smc_ppd: per-gate posterior predictive mean, variance and the data
        standardised to it, each [S, G]; with want_gates also the particles'
        predictions [P, G]."""
        G = self.system.G
        mean, var, z = (np.zeros((self.S, G)) for _ in range(3))
        gates = np.zeros((self.P, G), dtype=np.float32) if want_gates else None
        check(_lib.load().smc_ppd(self._h, mean.ctypes.data, var.ctypes.data, z.ctypes.data,
                                  gates.ctypes.data if want_gates else None), "smc_ppd")
        return (mean, var, z, gates) if want_gates else (mean, var, z)

    def checkpoint(self) -> bytes:
        """smc_checkpoint: the sampler's dynamic state as bytes."""
        lib = _lib.load()
        n = ctypes.c_size_t(0)
        check(lib.smc_checkpoint(self._h, None, ctypes.byref(n)), "smc_checkpoint")
        buf = ctypes.create_string_buffer(n.value)
        check(lib.smc_checkpoint(self._h, buf, ctypes.byref(n)), "smc_checkpoint")
        return buf.raw[:n.value]

    def restore(self, image: bytes):
        """smc_restore from bytes written by checkpoint()."""
        buf = ctypes.create_string_buffer(bytes(image), len(image))
        check(_lib.load().smc_restore(self._h, buf, len(image)), "smc_restore")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().smc_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _workspace(n, n_models, device):
    torch = _torch()
    nbytes = int(_lib.load().aem_smc_workspace_bytes(int(n), int(n_models)))
    return torch.empty(nbytes + 64, dtype=torch.uint8, device=device), nbytes


def _aligned(buf):
    p = buf.data_ptr()
    return p + ((64 - p % 64) % 64)


def reweight(ll, model, n_models, gamma_prev, alpha, bisect_iters=60, stream=None):
    """aem_reweight on device tensors: returns (dgamma, reached_one, logz_inc[n_models], W[n])."""
    torch = _torch()
    n = ll.numel()
    dev = ll.device
    ws, nbytes = _workspace(n, n_models, dev)
    dg = torch.empty(1, dtype=torch.float64, device=dev)
    done = torch.empty(1, dtype=torch.int32, device=dev)
    inc = torch.empty(n_models, dtype=torch.float64, device=dev)
    W = torch.empty(n, dtype=torch.float64, device=dev)
    check(_lib.load().aem_reweight(ll.data_ptr(), model.data_ptr(), n, n_models, float(gamma_prev), float(alpha),
                                   int(bisect_iters), dg.data_ptr(), done.data_ptr(), inc.data_ptr(), W.data_ptr(),
                                   _aligned(ws), nbytes, _stream(stream)), "aem_reweight")
    return dg, done, inc, W


def resample_systematic(W, model, n_models, u40, stream=None):
    """aem_resample_systematic on device tensors: ancestor index of every particle."""
    torch = _torch()
    n = W.numel()
    ws, nbytes = _workspace(n, n_models, W.device)
    anc = torch.empty(n, dtype=torch.int32, device=W.device)
    check(_lib.load().aem_resample_systematic(W.data_ptr(), model.data_ptr(), n, n_models, u40.data_ptr(),
                                              anc.data_ptr(), _aligned(ws), nbytes, _stream(stream)),
          "aem_resample_systematic")
    return anc


def resample_systematic_noalloc(W, model, n_models, u40, stream=None):
    """aem_resample_systematic_noalloc: the same resampling with the library's
    static scratch instead of a workspace (the output tensor is the caller's)."""
    torch = _torch()
    n = W.numel()
    anc = torch.empty(n, dtype=torch.int32, device=W.device)
    check(_lib.load().aem_resample_systematic_noalloc(W.data_ptr(), model.data_ptr(), n, n_models, u40.data_ptr(),
                                                      anc.data_ptr(), _stream(stream)),
          "aem_resample_systematic_noalloc")
    return anc


def philox4x32(counters, key0, key1, stream=None):
    """aem_philox4x32 on a device tensor of (n, 4) int32 counters (uint32 bit patterns)."""
    torch = _torch()
    n = counters.shape[0]
    out = torch.empty((n, 4), dtype=torch.int32, device=counters.device)
    check(_lib.load().aem_philox4x32(counters.data_ptr(), int(key0), int(key1), out.data_ptr(), n, _stream(stream)),
          "aem_philox4x32")
    return out
