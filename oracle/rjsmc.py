"""Serial FP64 reference of the RJSMC stage (Davies et al., arXiv 2109.00661,
Algorithm 1 with the adaptive choices of Section 3.2 and Appendices B-E).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain Python / numpy,
one particle at a time, in the order the paper states the steps:

  reweight   w = W L^(gamma_t - gamma_{t-1}) within each model, gamma_t by
             bisection so that TESS = sum_k ESS_k ~ alpha N (Section 3.2.1,
             App. C), Z_k <- Z_k sum_i w (App. D);
  resample   within-model systematic resampling, N_{t,k} held fixed (Alg. 1);
  mutate     R_t sweeps of an RJMCMC kernel: conductive / chargeable birth
             and death with properties drawn from the prior (App. E: the
             acceptance then reduces to the tempered likelihood ratio),
             interface-depth moves and component-wise Gaussian random walks;
  odds       pi(k|y) = N_k / N (Section 3.2.1) and the BFIPD statistic of
             Section 2.3.3.

Beyond the paper's kernels, an optional within-model Langevin (MALA) move on
the particle's continuous parameters, with the gradient of the tempered
target gamma_t l taken by central differences of the likelihood and the
Metropolis-Hastings test including the proposal-density ratio (Roberts &
Tweedie 1996); it leaves pi_t invariant like the paper's random walks do.

Random numbers come from Philox4x32-10 (Salmon et al., SC 2011) written out
here from its published definition, keyed per sounding and counted per
(particle, draw, stage, sweep), so the GPU sampler can reproduce the same
uniforms.  Where the paper leaves a choice open the readings are: the six
move types drawn uniformly, an impossible move counted as a rejection; one
systematic-resampling uniform per model and stage; 60 bisection steps for
the tempering increment with alpha = 0.5; the tempered likelihood in every
acceptance; P(kappa), P(lambda) uniform on 0..max (Section 2.3.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------- Philox4x32-10
_M0 = 0xD2511F53
_M1 = 0xCD9E8D57
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32(counter, key):
    """Philox4x32 with 10 rounds.  counter: (n, 4) uint32-valued, key: (k0, k1).
    Returns (n, 4) uint32 as uint64 array."""
    c = np.array(counter, dtype=np.uint64).reshape(-1, 4).copy()
    k0 = np.uint64(key[0] & _MASK)
    k1 = np.uint64(key[1] & _MASK)
    for r in range(10):
        p0 = c[:, 0] * np.uint64(_M0)
        p1 = c[:, 2] * np.uint64(_M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(_MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(_MASK)
        n0 = hi1 ^ c[:, 1] ^ k0
        n2 = hi0 ^ c[:, 3] ^ k1
        c = np.stack([n0, lo1, n2, lo0], axis=1)
        k0 = (k0 + np.uint64(_W0)) & np.uint64(_MASK)
        k1 = (k1 + np.uint64(_W1)) & np.uint64(_MASK)
    return c


def u01_from(x):
    """Uniform on (0, 1) from one 32-bit word: (x >> 8 + 1/2) * 2^-24."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(8)).astype(np.float64) + 0.5) * (2.0 ** -24)


def u01_53(x0, x1):
    """Uniform on (0, 1) with 53 bits from two words."""
    hi = (np.asarray(x0, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
    lo = (np.asarray(x1, dtype=np.uint64) >> np.uint64(5)).astype(np.float64)
    return (hi * 2.0 ** 27 + lo + 0.5) * (2.0 ** -53)


def gauss_pair(x0, x1):
    """Box-Muller from two 32-bit words (first output only)."""
    u1 = u01_from(x0)
    u2 = u01_from(x1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# Stream identities.  Counter words: (particle, purpose, stage, sweep);
# key: (seed low 32 bits, seed high 32 bits xor sounding).
PURPOSE_PRIOR0 = 0
PURPOSE_PRIOR_MAX = 63  # prior draws use purposes 0..63
PURPOSE_MOVE = 64
PURPOSE_VALUE = 65
PURPOSE_ACCEPT = 66
PURPOSE_RESAMPLE = 67


def stream_key(seed, sounding):
    return (seed & _MASK, ((seed >> 32) ^ sounding) & _MASK)


def philox4x32_one(c0, c1, c2, c3, k0, k1):
    """philox4x32 of one counter in plain Python integers (the same rounds)."""
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & _MASK, p1 & _MASK, ((p0 >> 32) ^ c3 ^ k1) & _MASK, p0 & _MASK
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def draws(seed, sounding, particle, purpose, stage, sweep):
    """Four 32-bit words for each particle index in `particle`."""
    if np.ndim(particle) == 0:
        k0, k1 = stream_key(seed, sounding)
        w = philox4x32_one(int(particle) & _MASK, purpose & _MASK, stage & _MASK, sweep & _MASK, k0, k1)
        return np.array([w], dtype=np.uint64)
    particle = np.atleast_1d(np.asarray(particle, dtype=np.uint64))
    ctr = np.zeros((len(particle), 4), dtype=np.uint64)
    ctr[:, 0] = particle
    ctr[:, 1] = purpose
    ctr[:, 2] = stage
    ctr[:, 3] = sweep
    return philox4x32(ctr, stream_key(seed, sounding))


# ------------------------------------------------------------------ settings
@dataclass
class SMCSettings:
    n_particles: int = 256
    kappa_max: int = 3
    lambda_max: int = 4
    zmax: float = 500.0
    alpha: float = 0.5          # TESS threshold proportion
    c_mut: float = 0.01         # 1 - c' (App. B)
    r_max: int = 10
    n_sweeps: int = 10          # > 0: fixed R_t; <= 0: adaptive R_t (App. B)
    step_phi: float = 0.2
    step_m: float = 0.05
    step_tau: float = 0.05
    step_c: float = 0.05
    step_z: float = 10.0
    phi_lo: float = -4.0
    phi_hi: float = 2.0
    tau_log_prior: bool = False  # False: tau ~ U(0, 1) s (Section 2.3.1); True: log10 tau ~ U(lo, hi)
    logtau_lo: float = -6.0
    logtau_hi: float = -1.0
    seed: int = 0
    sounding: int = 0
    bisect_iters: int = 60
    n_langevin: int = 0         # Langevin sweeps per stage after the random-walk sweeps
    langevin_h: float = 0.1     # initial Langevin step, in units of the random-walk scales
    langevin_adapt: bool = True  # adapt the step between stages towards LANGEVIN_TARGET acceptance
    adaptive: bool = False      # the paper's adaptive within-model proposal replaces the fixed-scale perturb move
    pca_target: float = 0.44    # acceptance rate the scale bisection aims at (Section 3.2)
    pca_bisect_iters: int = 6   # bisection steps on trial proposals per stage
    pca_ridge: float = 0.01     # ridge on the fitted covariance, as a fraction of the random-walk scales
    recycle: int = 0            # > 0: fit the adaptive proposal on the last `recycle` stages' particles (Section 3.2)
    zca: float = 0.0            # with adaptive: probability that a birth/death is the ZCA-coloured one of App. F

    @property
    def n_models(self):
        return (self.kappa_max + 1) * (self.lambda_max + 1)


# Move types, chosen uniformly (a move that is impossible in the current
# model is proposed and counted as a rejection).
MOVES = ("sigma_birth", "sigma_death", "m_birth", "m_death", "depth", "perturb")


@dataclass
class Particle:
    kappa: int
    lam: int
    phib: float
    zc: list
    phic: list
    zm: list
    mv: list
    tau: float
    c: float

    def model(self, s: SMCSettings):
        return self.kappa * (s.lambda_max + 1) + self.lam

    def copy(self):
        return Particle(self.kappa, self.lam, self.phib, list(self.zc), list(self.phic), list(self.zm),
                        list(self.mv), self.tau, self.c)


# -------------------------------------------------------------------- prior
# Prior draw layout: draw index d uses word d % 4 of the Philox block with
# purpose d // 4 (purposes 0..17).
PRIOR_SLOTS = 16  # reserved interface slots per profile
D_KAPPA, D_LAM, D_PHIB, D_TAU, D_C = 0, 1, 2, 3, 4
D_ZC = 5
D_PHIC = D_ZC + PRIOR_SLOTS
D_ZM = D_PHIC + PRIOR_SLOTS
D_MV = D_ZM + PRIOR_SLOTS
N_PRIOR_DRAWS = D_MV + PRIOR_SLOTS


def prior_uniforms(s: SMCSettings, i: int):
    words = np.concatenate([draws(s.seed, s.sounding, i, p, 0, 0)[0] for p in range((N_PRIOR_DRAWS + 3) // 4)])
    return u01_from(words)


def sample_prior(s: SMCSettings, i: int) -> Particle:
    """kappa ~ U{0..kappa_max}, lambda ~ U{0..lambda_max}; depths are sorted
    uniforms on (0, zmax) (density k!/zmax^k); log10 sigma ~ U(-4, 2); m ~ U(0,1);
    tau, c global (Section 2.3.1)."""
    u = prior_uniforms(s, i)
    kappa = min(int(u[D_KAPPA] * (s.kappa_max + 1)), s.kappa_max)
    lam = min(int(u[D_LAM] * (s.lambda_max + 1)), s.lambda_max)
    phib = s.phi_lo + (s.phi_hi - s.phi_lo) * u[D_PHIB]
    if s.tau_log_prior:
        tau = 10.0 ** (s.logtau_lo + (s.logtau_hi - s.logtau_lo) * u[D_TAU])
    else:
        tau = u[D_TAU]
    c = u[D_C]
    zc = [s.zmax * u[D_ZC + j] for j in range(kappa)]
    phic = [s.phi_lo + (s.phi_hi - s.phi_lo) * u[D_PHIC + j] for j in range(kappa)]
    zm = [s.zmax * u[D_ZM + j] for j in range(lam)]
    mv = [u[D_MV + j] for j in range(lam)]
    oc = np.argsort(zc, kind="stable")
    om = np.argsort(zm, kind="stable")
    return Particle(kappa, lam, phib, [zc[j] for j in oc], [phic[j] for j in oc], [zm[j] for j in om],
                    [mv[j] for j in om], tau, c)


def in_prior(p: Particle, s: SMCSettings) -> bool:
    if not (s.phi_lo < p.phib < s.phi_hi):
        return False
    if any(not (s.phi_lo < v < s.phi_hi) for v in p.phic):
        return False
    if any(not (0.0 < v < 1.0) for v in p.mv):
        return False
    if any(not (0.0 < z < s.zmax) for z in p.zc + p.zm):
        return False
    if s.tau_log_prior:
        if not (s.logtau_lo < math.log10(p.tau) < s.logtau_hi):
            return False
    elif not (0.0 < p.tau < 1.0):
        return False
    return 0.0 < p.c < 1.0


# ---------------------------------------------------------------- merge (a1)
def merge_particle(p: Particle, lmax: int):
    """Direct sum of the decoupled profiles (Section 2.1, Fig. 2): returns
    (L, logsig[lmax], logh[lmax], m[lmax], logtau[lmax], c[lmax])."""
    z = sorted(p.zc + p.zm)
    L = len(z) + 1
    logsig = np.zeros(lmax)
    logh = np.zeros(lmax)
    m = np.zeros(lmax)
    for n in range(L):
        top = 0.0 if n == 0 else z[n - 1]
        ic = sum(1 for v in p.zc if v <= top) if n > 0 else 0
        jm = sum(1 for v in p.zm if v <= top) if n > 0 else 0
        logsig[n] = p.phib if ic == 0 else p.phic[ic - 1]
        m[n] = 0.0 if jm == 0 else p.mv[jm - 1]
        if n < L - 1:
            # coincident conductive and chargeable interfaces leave a
            # zero-thickness merged layer (thickness floored at 1e-30 m)
            logh[n] = math.log10(max(z[n] - top, 1e-30))
    return L, logsig, logh, m, np.full(lmax, math.log10(p.tau)), np.full(lmax, p.c)


def merged_batch(parts, lmax):
    P = len(parts)
    out = dict(nlayers=np.zeros(P, dtype=np.int8), logsig=np.zeros((P, lmax)), logh=np.zeros((P, lmax)),
               m=np.zeros((P, lmax)), logtau=np.zeros((P, lmax)), c=np.zeros((P, lmax)))
    for i, p in enumerate(parts):
        L, ls, lh, mm, lt, cc = merge_particle(p, lmax)
        out["nlayers"][i] = L
        out["logsig"][i] = ls
        out["logh"][i] = lh
        out["m"][i] = mm
        out["logtau"][i] = lt
        out["c"][i] = cc
    return out


# -------------------------------------------------------------- reweight (a7)
def _lse(v):
    v = np.asarray(v, dtype=np.float64)
    if v.size == 0:
        return -np.inf
    m = np.max(v)
    if not np.isfinite(m):
        return m
    return m + math.log(float(np.sum(np.exp(v - m))))


def tess(ll, model, n_models, dgamma):
    """TESS = sum_k ESS_k with ESS_k = (sum_i w_i)^2 / sum_i w_i^2 over model k's
    particles, w_i = L_i^dgamma with uniform W within each model (App. C)."""
    total = 0.0
    for k in range(n_models):
        a = dgamma * ll[model == k]
        if a.size == 0:
            continue
        total += math.exp(2.0 * _lse(a) - _lse(2.0 * a))
    return total


def choose_dgamma(ll, model, n_models, gamma_prev, alpha, iters=60):
    """Bisection on dgamma in (0, 1 - gamma_prev] so that TESS ~ alpha N
    (Alg. 1, Section 3.2.1).  Takes the whole remaining step when it keeps
    TESS >= alpha N; otherwise the largest bisection point found with
    TESS >= alpha N (the smallest failing point if none was found)."""
    N = len(ll)
    target = alpha * N
    hi = 1.0 - gamma_prev
    if tess(ll, model, n_models, hi) >= target:
        return hi, True
    lo = 0.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if tess(ll, model, n_models, mid) >= target:
            lo = mid
        else:
            hi = mid
    return (lo if lo > 0.0 else hi), False


def reweight(ll, model, n_models, gamma_prev, alpha, iters=60):
    """One re-weighting step.  Returns (dgamma, reached_one, logz_increment[k],
    W[i] normalised within each model)."""
    dg, done = choose_dgamma(ll, model, n_models, gamma_prev, alpha, iters)
    inc = np.zeros(n_models)
    W = np.zeros(len(ll))
    for k in range(n_models):
        idx = np.nonzero(model == k)[0]
        if idx.size == 0:
            continue
        a = dg * ll[idx]
        l = _lse(a)
        inc[k] = l - math.log(idx.size)  # log of sum_i W_{t-1} w, W_{t-1} = 1/N_k (App. D)
        W[idx] = np.exp(a - l)
    return dg, done, inc, W


# -------------------------------------------------------------- resample (a8)
CDF_BITS = 40


def resample_systematic(W, model, n_models, u40):
    """Within-model systematic resampling with an integer CDF.

    For model k with particles i_0 < i_1 < ... (index order), q_j =
    round(W_{i_j} 2^40), C_j = q_0 + ... + q_j with the last C forced to 2^40;
    the j-th output slot (the j-th particle of model k in index order) takes the
    smallest j' with C_{j'} > floor((j 2^40 + u40_k) / N_k).  Returns the
    ancestor index of every particle."""
    one = 1 << CDF_BITS
    anc = np.arange(len(W))
    for k in range(n_models):
        idx = np.nonzero(model == k)[0]
        n = idx.size
        if n == 0:
            continue
        q = [int(round(float(W[i]) * one)) for i in idx]
        C = []
        acc = 0
        for v in q:
            acc += v
            C.append(acc)
        C[-1] = one
        for j in range(n):
            thr = (j * one + int(u40[k])) // n
            sel = next(jj for jj in range(n) if C[jj] > thr)
            anc[idx[j]] = idx[sel]
    return anc


def resample_uniforms(s: SMCSettings, stage: int):
    """u40_k for each model: the low 40 bits of (x0 << 8 | x1 >> 24)."""
    d = draws(s.seed, s.sounding, np.arange(s.n_models), PURPOSE_RESAMPLE, stage, 0)
    return ((d[:, 0] << np.uint64(8)) | (d[:, 1] >> np.uint64(24))) & np.uint64((1 << CDF_BITS) - 1)


# --------------------------------------------------------------- mutate (a9)
def sweeps_needed(p_acc_min, c_mut, r_max):
    """R = ceil(log c / log(1 - p_acc^min)) (App. B), clamped to [1, r_max]."""
    if p_acc_min <= 0.0:
        return r_max
    if p_acc_min >= 1.0:
        return 1
    r = math.ceil(math.log(c_mut) / math.log(1.0 - p_acc_min))
    return max(1, min(r_max, r))


def propose(p: Particle, s: SMCSettings, i: int, stage: int, sweep: int):
    """One proposal for particle i.  Returns (move_index, proposal or None if the
    move is impossible or leaves the prior support)."""
    d0 = draws(s.seed, s.sounding, i, PURPOSE_MOVE, stage, sweep)[0]
    d1 = draws(s.seed, s.sounding, i, PURPOSE_VALUE, stage, sweep)[0]
    u = u01_from(np.concatenate([d0, d1]))
    move = min(int(u[0] * 6), 5)
    q = p.copy()
    if move == 0:  # conductive birth: depth U(0, zmax), log10 sigma from the prior
        if p.kappa >= s.kappa_max:
            return move, None
        z = s.zmax * u[1]
        v = s.phi_lo + (s.phi_hi - s.phi_lo) * u[2]
        j = sum(1 for zz in p.zc if zz < z)
        q.zc.insert(j, z)
        q.phic.insert(j, v)
        q.kappa += 1
    elif move == 1:  # conductive death: a uniformly chosen interface
        if p.kappa == 0:
            return move, None
        j = min(int(u[1] * p.kappa), p.kappa - 1)
        del q.zc[j]
        del q.phic[j]
        q.kappa -= 1
    elif move == 2:  # chargeable birth: depth U(0, zmax), m from the prior
        if p.lam >= s.lambda_max:
            return move, None
        z = s.zmax * u[1]
        v = u[2]
        j = sum(1 for zz in p.zm if zz < z)
        q.zm.insert(j, z)
        q.mv.insert(j, v)
        q.lam += 1
    elif move == 3:  # chargeable death
        if p.lam == 0:
            return move, None
        j = min(int(u[1] * p.lam), p.lam - 1)
        del q.zm[j]
        del q.mv[j]
        q.lam -= 1
    elif move == 4:  # depth move of one interface; keeps the order within its profile
        n_int = p.kappa + p.lam
        if n_int == 0:
            return move, None
        j = min(int(u[1] * n_int), n_int - 1)
        step = s.step_z * float(gauss_pair(d1[1], d1[2]))
        if j < p.kappa:
            arr, jj = q.zc, j
        else:
            arr, jj = q.zm, j - p.kappa
        z = arr[jj] + step
        lo = arr[jj - 1] if jj > 0 else 0.0
        hi = arr[jj + 1] if jj + 1 < len(arr) else s.zmax
        if not (lo < z < hi):
            return move, None
        arr[jj] = z
    else:  # component-wise Gaussian random walk
        n_comp = 1 + p.kappa + p.lam + 2
        j = min(int(u[1] * n_comp), n_comp - 1)
        g = float(gauss_pair(d1[1], d1[2]))
        if j == 0:
            q.phib = p.phib + s.step_phi * g
        elif j <= p.kappa:
            q.phic[j - 1] = p.phic[j - 1] + s.step_phi * g
        elif j <= p.kappa + p.lam:
            q.mv[j - 1 - p.kappa] = p.mv[j - 1 - p.kappa] + s.step_m * g
        elif j == p.kappa + p.lam + 1:
            if s.tau_log_prior:
                q.tau = 10.0 ** (math.log10(p.tau) + s.step_tau * g)
            else:
                q.tau = p.tau + s.step_tau * g
        else:
            q.c = p.c + s.step_c * g
        if not in_prior(q, s):
            return move, None
    return move, q


def accept_uniform(s: SMCSettings, i: int, stage: int, sweep: int):
    d = draws(s.seed, s.sounding, i, PURPOSE_ACCEPT, stage, sweep)[0]
    return float(u01_53(d[0], d[1]))


# ------------------------------------------------- Langevin (MALA) moves
PURPOSE_LANGEVIN_ACCEPT = 68
LANGEVIN_TARGET = 0.574          # optimal MALA acceptance rate (Roberts & Rosenthal 1998)
LANGEVIN_H_MIN, LANGEVIN_H_MAX = 1e-6, 10.0
PURPOSE_LANGEVIN0 = 72  # normal j: purpose 72 + j // 2, words 2 (j % 2) and 2 (j % 2) + 1


def theta_of(p: Particle, s: SMCSettings):
    """The continuous parameters of a particle in a fixed order:
    (phi_b, phi_c[0..kappa), z_c[0..kappa), z_m[0..lambda), m[0..lambda), tau, c),
    tau as log10 tau under the log-uniform prior (the random walk's coordinate)."""
    t = math.log10(p.tau) if s.tau_log_prior else p.tau
    return np.array([p.phib] + list(p.phic) + list(p.zc) + list(p.zm) + list(p.mv) + [t, p.c], dtype=np.float64)


def with_theta(p: Particle, s: SMCSettings, theta) -> Particle:
    k, l = p.kappa, p.lam
    th = [float(v) for v in theta]
    tau = 10.0 ** th[1 + 2 * k + 2 * l] if s.tau_log_prior else th[1 + 2 * k + 2 * l]
    return Particle(k, l, th[0], th[1 + k:1 + 2 * k], th[1:1 + k], th[1 + 2 * k:1 + 2 * k + l],
                    th[1 + 2 * k + l:1 + 2 * k + 2 * l], tau, th[2 + 2 * k + 2 * l])


def theta_scales(p: Particle, s: SMCSettings):
    """Per-component scale of the preconditioner: the random-walk step of the
    component's kind."""
    k, l = p.kappa, p.lam
    return np.array([s.step_phi] * (1 + k) + [s.step_z] * (k + l) + [s.step_m] * l + [s.step_tau, s.step_c])


def theta_in_support(p: Particle, s: SMCSettings) -> bool:
    """Uniform prior support with ordered interfaces in each profile."""
    if not in_prior(p, s):
        return False
    return all(a < b for a, b in zip(p.zc, p.zc[1:])) and all(a < b for a, b in zip(p.zm, p.zm[1:]))


def theta_grad_fd(parts, s: SMCSettings, loglik, step=1e-5):
    """d l / d theta by central differences of l(merge(theta)) with step
    step * max(|theta_j|, 1e-3) in each component.  Returns (l, [grad per particle])."""
    ll = np.asarray(loglik(parts), dtype=np.float64)
    grads = []
    for p in parts:
        th = theta_of(p, s)
        plus, minus, hs = [], [], []
        for j in range(len(th)):
            hj = step * max(abs(th[j]), 1e-3)
            a = th.copy()
            b = th.copy()
            a[j] += hj
            b[j] -= hj
            plus.append(with_theta(p, s, a))
            minus.append(with_theta(p, s, b))
            hs.append(hj)
        lp = np.asarray(loglik(plus), dtype=np.float64)
        lm = np.asarray(loglik(minus), dtype=np.float64)
        grads.append((lp - lm) / (2.0 * np.asarray(hs)))
    return ll, grads


def langevin_normals(s: SMCSettings, i: int, stage: int, sweep: int, d: int):
    out = np.zeros(d)
    for j in range(d):
        w = draws(s.seed, s.sounding, i, PURPOSE_LANGEVIN0 + j // 2, stage, sweep)[0]
        out[j] = float(gauss_pair(w[2 * (j % 2)], w[2 * (j % 2) + 1]))
    return out


def langevin_log_q(theta_to, theta_from, grad_from, scales, gamma, h):
    """log q(theta_to | theta_from) up to a constant for the preconditioned
    Langevin proposal N(theta + (h^2/2) D gamma grad, h^2 D), D = diag(scales^2)."""
    mean = theta_from + 0.5 * h * h * scales * scales * gamma * grad_from
    z = (theta_to - mean) / (h * scales)
    return -0.5 * float(np.sum(z * z))


def langevin_propose(p: Particle, grad, s: SMCSettings, i: int, stage: int, sweep: int, gamma: float, h=None):
    """Returns (proposal or None outside the support, log q(proposal | p))."""
    th = theta_of(p, s)
    sc = theta_scales(p, s)
    h = s.langevin_h if h is None else h
    xi = langevin_normals(s, i, stage, sweep, len(th))
    th_new = th + 0.5 * h * h * sc * sc * gamma * np.asarray(grad) + h * sc * xi
    q = with_theta(p, s, th_new)
    if not theta_in_support(q, s):
        return None, 0.0
    return q, -0.5 * float(np.sum(xi * xi))


def langevin_accept_uniform(s: SMCSettings, i: int, stage: int, sweep: int):
    d = draws(s.seed, s.sounding, i, PURPOSE_LANGEVIN_ACCEPT, stage, sweep)[0]
    return float(u01_53(d[0], d[1]))


def langevin_step_update(h, accepted, proposed):
    """Between stages: h <- h exp(2 (rate - LANGEVIN_TARGET)), clamped."""
    rate = accepted / proposed if proposed > 0 else LANGEVIN_TARGET
    return min(max(h * math.exp(2.0 * (rate - LANGEVIN_TARGET)), LANGEVIN_H_MIN), LANGEVIN_H_MAX)


def langevin_sweeps(parts, s: SMCSettings, stage: int, gamma: float, grad_fn, n_sweeps: int, h=None):
    """n_sweeps MALA sweeps over every particle at gamma_t with step h (default
    s.langevin_h).  grad_fn maps a list of particles to (l, [d l / d theta]).
    Returns (particles, l, accepted, proposed)."""
    h = s.langevin_h if h is None else h
    ll, grads = grad_fn(parts)
    parts = list(parts)
    grads = list(grads)
    ll = np.array(ll, dtype=np.float64)
    acc = 0
    for sweep in range(n_sweeps):
        props = [langevin_propose(parts[i], grads[i], s, i, stage, sweep, gamma, h) for i in range(len(parts))]
        live = [i for i in range(len(parts)) if props[i][0] is not None]
        if live:
            ll_new, g_new = grad_fn([props[i][0] for i in live])
        for n, i in enumerate(live):
            q, lq_fwd = props[i]
            lq_rev = langevin_log_q(theta_of(parts[i], s), theta_of(q, s), g_new[n], theta_scales(q, s), gamma, h)
            u = langevin_accept_uniform(s, i, stage, sweep)
            if math.log(u) < gamma * (ll_new[n] - ll[i]) + lq_rev - lq_fwd:
                parts[i] = q
                ll[i] = ll_new[n]
                grads[i] = g_new[n]
                acc += 1
    return parts, ll, acc, n_sweeps * len(parts)


# ------------------------------------------------------------------- driver
@dataclass
class SMCResult:
    gammas: list = field(default_factory=list)
    log_z: np.ndarray = None
    counts: np.ndarray = None
    particles: list = None
    ll: np.ndarray = None
    accept: np.ndarray = None
    proposed: np.ndarray = None
    sweeps: list = field(default_factory=list)
    langevin_accept: int = 0
    langevin_proposed: int = 0
    langevin_h: list = field(default_factory=list)
    pca_scales: list = field(default_factory=list)


class ForwardLik:
    """Log-likelihood of merged particles through the oracle forward model."""

    def __init__(self, system, y_obs, eps_an, eps_mn, lmax, mode=None, nthreads=None):
        import oracle as O
        self.O = O
        self.nthreads = nthreads
        self.system = dict(system)
        if self.system.get("T") is None:
            self.system["T"] = O.tmatrix(self.system["freqs"], self.system["times"])
        self.y_obs = np.asarray(y_obs, dtype=np.float64)
        self.eps_an = eps_an
        self.eps_mn = eps_mn
        self.lmax = lmax
        self.mode = O.HANKEL_RULE if mode is None else mode

    def __call__(self, parts):
        if not parts:
            return np.zeros(0)
        mb = merged_batch(parts, self.lmax)
        y = self.O.forward(mb, self.system, mode=self.mode, nthreads=self.nthreads)
        return self.O.loglik(y, self.y_obs, self.eps_an, self.eps_mn)


def run(s: SMCSettings, loglik, max_stages=500, prior=sample_prior, proposer=propose, grad_fn=None):
    """Algorithm 1: initialise from the prior, then reweight / resample /
    mutate until gamma = 1.  `loglik` maps a list of particles to their
    log-likelihoods; with s.n_langevin > 0 every stage ends with that many
    Langevin sweeps driven by grad_fn (default: theta_grad_fd on loglik)."""
    N = s.n_particles
    parts = [prior(s, i) for i in range(N)]
    ll = np.asarray(loglik(parts), dtype=np.float64)
    gamma = 0.0
    log_z = np.zeros(s.n_models)
    res = SMCResult()
    acc = np.zeros(6)
    prop = np.zeros(6)
    p_min = 0.0
    h_lang = s.langevin_h
    pca_scale = {}
    history = [(0, [p.copy() for p in parts], ll.copy())] if s.recycle > 0 else []
    gamma_hist = [0.0]
    logz_hist = [np.zeros(s.n_models)]
    for stage in range(1, max_stages + 1):
        model = np.array([p.model(s) for p in parts])
        dg, done, inc, W = reweight(ll, model, s.n_models, gamma, s.alpha, s.bisect_iters)
        gamma = 1.0 if done else gamma + dg
        log_z += inc
        res.gammas.append(gamma)
        anc = resample_systematic(W, model, s.n_models, resample_uniforms(s, stage))
        parts = [parts[a].copy() for a in anc]
        ll = ll[anc].copy()
        gamma_hist.append(gamma)
        logz_hist.append(log_z.copy())
        if s.recycle > 0:
            history = (history + [(stage, [p.copy() for p in parts], ll.copy())])[-s.recycle:]
        R = s.n_sweeps if s.n_sweeps > 0 else (s.r_max if stage == 1 else sweeps_needed(p_min, s.c_mut, s.r_max))
        res.sweeps.append(R)
        if s.adaptive:
            fits = (fit_model_gaussians_recycled(history, s, stage, gamma_hist, logz_hist) if s.recycle > 0
                    else fit_model_gaussians(parts, s))
            pca_scale = pca_bisect_scales(parts, ll, fits, s, stage, gamma, loglik, pca_scale)
            res.pca_scales.append(dict(pca_scale))
            proposer = (lambda p_, s_, i_, st_, sw_: propose_adaptive(p_, s_, i_, st_, sw_, fits, pca_scale))
        acc_stage = np.zeros(6)
        prop_stage = np.zeros(6)
        for sweep in range(R):
            props = [proposer(parts[i], s, i, stage, sweep) for i in range(N)]
            live = [i for i in range(N) if props[i][1] is not None]
            ll_new = np.full(N, -np.inf)
            if live:
                ll_new[live] = loglik([props[i][1] for i in live])
            for i in range(N):
                mv, q = props[i][:2]
                log_f = props[i][2] if len(props[i]) > 2 else 0.0
                prop_stage[mv] += 1
                if q is None:
                    continue
                u = accept_uniform(s, i, stage, sweep)
                if math.log(u) < gamma * (ll_new[i] - ll[i]) + log_f:
                    parts[i] = q
                    ll[i] = ll_new[i]
                    acc_stage[mv] += 1
        if s.n_langevin > 0:
            gfn = grad_fn if grad_fn is not None else (lambda ps: theta_grad_fd(ps, s, loglik))
            parts, ll, la, lp = langevin_sweeps(parts, s, stage, gamma, gfn, s.n_langevin, h_lang)
            res.langevin_accept += la
            res.langevin_proposed += lp
            res.langevin_h.append(h_lang)
            if s.langevin_adapt:
                h_lang = langevin_step_update(h_lang, la, lp)
        acc += acc_stage
        prop += prop_stage
        rates = np.where(prop_stage > 0, acc_stage / np.maximum(prop_stage, 1), 1.0)
        p_min = float(np.min(rates))
        if gamma >= 1.0:
            break
    model = np.array([p.model(s) for p in parts])
    res.log_z = log_z
    res.counts = np.bincount(model, minlength=s.n_models)
    res.particles = parts
    res.ll = ll
    res.accept = acc
    res.proposed = prop
    return res


def grouped_bayes_factor(post, prior, chargeable):
    """The BFIPD statistic of Section 2.3.3, written out as the paper defines
    it: with M_lambda the chargeable models and M_kappa the others,

        B = |M_kappa| sum_{k in M_lambda} post_k / prior_k
            / ( |M_lambda| sum_{k in M_kappa} post_k / prior_k ).

    post: estimated posterior model probabilities pi(k|y); prior: p(k) > 0;
    chargeable: boolean per model.  Returns log B (+inf when no non-chargeable
    model has posterior mass, -inf when no chargeable one has)."""
    post = np.asarray(post, dtype=np.float64)
    prior = np.asarray(prior, dtype=np.float64)
    ip = np.asarray(chargeable, dtype=bool)
    n_ip, n_non = int(ip.sum()), int((~ip).sum())
    s_ip = float(np.sum(post[ip] / prior[ip]))
    s_non = float(np.sum(post[~ip] / prior[~ip]))
    if s_non == 0.0:
        return math.inf
    if s_ip == 0.0:
        return -math.inf
    return math.log(n_non * s_ip) - math.log(n_ip * s_non)


def model_odds(counts, kappa_max, lambda_max, prior=None):
    """pi(k|y) = N_k / N (Section 3.2.1) and log BFIPD (Section 2.3.3) over the
    (kappa_max + 1) x (lambda_max + 1) grid of decoupled models, k = kappa
    (lambda_max + 1) + lambda, chargeable when lambda >= 1.  prior: p(k); None
    is the sampler's prior, uniform on kappa and on lambda, under which B
    reduces to the posterior odds over the prior odds, N_IP / (lambda_max N_nonIP)."""
    counts = np.asarray(counts, dtype=np.float64)
    post = counts / counts.sum()
    M = (kappa_max + 1) * (lambda_max + 1)
    if prior is None:
        prior = np.full(M, 1.0 / M)
    chargeable = (np.arange(M) % (lambda_max + 1)) >= 1
    return post, grouped_bayes_factor(post, prior, chargeable)


# ------------------------------------------- adaptive within-model proposal
# Section 3.2 ("Transdimensional and within-model adaptive proposals"): a
# Gaussian N(mu_k, Sigma_k) fitted to the particles of each model k, the
# eigen-decomposition Sigma_k = U Lambda U^T, a component-wise random walk
# along a uniformly chosen principal direction U_r with standard deviation
# a_k sqrt(Lambda_r), and the scale a_k chosen per stage by bisection on trial
# proposals so that their mean acceptance probability is pca_target.
PURPOSE_PCA_TRIAL = 69
PCA_LOG_SPAN = 3.0   # bisection bracket: log a within +-3 of the previous stage's


def fit_model_gaussians(parts, s: SMCSettings):
    """{model k: (mu, U, Lam)} over the (equally weighted) particles of each
    model with at least two particles; Sigma is the biased sample covariance
    plus (pca_ridge * step_j)^2 on the diagonal."""
    out = {}
    by_model = {}
    for p in parts:
        by_model.setdefault(p.model(s), []).append(theta_of(p, s))
    for k, th in by_model.items():
        if len(th) < 2:
            continue
        X = np.array(th)
        mu = X.mean(axis=0)
        C = (X - mu).T @ (X - mu) / len(th)
        sc = theta_scales(parts[[q.model(s) for q in parts].index(k)], s)
        C = C + np.diag((s.pca_ridge * sc) ** 2)
        lam, U = np.linalg.eigh(C)
        out[k] = (mu, U, np.maximum(lam, 0.0))
    return out


def pca_step(p: Particle, fit, a, s: SMCSettings, u_comp, xi):
    """theta' = theta + a sqrt(Lambda_r) xi U_r with r = floor(u_comp d);
    None outside the prior support or the interface order."""
    _, U, lam = fit
    d = len(lam)
    r = min(int(u_comp * d), d - 1)
    th = theta_of(p, s) + a * math.sqrt(lam[r]) * xi * U[:, r]
    q = with_theta(p, s, th)
    return q if theta_in_support(q, s) else None


def pca_trial_draws(s: SMCSettings, i: int, stage: int):
    w = draws(s.seed, s.sounding, i, PURPOSE_PCA_TRIAL, stage, 0)[0]
    return float(u01_from(w[0])), float(gauss_pair(w[1], w[2]))


def pca_bisect_scales(parts, ll, fits, s: SMCSettings, stage: int, gamma: float, loglik, a_prev):
    """Per model: bisection on log a in [log a_prev - 3, log a_prev + 3] with
    the same trial draws at every step; the mean over the model's particles of
    min(1, (L'/L)^gamma) (0 outside the support) is compared with pca_target.
    Returns {k: a}."""
    lo = {k: math.log(a_prev.get(k, 1.0)) - PCA_LOG_SPAN for k in fits}
    hi = {k: math.log(a_prev.get(k, 1.0)) + PCA_LOG_SPAN for k in fits}
    trial = [pca_trial_draws(s, i, stage) for i in range(len(parts))]
    for _ in range(s.pca_bisect_iters):
        mid = {k: 0.5 * (lo[k] + hi[k]) for k in fits}
        props = [pca_step(p, fits[p.model(s)], math.exp(mid[p.model(s)]), s, *trial[i])
                 if p.model(s) in fits else None for i, p in enumerate(parts)]
        live = [i for i in range(len(parts)) if props[i] is not None]
        ll_new = np.full(len(parts), -np.inf)
        if live:
            ll_new[live] = loglik([props[i] for i in live])
        acc = {k: [] for k in fits}
        for i, p in enumerate(parts):
            k = p.model(s)
            if k in fits:
                acc[k].append(0.0 if props[i] is None else min(1.0, math.exp(min(0.0, gamma * (ll_new[i] - ll[i])))))
        for k in fits:
            if np.mean(acc[k]) > s.pca_target:
                lo[k] = mid[k]
            else:
                hi[k] = mid[k]
    return {k: math.exp(0.5 * (lo[k] + hi[k])) for k in fits}


def recycle_log_weights(ll, gammas, log_z_k, t):
    """Deterministic-mixture weights of recycled particles for model k at
    stage t (Section 3.2, "Overcoming particle impoverishment"):
      log nu = gamma_t l - log( (1/(t+1)) sum_{l=0}^{t} exp(gamma_l l - log Z_{l,k}) ),
    the prior cancelling between numerator and denominator.  The printed
    normaliser 1/t over t + 1 terms is read as 1/(t+1).  ll: log-likelihoods
    of the particles (from any stage s <= t); gammas[l], log_z_k[l] for l = 0..t."""
    ll = np.asarray(ll, dtype=np.float64)[:, None]
    g = np.asarray(gammas[:t + 1], dtype=np.float64)[None, :]
    lz = np.asarray(log_z_k[:t + 1], dtype=np.float64)[None, :]
    a = g * ll - lz
    m = a.max(axis=1, keepdims=True)
    lden = m[:, 0] + np.log(np.exp(a - m).sum(axis=1)) - math.log(t + 1)
    return g[0, -1] * ll[:, 0] - lden


def fit_model_gaussians_recycled(history, s: SMCSettings, t: int, gammas, log_z):
    """As fit_model_gaussians, on the particles of every stored stage (history:
    list of (stage, particles, ll), the last `recycle` stages up to t) with the
    normalised recycling weights of recycle_log_weights per model; a model is
    fitted when its current stage holds at least two particles."""
    out = {}
    cur = history[-1][1]
    counts = {}
    for p in cur:
        counts[p.model(s)] = counts.get(p.model(s), 0) + 1
    for k, n in counts.items():
        if n < 2:
            continue
        th, ll = [], []
        for _, parts, lls in history:
            for p, l in zip(parts, lls):
                if p.model(s) == k:
                    th.append(theta_of(p, s))
                    ll.append(l)
        lw = recycle_log_weights(ll, gammas, [z[k] for z in log_z], t)
        w = np.exp(lw - lw.max())
        w /= w.sum()
        X = np.array(th)
        mu = w @ X
        C = (X - mu).T @ ((X - mu) * w[:, None])
        sc = theta_scales(next(p for p in cur if p.model(s) == k), s)
        C = C + np.diag((s.pca_ridge * sc) ** 2)
        lam, U = np.linalg.eigh(C)
        out[k] = (mu, U, np.maximum(lam, 0.0))
    return out


# ----------------------------------------- ZCA-coloured birth/death (App. F)
# Birth k -> k+1 at depth u_d ~ U(0, zmax): the new layer's value starts as a
# copy of the value of the layer it splits (0 for a chargeable layer inserted
# above every chargeable interface, whose background m = 0 is fixed); then
# every component but the new depth moves by u Sigma^(1/2)[i, j], u ~ N(0, 1),
# with Sigma^(1/2) = U Lambda^(1/2) U^T the ZCA root of model k+1's fitted
# covariance and i the new value's component.  The Jacobian of
# (theta_k, u_d, u) -> theta_{k+1} is Sigma^(1/2)[i, j_new] - Sigma^(1/2)[i, h]
# (h the copied value; 0 without one).  With uniform priors, the uniform
# depth draw, uniform move selection and a uniformly chosen death interface,
# the prior and proposal densities leave the birth acceptance
#   min(1, (L'/L)^gamma |J| / (width phi(u))),
# width the prior width of the new value (phi_hi - phi_lo, or 1 for m), and
# the death the reciprocal with u solved from the two values.
def zca_root(fit):
    _, U, lam = fit
    return (U * np.sqrt(np.maximum(lam, 0.0))) @ U.T


def _profile_offsets(k, l):
    """Component offsets in theta of (phi_c, z_c, z_m, m) for kappa = k, lambda = l."""
    return 1, 1 + k, 1 + 2 * k, 1 + 2 * k + l


def zca_birth(p: Particle, s: SMCSettings, fit_next, cond: bool, u_depth: float, u: float):
    """Returns (proposal or None outside the support, log of the factor that
    multiplies (L'/L)^gamma)."""
    z = s.zmax * u_depth
    q = p.copy()
    if cond:
        j = sum(1 for v in p.zc if v < z)
        src = p.phib if j == 0 else p.phic[j - 1]
        q.zc.insert(j, z)
        q.phic.insert(j, src)
        q.kappa += 1
        o_val, o_dep, _, _ = _profile_offsets(q.kappa, q.lam)
        width = s.phi_hi - s.phi_lo
        j_new, h = o_val + j, (0 if j == 0 else o_val + j - 1)
    else:
        j = sum(1 for v in p.zm if v < z)
        src = 0.0 if j == 0 else p.mv[j - 1]
        q.zm.insert(j, z)
        q.mv.insert(j, src)
        q.lam += 1
        _, _, o_dep, o_val = _profile_offsets(q.kappa, q.lam)
        width = 1.0
        j_new, h = o_val + j, (None if j == 0 else o_val + j - 1)
    j_z = o_dep + j
    Z = zca_root(fit_next)
    th = theta_of(q, s)
    for jj in range(len(th)):
        if jj != j_z:
            th[jj] += Z[j_new, jj] * u
    jac = Z[j_new, j_new] - (Z[j_new, h] if h is not None else 0.0)
    log_f = math.log(abs(jac)) - math.log(width) - (-0.5 * u * u - 0.5 * math.log(2 * math.pi))
    q = with_theta(q, s, th)
    return (q if theta_in_support(q, s) else None), log_f


def zca_death(p: Particle, s: SMCSettings, fit_own, cond: bool, u_choice: float):
    n = p.kappa if cond else p.lam
    j = min(int(u_choice * n), n - 1)
    o_phic, o_zc, o_zm, o_mv = _profile_offsets(p.kappa, p.lam)
    if cond:
        j_new, j_z, h, width = o_phic + j, o_zc + j, (0 if j == 0 else o_phic + j - 1), s.phi_hi - s.phi_lo
    else:
        j_new, j_z, h, width = o_mv + j, o_zm + j, (None if j == 0 else o_mv + j - 1), 1.0
    Z = zca_root(fit_own)
    th = theta_of(p, s)
    jac = Z[j_new, j_new] - (Z[j_new, h] if h is not None else 0.0)
    u = (th[j_new] - (th[h] if h is not None else 0.0)) / jac
    back = th.copy()
    for jj in range(len(th)):
        if jj not in (j_z, j_new):
            back[jj] -= Z[j_new, jj] * u
    keep = [jj for jj in range(len(th)) if jj not in (j_z, j_new)]
    q = p.copy()
    if cond:
        del q.zc[j]
        del q.phic[j]
        q.kappa -= 1
    else:
        del q.zm[j]
        del q.mv[j]
        q.lam -= 1
    q = with_theta(q, s, back[keep])
    log_f = math.log(width) + (-0.5 * u * u - 0.5 * math.log(2 * math.pi)) - math.log(abs(jac))
    return (q if theta_in_support(q, s) else None), log_f


def propose_adaptive(p: Particle, s: SMCSettings, i: int, stage: int, sweep: int, fits, scales):
    """The move set of propose() with the perturb move replaced by the
    adaptive principal-direction random walk (models without a fit keep the
    fixed-scale one)."""
    d0 = draws(s.seed, s.sounding, i, PURPOSE_MOVE, stage, sweep)[0]
    move = min(int(u01_from(d0[0]) * 6), 5)
    k = p.model(s)
    if s.zca > 0 and move <= 3:
        # a state-independent choice between the ZCA-coloured and the
        # prior-drawn pair keeps the mixture reversible
        d1 = draws(s.seed, s.sounding, i, PURPOSE_VALUE, stage, sweep)[0]
        use = float(u01_from(d1[3])) < s.zca
        cond = move in (0, 1)
        L1 = s.lambda_max + 1
        if use and move in (0, 2):
            n, nmax = (p.kappa, s.kappa_max) if cond else (p.lam, s.lambda_max)
            k_next = k + (L1 if cond else 1)
            if n < nmax and k_next in fits:
                q, lf = zca_birth(p, s, fits[k_next], cond, float(u01_from(d0[1])), float(gauss_pair(d1[1], d1[2])))
                return move, q, lf
        elif use:
            n = p.kappa if cond else p.lam
            if n > 0 and k in fits:
                q, lf = zca_death(p, s, fits[k], cond, float(u01_from(d0[1])))
                return move, q, lf
    if move != 5 or k not in fits:
        return propose(p, s, i, stage, sweep)
    d1 = draws(s.seed, s.sounding, i, PURPOSE_VALUE, stage, sweep)[0]
    return move, pca_step(p, fits[k], scales[k], s, float(u01_from(d0[1])), float(gauss_pair(d1[1], d1[2])))


# ------------------------------------------------ posterior predictive (PPD)
def ppd_summary(y_model, y_obs, eps_an, eps_mn):
    """Per-gate summaries of the posterior predictive distribution
    p(y~ | y) = int p(y~ | theta) pi(theta | y) d theta (the goodness of fit
    of Section 4.1) over equally weighted posterior particles with predictions
    y_model [N, G] and Gaussian noise of variance v = eps_an^2 + (eps_mn yhat)^2:
      mean_g = (1/N) sum_i yhat_ig,
      var_g  = (1/N) sum_i [ v_ig + (yhat_ig - mean_g)^2 ]   (law of total variance),
      z_g    = (y_g - mean_g) / sqrt(var_g)  (the data standardised to the PPD).
    Returns (mean [G], var [G], z [G])."""
    y_model = np.asarray(y_model, dtype=np.float64)
    N = y_model.shape[0]
    mean = y_model.sum(axis=0) / N
    v = np.asarray(eps_an, dtype=np.float64) ** 2 + (eps_mn * y_model) ** 2
    var = (v + (y_model - mean) ** 2).sum(axis=0) / N
    z = (np.asarray(y_obs, dtype=np.float64) - mean) / np.sqrt(var)
    return mean, var, z
