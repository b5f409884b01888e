"""Pins of the oracle's Langevin (MALA) move and of its particle-space
gradient, on the CPU.

* invariance: on a Gaussian target with known mean and variance, chains of the
  oracle's MALA kernel keep the target's first two moments (a dropped
  proposal-density ratio halves the pooled variance at these steps; a
  mis-signed drift gradient stops the chains);
* SMC with Langevin sweeps still reproduces the closed-form evidence of the
  toy model of the random-walk tests;
* the central-difference gradient in the particle coordinates equals the
  chain rule applied to the merged-layer gradient (two independent routes:
  perturbing the particle, or perturbing the merged layers and mapping back
  through the direct sum of Section 2.1)."""
import math

import numpy as np
import pytest
from scipy.stats import norm

import oracle as O
import oracle.rjsmc as R
from paper_2109_00661_gb300 import inputs as I

MU = np.array([-2.0, -1.0, 100.0, 200.0, 0.4, 0.5, 0.5])
SD = np.array([0.1, 0.1, 5.0, 5.0, 0.05, 0.05, 0.05])


def gauss_target(s):
    def loglik(parts):
        th = np.array([R.theta_of(p, s) for p in parts])
        return -0.5 * np.sum(((th - MU) / SD) ** 2, axis=1)

    def grad_fn(parts):
        th = np.array([R.theta_of(p, s) for p in parts])
        return loglik(parts), list(-(th - MU) / SD ** 2)

    return loglik, grad_fn


def test_theta_roundtrip():
    s = R.SMCSettings(kappa_max=3, lambda_max=4)
    for i in range(20):
        p = R.sample_prior(s, i)
        q = R.with_theta(p, s, R.theta_of(p, s))
        assert q == p


@pytest.mark.parametrize("h", [0.7, 1.4])
def test_mala_keeps_gaussian_target_invariant(h):
    """kappa = lambda = 1 (7 parameters) started in the target: after 400
    sweeps of 24 chains the pooled mean and variance match the target."""
    s = R.SMCSettings(kappa_max=1, lambda_max=1, step_phi=0.1, step_z=5.0, step_m=0.05, step_tau=0.05,
                      step_c=0.05, langevin_h=h, seed=3)
    loglik, grad_fn = gauss_target(s)
    rng = np.random.default_rng(0)
    parts = []
    for _ in range(24):
        th = MU + SD * rng.standard_normal(7)
        parts.append(R.with_theta(R.Particle(1, 1, 0.0, [0.0], [0.0], [0.0], [0.0], 0.5, 0.5), s, th))
    samples = []
    acc_total = 0
    for stage in range(1, 401):
        parts, _, acc, _ = R.langevin_sweeps(parts, s, stage, 1.0, grad_fn, 1)
        acc_total += acc
        if stage > 20:
            samples.extend(R.theta_of(p, s) for p in parts)
    x = (np.array(samples) - MU) / SD
    rate = acc_total / (400 * 24)
    assert 0.2 < rate < 0.99, rate
    assert np.all(np.abs(x.mean(axis=0)) < 0.12), x.mean(axis=0)
    assert np.all(np.abs(x.var(axis=0) - 1.0) < 0.15), x.var(axis=0)


@pytest.mark.slow
def test_smc_with_langevin_keeps_toy_evidence():
    """The toy of the random-walk tests (phi_b, tau, c with Gaussian
    likelihoods): SMC with two Langevin sweeps per stage reproduces the
    closed-form log evidence."""
    Y3 = np.array([0.5, 0.3, 0.6])
    SIG = 0.1

    def loglik(parts):
        th = np.array([[p.phib, p.tau, p.c] for p in parts])
        return np.sum(norm.logpdf(Y3[None, :], th, SIG), axis=1)

    def grad_fn(parts):
        th = np.array([[p.phib, p.tau, p.c] for p in parts])
        return loglik(parts), list((Y3[None, :] - th) / SIG ** 2)

    lo = np.array([-4.0, 0.0, 0.0])
    hi = np.array([2.0, 1.0, 1.0])
    log_z = float(np.sum(np.log((norm.cdf((hi - Y3) / SIG) - norm.cdf((lo - Y3) / SIG)) / (hi - lo))))
    est = []
    acc = prop = 0
    for seed in range(10):
        s = R.SMCSettings(n_particles=200, kappa_max=0, lambda_max=0, n_sweeps=3, n_langevin=2, langevin_h=0.8,
                          seed=seed)
        res = R.run(s, loglik, grad_fn=grad_fn)
        assert res.gammas[-1] == 1.0
        est.append(res.log_z[0])
        acc += res.langevin_accept
        prop += res.langevin_proposed
    est = np.array(est)
    se = est.std(ddof=1) / math.sqrt(len(est))
    assert abs(est.mean() - log_z) < 3 * se + 0.03
    assert acc / prop > 0.2


def chain_rule(p, s, g_merged):
    """d l / d theta from the merged-layer gradient [lmax, 5] of
    (log10 sigma, log10 h, m, log10 tau, c), following the direct sum."""
    k, l = p.kappa, p.lam
    src = sorted([(z, 0, j) for j, z in enumerate(p.zc)] + [(z, 1, j) for j, z in enumerate(p.zm)])
    L = len(src) + 1
    z = [v[0] for v in src]
    g = np.zeros(3 + 2 * k + 2 * l)
    dl_dh = np.zeros(L)
    for n in range(L):
        top = 0.0 if n == 0 else z[n - 1]
        ic = sum(1 for v in p.zc if v <= top) if n > 0 else 0
        jm = sum(1 for v in p.zm if v <= top) if n > 0 else 0
        g[0 if ic == 0 else ic] += g_merged[n, 0]
        if jm > 0:
            g[1 + 2 * k + l + jm - 1] += g_merged[n, 2]
        if n < L - 1:
            dl_dh[n] = g_merged[n, 1] / ((z[n] - top) * math.log(10.0))
    for n, (_, kind, j) in enumerate(src):
        d = dl_dh[n] - dl_dh[n + 1]  # h_n grows, h_{n+1} shrinks (basement has none)
        g[(1 + k + j) if kind == 0 else (1 + 2 * k + j)] += d
    dlt = float(np.sum(g_merged[:L, 3]))
    g[1 + 2 * k + 2 * l] = dlt if s.tau_log_prior else dlt / (p.tau * math.log(10.0))
    g[2 + 2 * k + 2 * l] = float(np.sum(g_merged[:L, 4]))
    return g


@pytest.mark.parametrize("tau_log_prior", [False, True])
def test_theta_gradient_matches_chain_rule_of_merged_gradient(tau_log_prior):
    name = "sounding-g20-f40-k120"
    sysd = I.oracle_system(name)
    sysd["T"] = O.tmatrix(sysd["freqs"], sysd["times"])
    y_obs = I.noisy(O.forward(I.truth_3layer(), sysd, mode=O.HANKEL_RULE)[0], seed=0)
    s = R.SMCSettings(kappa_max=2, lambda_max=2, tau_log_prior=tau_log_prior)
    lmax = s.kappa_max + s.lambda_max + 1
    f = R.ForwardLik(sysd, y_obs, I.EPS_AN, I.EPS_MN, lmax)
    parts = [R.Particle(2, 1, -2.0, [20.0, 55.0], [-1.1, -2.2], [35.0], [0.3], 1e-3, 0.5),
             R.Particle(1, 2, -1.8, [40.0], [-1.0], [15.0, 70.0], [0.2, 0.4], 2e-3, 0.6),
             R.Particle(0, 1, -2.0, [], [], [25.0], [0.35], 5e-4, 0.7)]
    ll, g_theta = R.theta_grad_fd(parts, s, f)
    mb = R.merged_batch(parts, lmax)
    ll_m, g_m = O.loglik_grad_fd(mb, sysd, y_obs, I.EPS_AN, I.EPS_MN)
    assert np.allclose(ll, ll_m, rtol=1e-12)
    for i, p in enumerate(parts):
        ref = chain_rule(p, s, g_m[i])
        err = np.abs(g_theta[i] - ref) / np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))
        assert err.max() < 1e-4, (i, g_theta[i], ref)
