"""Langevin (MALA) moves of the CUDA sampler against the oracle, through the
C ABI:

* the particle-space gradient (adjoint kernel + chain rule through the direct
  sum) against central differences of the FP64 oracle in the particle's own
  coordinates;
* the proposal arithmetic: given the same state, gradient and Philox stream,
  the GPU's proposals equal the oracle's to float32 rounding, with the same
  support decisions;
* the Metropolis-Hastings test: every GPU accept / reject decision is the
  oracle formula's on the GPU's own likelihoods and gradients, and agrees with
  the FP64 oracle's own inputs wherever the margin exceeds their measured
  difference;
* statistics: P(IP) with Langevin sweeps agrees with the random-walk-only
  sampler over independent seeds."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import rjsmc as R
from paper_2109_00661_gb300 import inputs as I
from parity_util import oracle_system

pytestmark = pytest.mark.gpu

NAME = "sounding-g20-f40-k120"
KS = 10
G_PHIB, G_PHIC, G_ZC, G_ZM, G_MV, G_TAU, G_C = 0, 1, 1 + KS, 1 + 2 * KS, 1 + 3 * KS, 1 + 4 * KS, 2 + 4 * KS


@pytest.fixture(scope="module")
def env():
    import paper_2109_00661_gb300 as L
    from paper_2109_00661_gb300 import smc as S
    gsys = L.System(**I.system_kwargs(NAME))
    s = oracle_system(NAME)
    data = I.noisy(O.forward(I.truth_3layer(), s, mode=O.HANKEL_RULE)[0], seed=0)
    return S, gsys, s, data


def settings(**kw):
    base = dict(n_particles=24, kappa_max=2, lambda_max=2, n_sweeps=0, seed=5)
    base.update(kw)
    return R.SMCSettings(**base)


def gpu_smc(S, gsys, data, st):
    return S.SMC(gsys, data, I.EPS_AN, I.EPS_MN, n_particles=st.n_particles, kappa_max=st.kappa_max,
                 lambda_max=st.lambda_max, zmax=st.zmax, seed=st.seed, langevin_h=st.langevin_h,
                 n_langevin=st.n_langevin, tau_log_prior=int(st.tau_log_prior))


def near_truth_particles(N, seed, st):
    """Particles near the three-layer truth (conductive interfaces and
    chargeable layers within 10..80 m), every value already a float32."""
    rng = np.random.default_rng(seed)
    f = lambda v: float(np.float32(v))
    out = []
    for _ in range(N):
        k = int(rng.integers(1, st.kappa_max + 1))
        l = int(rng.integers(0, st.lambda_max + 1))
        zc = sorted(f(v) for v in rng.uniform(10.0, 80.0, k))
        zm = sorted(f(v) for v in rng.uniform(10.0, 80.0, l))
        tau = f(10 ** rng.uniform(-3.5, -2.5))
        out.append(R.Particle(k, l, f(rng.uniform(-2.2, -1.8)), zc, [f(v) for v in rng.uniform(-2.3, -0.8, k)], zm,
                              [f(v) for v in rng.uniform(0.05, 0.5, l)], tau, f(rng.uniform(0.3, 0.9))))
    return out


def to_host(S, parts):
    h = S.Particles(len(parts))
    for i, p in enumerate(parts):
        h.kappa[i], h.lam[i] = p.kappa, p.lam
        h.phib[i], h.tau[i], h.c[i] = p.phib, p.tau, p.c
        h.zc[i, :p.kappa] = p.zc
        h.phic[i, :p.kappa] = p.phic
        h.zm[i, :p.lam] = p.zm
        h.mv[i, :p.lam] = p.mv
    return h


def to_oracle(h, i):
    k, l = int(h.kappa[i]), int(h.lam[i])
    f = lambda v: float(np.float64(v))
    return R.Particle(k, l, f(h.phib[i]), [f(v) for v in h.zc[i, :k]], [f(v) for v in h.phic[i, :k]],
                      [f(v) for v in h.zm[i, :l]], [f(v) for v in h.mv[i, :l]], f(h.tau[i]), f(h.c[i]))


def theta_slots(k, l):
    return ([G_PHIB] + [G_PHIC + j for j in range(k)] + [G_ZC + j for j in range(k)] + [G_ZM + j for j in range(l)]
            + [G_MV + j for j in range(l)] + [G_TAU, G_C])


def gpu_theta_grad(g, p):
    return g[theta_slots(p.kappa, p.lam)].astype(np.float64)


@pytest.mark.parametrize("tau_log_prior", [False, True])
def test_particle_gradient_matches_oracle_fd(env, tau_log_prior):
    S, gsys, s, data = env
    st = settings(n_particles=16, tau_log_prior=tau_log_prior)
    parts = near_truth_particles(st.n_particles, seed=1, st=st)
    sm = gpu_smc(S, gsys, data, st)
    sm.set_particles(to_host(S, parts))
    g = sm.grad_current()
    lik = R.ForwardLik(s, data, I.EPS_AN, I.EPS_MN, st.kappa_max + st.lambda_max + 1)
    _, g_ref = R.theta_grad_fd(parts, st, lik)
    worst = 0.0
    for i, p in enumerate(parts):
        got = gpu_theta_grad(g[i], p)
        ref = g_ref[i]
        ne = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        ce = np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-2 * np.max(np.abs(ref))))
        worst = max(worst, ne)
        assert ne <= 1e-3 and ce <= 5e-3, (i, got, ref)
        # unused slots are zero
        mask = np.ones(g.shape[1], dtype=bool)
        mask[theta_slots(p.kappa, p.lam)] = False
        assert np.all(g[i][mask] == 0.0)
    print(f"\nparticle gradient: worst relative norm error {worst:.2e}")


@pytest.mark.parametrize("tau_log_prior", [False, True])
def test_langevin_proposals_match_oracle(env, tau_log_prior):
    S, gsys, s, data = env
    st = settings(n_particles=64, tau_log_prior=tau_log_prior, langevin_h=0.02)
    parts = near_truth_particles(st.n_particles, seed=2, st=st)
    gamma, stage, sweep = 0.35, 4, 3
    sm = gpu_smc(S, gsys, data, st)
    sm.set_particles(to_host(S, parts), gamma=np.array([gamma]), stage=stage)
    g = sm.grad_current()
    sm.langevin_propose(stage, sweep)
    prop = sm.get_particles(1)
    n_valid = 0
    for i, p in enumerate(parts):
        q, _ = R.langevin_propose(p, gpu_theta_grad(g[i], p), st, i, stage, sweep, gamma)
        assert bool(prop.valid[i]) == (q is not None), i
        if q is None:
            assert R.theta_of(to_oracle(prop, i), st).tolist() == R.theta_of(p, st).tolist()
            continue
        n_valid += 1
        got = np.array([prop.phib[i], *prop.phic[i, :p.kappa], *prop.zc[i, :p.kappa], *prop.zm[i, :p.lam],
                        *prop.mv[i, :p.lam], prop.tau[i], prop.c[i]], dtype=np.float64)
        ref = np.array([q.phib, *q.phic, *q.zc, *q.zm, *q.mv, q.tau, q.c]).astype(np.float32).astype(np.float64)
        assert np.allclose(got, ref, rtol=2.5e-7, atol=0), (i, got, ref)
    assert 0 < n_valid


def test_langevin_decisions_match_oracle(env):
    S, gsys, s, data = env
    st = settings(n_particles=48, langevin_h=0.01)
    parts = near_truth_particles(st.n_particles, seed=3, st=st)
    gamma, stage = 0.5, 6
    host = to_host(S, parts)
    sm = gpu_smc(S, gsys, data, st)
    sm.set_particles(host, gamma=np.array([gamma]), stage=stage)
    g0 = sm.grad_current()
    ll0 = sm.get_particles(0).ll.copy()
    sm.langevin_propose(stage, 0)
    prop = sm.get_particles(1)
    # the GPU's likelihoods and gradients at the proposals
    sm2 = gpu_smc(S, gsys, data, st)
    sm2.set_particles(prop, gamma=np.array([gamma]), stage=stage)
    g1 = sm2.grad_current()
    ll1 = sm2.get_particles(0).ll.copy()
    # one full Langevin sweep from the same state
    sm.set_particles(host, gamma=np.array([gamma]), stage=stage)
    sm.langevin(1)
    fin = sm.get_particles(0)
    acc, nprop, _ = sm.langevin_stats()
    assert nprop[0] == st.n_particles
    lik = R.ForwardLik(s, data, I.EPS_AN, I.EPS_MN, st.kappa_max + st.lambda_max + 1)
    n_acc = 0
    n_valid = 0
    agree_orc = 0
    checked_orc = 0
    for i, p in enumerate(parts):
        th = R.theta_of(p, st)
        q = to_oracle(prop, i)
        thq = R.theta_of(q, st)
        moved = R.theta_of(to_oracle(fin, i), st).tolist() == thq.tolist() and bool(prop.valid[i])
        if not prop.valid[i]:
            assert R.theta_of(to_oracle(fin, i), st).tolist() == th.tolist()
            continue
        n_acc += moved
        n_valid += 1
        sc = R.theta_scales(p, st)
        lu = math.log(R.langevin_accept_uniform(st, i, stage, 0))
        # oracle formula on the GPU's own likelihoods and gradients
        m_gpu = (gamma * (ll1[i] - ll0[i]) + R.langevin_log_q(th, thq, gpu_theta_grad(g1[i], q), sc, gamma, st.langevin_h)
                 - R.langevin_log_q(thq, th, gpu_theta_grad(g0[i], p), sc, gamma, st.langevin_h) - lu)
        if abs(m_gpu) > 1e-4:
            assert moved == (m_gpu > 0), (i, m_gpu)
        # and on the FP64 oracle's likelihoods and central-difference gradients
        (l0r, l1r), (g0r, g1r) = R.theta_grad_fd([p, q], st, lik)
        m_orc = (gamma * (l1r - l0r) + R.langevin_log_q(th, thq, g1r, sc, gamma, st.langevin_h)
                 - R.langevin_log_q(thq, th, g0r, sc, gamma, st.langevin_h) - lu)
        tol = (gamma * (abs(ll1[i] - l1r) + abs(ll0[i] - l0r))
               + abs(R.langevin_log_q(th, thq, g1r, sc, gamma, st.langevin_h)
                     - R.langevin_log_q(th, thq, gpu_theta_grad(g1[i], q), sc, gamma, st.langevin_h))
               + abs(R.langevin_log_q(thq, th, g0r, sc, gamma, st.langevin_h)
                     - R.langevin_log_q(thq, th, gpu_theta_grad(g0[i], p), sc, gamma, st.langevin_h)) + 1e-4)
        if abs(m_orc) > tol:
            checked_orc += 1
            agree_orc += moved == (m_orc > 0)
    assert acc[0] == n_acc
    assert 0 < n_acc < st.n_particles
    assert agree_orc == checked_orc and checked_orc >= n_valid // 2
    print(f"\nLangevin sweep: {n_acc} accepted of {st.n_particles}; {checked_orc} decisions checked against FP64")


def test_langevin_propose_needs_gradient(env):
    S, gsys, s, data = env
    st = settings(n_particles=8)
    sm = gpu_smc(S, gsys, data, st)
    sm.init()
    with pytest.raises(Exception):
        sm.langevin_propose(1, 0)
    sm.grad_current()
    sm.langevin_propose(1, 0)
    sm.loglik_current()
    with pytest.raises(Exception):
        sm.langevin_propose(1, 0)


@pytest.mark.slow
def test_langevin_keeps_posterior(env):
    """Over 10 seeds with two Langevin sweeps per stage, P(IP) and the
    posterior mean of phi_b (log10 sigma of the top layer) agree with the
    random-walk-only sampler within 3 pooled standard errors, and the adapted
    Langevin moves are accepted at a useful rate."""
    S, gsys, s, data = env
    res = {0: ([], []), 2: ([], [])}
    rates, hs = [], []
    for nl in (0, 2):
        for seed in range(10):
            st = settings(n_particles=256, kappa_max=3, lambda_max=4, n_langevin=nl, seed=300 + seed)
            sm = gpu_smc(S, gsys, data, st)
            sm.init()
            sm.run(max_stages=200, n_sweeps=10)
            post, _, _ = sm.model_odds()
            res[nl][0].append(post[0].reshape(4, 5)[:, 1:].sum())
            res[nl][1].append(float(np.mean(sm.get_particles(0).phib)))
            if nl:
                a, p, h = sm.langevin_stats()
                rates.append(a[0] / p[0])
                hs.append(h[0])
    for j, what in enumerate(("P(IP)", "mean phi_b")):
        g, o = np.asarray(res[2][j]), np.asarray(res[0][j])
        se = math.sqrt(g.var(ddof=1) / len(g) + o.var(ddof=1) / len(o))
        print(f"\n{what}: Langevin {g.mean():.4f} +- {g.std():.4f}, random walk {o.mean():.4f} +- {o.std():.4f}")
        assert abs(g.mean() - o.mean()) <= 3 * se + 0.01
    print(f"final-stage Langevin acceptance {np.mean(rates):.2f}, step h {np.mean(hs):.3g}")
    assert np.mean(rates) > 0.05
