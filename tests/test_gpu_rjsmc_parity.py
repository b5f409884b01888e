"""The tempered Metropolis-Hastings step and the model odds of the CUDA
sampler against the oracle, through the C ABI:

* decisions: for every particle of a sweep (all six move types, three
  tempering exponents gamma_t < 1), the GPU accepts exactly when the oracle's
  rule ln u < gamma_t (l' - l) (Appendix E: prior-drawn births make the prior
  and proposal ratios cancel) holds on the GPU's own likelihoods and the same
  Philox uniform, and agrees with the FP64 oracle's likelihoods wherever the
  margin exceeds their FP32 difference;
* model odds: on a weakly chargeable sounding (P(IP) near its prior value,
  log BFIPD near 0, so most runs sit at no limit), the GPU sampler's pi(k|y)
  for every model, P(IP), the fraction of runs with every particle on one
  side (log BFIPD = +-inf) and the mean of the finite, unclipped log BFIPD
  agree with the serial FP64 oracle's over independent seeds (>= 10 each
  side) within 3 pooled standard errors (3.5 for the per-model family);
* precision: the plain FP64 forward model inside the sampler gives prior
  log-likelihoods equal to the oracle's to rounding, and model odds
  statistically equal to the FP32 sampler's."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import rjsmc as R
from oracle_pool import oracle_odds
from paper_2109_00661_gb300 import inputs as I
from parity_util import bound32, kappa, loglik_bound, oracle_system

pytestmark = pytest.mark.gpu

NAME = "sounding-g20-f40-k120"
KS = 10


@pytest.fixture(scope="module")
def env():
    import paper_2109_00661_gb300 as L
    from paper_2109_00661_gb300 import smc as S
    gsys = L.System(**I.system_kwargs(NAME))
    s = oracle_system(NAME)
    data = I.noisy(O.forward(I.truth_3layer(), s, mode=O.HANKEL_RULE)[0], seed=0)
    marginal = I.noisy(O.forward(I.truth_marginal(), s, mode=O.HANKEL_RULE)[0], seed=0)
    return L, S, gsys, s, data, marginal


def near_truth_particles(N, seed, km, lm):
    """Particles near the three-layer truth, every value already a float32."""
    rng = np.random.default_rng(seed)
    f = lambda v: float(np.float32(v))
    out = []
    for _ in range(N):
        k = int(rng.integers(0, km + 1))
        l = int(rng.integers(0, lm + 1))
        zc = sorted(f(v) for v in rng.uniform(10.0, 90.0, k))
        zm = sorted(f(v) for v in rng.uniform(10.0, 90.0, l))
        out.append(R.Particle(k, l, f(rng.uniform(-2.3, -1.7)), zc, [f(v) for v in rng.uniform(-2.3, -0.8, k)], zm,
                              [f(v) for v in rng.uniform(0.05, 0.5, l)], f(10 ** rng.uniform(-3.5, -2.5)),
                              f(rng.uniform(0.3, 0.9))))
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


def same_particle(h, i, g, j):
    return (h.kappa[i] == g.kappa[j] and h.lam[i] == g.lam[j] and h.phib[i] == g.phib[j] and h.tau[i] == g.tau[j]
            and h.c[i] == g.c[j] and np.array_equal(h.zc[i], g.zc[j]) and np.array_equal(h.phic[i], g.phic[j])
            and np.array_equal(h.zm[i], g.zm[j]) and np.array_equal(h.mv[i], g.mv[j]))


@pytest.mark.parametrize("gamma", [0.02, 0.2, 0.7])
def test_accept_decisions_match_oracle(env, gamma):
    L, S, gsys, s, data, _ = env
    km, lm, N, stage, seed = 3, 4, 768, 5, 17
    st = R.SMCSettings(n_particles=N, kappa_max=km, lambda_max=lm, seed=seed)
    parts = near_truth_particles(N, seed=int(gamma * 100), km=km, lm=lm)
    host = to_host(S, parts)
    mk = lambda: S.SMC(gsys, data, I.EPS_AN, I.EPS_MN, n_particles=N, kappa_max=km, lambda_max=lm, seed=seed)
    sm = mk()
    sm.set_particles(host, gamma=np.array([gamma]), stage=stage)
    sm.loglik_current()
    cur = sm.get_particles(0)
    ll0 = cur.ll.copy()
    sm.propose(stage, 0)
    prop = sm.get_particles(1)
    # the GPU's likelihoods of the proposals
    sm2 = mk()
    sm2.set_particles(prop, gamma=np.array([gamma]), stage=stage)
    sm2.loglik_current()
    ll1 = sm2.get_particles(0).ll.copy()
    # one sweep from the same state
    sm.set_particles(cur, gamma=np.array([gamma]), stage=stage)
    sm.mutate(1)
    fin = sm.get_particles(0)
    info = sm.stats()
    # the FP64 oracle's likelihoods of both sets
    lik = R.ForwardLik(s, data, I.EPS_AN, I.EPS_MN, km + lm + 1)
    valid = prop.valid.astype(bool)
    l0r = lik([to_oracle(cur, i) for i in range(N)])
    l1r = np.full(N, -np.inf)
    l1r[valid] = lik([to_oracle(prop, i) for i in np.nonzero(valid)[0]])
    acc = np.zeros(6, int)
    tried = np.zeros(6, int)
    checked = agree = 0
    for i in range(N):
        mv = int(prop.move[i])
        tried[mv] += 1
        moved = bool(valid[i]) and same_particle(fin, i, prop, i)
        stayed = same_particle(fin, i, cur, i)
        assert moved or stayed, i
        if not valid[i]:
            assert stayed
            continue
        assert not same_particle(cur, i, prop, i), i  # a valid move changes the particle
        lu = math.log(R.accept_uniform(st, i, stage, 0))
        margin = gamma * (ll1[i] - ll0[i]) - lu
        if abs(margin) > 1e-9 * (1.0 + gamma * abs(ll1[i] - ll0[i])):
            assert moved == (margin > 0), (i, mv, margin)
        acc[mv] += moved
        # the FP64 oracle's decision, where the FP32 likelihoods cannot flip it
        m_orc = gamma * (l1r[i] - l0r[i]) - lu
        tol = gamma * (abs(ll1[i] - l1r[i]) + abs(ll0[i] - l0r[i])) + 1e-9
        if abs(m_orc) > tol:
            checked += 1
            agree += moved == (m_orc > 0)
    assert np.array_equal(info["accepted"][0], acc) and np.array_equal(info["proposed"][0], tried)
    print(f"\ngamma {gamma}: accepted {acc.tolist()} of {tried.tolist()} by move type; "
          f"{checked} decisions checked against FP64 likelihoods")
    assert np.all(tried > 0) and acc.sum() > 0 and acc.sum() < valid.sum()
    assert agree == checked and checked >= 0.8 * valid.sum()


MARGINAL = dict(n_particles=128, kappa_max=2, lambda_max=2, n_sweeps=10)


def gpu_odds(S, gsys, y, n_runs, seed, **extra):
    """n_runs independent samplers as the soundings of one sampler (each
    sounding draws from its own Philox key)."""
    st = MARGINAL
    sm = S.SMC(gsys, np.tile(y, (n_runs, 1)), I.EPS_AN, I.EPS_MN, n_particles=st["n_particles"], n_soundings=n_runs,
               kappa_max=st["kappa_max"], lambda_max=st["lambda_max"], seed=seed, r_max=10, **extra)
    sm.init()
    stages = sm.run(max_stages=300, n_sweeps=st["n_sweeps"])
    post, lb, _ = sm.model_odds()
    return post, lb, stages


def p_ip(post):
    return post.reshape(len(post), MARGINAL["kappa_max"] + 1, MARGINAL["lambda_max"] + 1)[:, :, 1:].sum(axis=(1, 2))


def compare(a, b, z):
    a, b = np.asarray(a, float), np.asarray(b, float)
    se = math.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b))
    d = abs(a.mean() - b.mean())
    return d, se, d <= z * se + 1e-12


def check_odds(pa, la, pb, lb, what):
    lines = []
    ok = True
    d, se, good = compare(p_ip(pa), p_ip(pb), 3.0)
    ok &= good
    lines.append(f"P(IP): {p_ip(pa).mean():.3f} vs {p_ip(pb).mean():.3f}, |diff| {d / max(se, 1e-300):.2f} SE")
    # log BFIPD unclipped: a run with every particle on one side has +-inf;
    # the fraction of such runs is compared as a proportion and the finite
    # values by their mean
    fa, fb = np.isfinite(la), np.isfinite(lb)
    d, se, good = compare(~fa, ~fb, 3.0)
    ok &= good or (fa.all() and fb.all())
    lines.append(f"one-sided runs: {np.mean(~fa):.3f} vs {np.mean(~fb):.3f}, |diff| {d / max(se, 1e-300):.2f} SE")
    assert fa.sum() >= 5 and fb.sum() >= 5
    d, se, good = compare(la[fa], lb[fb], 3.0)
    ok &= good
    lines.append(f"finite log BFIPD: {la[fa].mean():.3f} vs {lb[fb].mean():.3f}, |diff| {d / se:.2f} SE")
    diffs = []
    for k in range(pa.shape[1]):
        d, se, good = compare(pa[:, k], pb[:, k], 3.5)
        ok &= good
        diffs.append(d / max(se, 1e-300))
    lines.append("pi(k|y) per model: " + " ".join(f"{a:.3f}/{b:.3f}" for a, b in zip(pa.mean(0), pb.mean(0))) +
                 "; |diff| / SE " + " ".join(f"{v:.2f}" for v in diffs))
    print(f"\n{what}: " + "; ".join(lines))
    assert ok


@pytest.mark.slow
def test_model_odds_statistical_parity_marginal(env):
    L, S, gsys, s, data, marginal = env
    pg, lg, sg = gpu_odds(S, gsys, marginal, 32, seed=101)
    po, lo, so = oracle_odds(NAME, "truth_marginal", list(range(300, 316)), **MARGINAL)
    print(f"\nstages: GPU {sg}, oracle {so.tolist()}")
    assert 0.2 < p_ip(pg).mean() < 0.8 and 0.2 < p_ip(po).mean() < 0.8
    check_odds(pg, lg, po, lo, "GPU FP32 (32 runs) vs oracle FP64 (16 runs)")


def test_fp64_sampler_prior_loglik_matches_oracle(env):
    L, S, gsys, s, data, _ = env
    sm = S.SMC(gsys, data, I.EPS_AN, I.EPS_MN, n_particles=256, kappa_max=3, lambda_max=4, seed=11, precision=1)
    sm.init()
    p = sm.get_particles(0)
    parts = [to_oracle(p, i) for i in range(256)]
    mb = R.merged_batch(parts, 8)
    y, imh, absh = O.forward(mb, s, mode=O.HANKEL_RULE, want_imh=True, want_absh=True)
    ll_ref = O.loglik(y, data, I.EPS_AN, I.EPS_MN)
    # FP64 on both sides: the bound of the FP64 forward tests
    kap = kappa(imh, s["T"], y, absh)
    b = 1e-7 + kap[2] * 1e-12 + kap[0] * 2.0 ** -52 * 64 + kap[1] * 1e-8
    assert np.all(np.abs(p.ll - ll_ref) <= loglik_bound(y, data, b) + 1e-10 * np.abs(ll_ref))
    # and the FP32 sampler on the same particles within the FP32 bound
    sm32 = S.SMC(gsys, data, I.EPS_AN, I.EPS_MN, n_particles=256, kappa_max=3, lambda_max=4, seed=11)
    sm32.set_particles(p)
    sm32.loglik_current()
    ll32 = sm32.get_particles(0).ll
    assert np.all(np.abs(ll32 - ll_ref) <= loglik_bound(y, data, bound32(kap, s["T"].shape[1])) + 1e-9 * np.abs(ll_ref))


def test_fp64_sampler_rejects_langevin(env):
    L, S, gsys, s, data, _ = env
    with pytest.raises(L.AEMError):
        S.SMC(gsys, data, I.EPS_AN, I.EPS_MN, n_particles=64, precision=1, n_langevin=1)
    with pytest.raises(L.AEMError):
        S.SMC(gsys, data, I.EPS_AN, I.EPS_MN, n_particles=64, precision=2)


@pytest.mark.slow
def test_fp64_sampler_odds_match_fp32(env):
    """The chosen FP32 forward model against the plain FP64 one inside the
    same sampler (different trajectories after the first flipped decision):
    statistically equal model odds on the weakly chargeable sounding."""
    L, S, gsys, s, data, marginal = env
    p32, l32, s32 = gpu_odds(S, gsys, marginal, 48, seed=7)
    p64, l64, s64 = gpu_odds(S, gsys, marginal, 48, seed=8, precision=1)
    print(f"\nstages: FP32 {s32}, FP64 {s64}")
    check_odds(p32, l32, p64, l64, "GPU FP32 (48 runs) vs GPU FP64 (48 runs)")
