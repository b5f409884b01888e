"""The adaptive within-model proposal of Section 3.2 on the GPU against the
oracle, through the C ABI:

* the fit: per (sounding, model) mean and ridged covariance of the
  particles' parameters equal numpy's, reconstructed from the GPU's U, Lambda
  (orthonormal U; eigenvalues equal numpy's eigvalsh);
* the moves: given the GPU's fit and scales, every proposal of a sweep equals
  the oracle's propose_adaptive to float32 rounding;
* the scale bisection: the oracle's pca_bisect_scales on the GPU's own
  likelihoods and fit takes the same decisions;
* the adaptation itself: in the sweeps of the final stage the adaptive
  perturb move is accepted near its 0.44 target (the convergence of both
  samplers on eight soundings is printed)."""
import numpy as np
import pytest

import oracle as O
from oracle import rjsmc as R
from paper_2109_00661_gb300 import inputs as I
from parity_util import oracle_system

pytestmark = pytest.mark.gpu

NAME = "sounding-g20-f40-k120"


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2109_00661_gb300 as L
    from paper_2109_00661_gb300 import smc as S
    gsys = L.System(**I.system_kwargs(NAME))
    s = oracle_system(NAME)
    y_true = O.forward(I.truth_3layer(), s, mode=O.HANKEL_RULE)[0]
    return torch, L, S, gsys, s, y_true


def settings(**kw):
    base = dict(n_particles=512, kappa_max=2, lambda_max=2, n_sweeps=10, adaptive=True, seed=7)
    base.update(kw)
    return R.SMCSettings(**base)


def gpu_smc(S, gsys, data, st, soundings=1):
    return S.SMC(gsys, np.tile(data, (soundings, 1)), I.EPS_AN, I.EPS_MN, n_particles=st.n_particles,
                 n_soundings=soundings, kappa_max=st.kappa_max, lambda_max=st.lambda_max, seed=st.seed,
                 adaptive=int(st.adaptive), pca_target=st.pca_target, pca_bisect_iters=st.pca_bisect_iters,
                 pca_ridge=st.pca_ridge, zca=float(st.zca))


def to_oracle(h, i):
    k, l = int(h.kappa[i]), int(h.lam[i])
    f = lambda v: float(np.float64(v))
    return R.Particle(k, l, f(h.phib[i]), [f(v) for v in h.zc[i, :k]], [f(v) for v in h.phic[i, :k]],
                      [f(v) for v in h.zm[i, :l]], [f(v) for v in h.mv[i, :l]], f(h.tau[i]), f(h.c[i]))


def staged(S, gsys, data, st):
    """A sampler after its first reweight and resample, with the stage's fit."""
    sm = gpu_smc(S, gsys, data, st)
    sm.init()
    g = sm.reweight()
    sm.resample()
    sm.adapt()
    return sm, g[0]


def gpu_fits(ad, st, s_idx=0):
    fits, scales = {}, {}
    for k in range(st.n_models):
        if ad["ok"][s_idx, k]:
            kap, lam = divmod(k, st.lambda_max + 1)
            d = 3 + 2 * kap + 2 * lam
            fits[k] = (ad["mu"][s_idx, k, :d], ad["U"][s_idx, k, :d, :d], ad["lam"][s_idx, k, :d])
            scales[k] = float(ad["scale"][s_idx, k])
    return fits, scales


def test_fit_matches_numpy(env):
    torch, L, S, gsys, s, y_true = env
    st = settings()
    sm, _ = staged(S, gsys, I.noisy(y_true, seed=0), st)
    ad = sm.adaptation()
    p = sm.get_particles(0)
    parts = [to_oracle(p, i) for i in range(st.n_particles)]
    model = np.array([q.model(st) for q in parts])
    n_ok = 0
    for k in range(st.n_models):
        members = [q for q in parts if q.model(st) == k]
        assert bool(ad["ok"][0, k]) == (len(members) >= 2)
        if len(members) < 2:
            continue
        n_ok += 1
        X = np.array([R.theta_of(q, st) for q in members])
        d = X.shape[1]
        mu = X.mean(axis=0)
        C = (X - mu).T @ (X - mu) / len(members) + np.diag((st.pca_ridge * R.theta_scales(members[0], st)) ** 2)
        U = ad["U"][0, k, :d, :d]
        lam = ad["lam"][0, k, :d]
        assert np.allclose(ad["mu"][0, k, :d], mu, rtol=1e-12, atol=1e-12 * np.abs(mu).max())
        assert np.allclose(U.T @ U, np.eye(d), atol=1e-10)
        assert np.allclose(U @ np.diag(lam) @ U.T, C, atol=1e-9 * np.abs(C).max())
        assert np.allclose(np.sort(lam), np.linalg.eigvalsh(C), atol=1e-9 * np.abs(C).max())
    assert n_ok >= 3 and len(set(model)) == st.n_models


@pytest.mark.parametrize("sweep", [0, 5])
def test_moves_match_oracle(env, sweep):
    torch, L, S, gsys, s, y_true = env
    st = settings()
    sm, _ = staged(S, gsys, I.noisy(y_true, seed=0), st)
    fits, scales = gpu_fits(sm.adaptation(), st)
    stage = 1
    sm.propose(stage, sweep)
    cur, prop = sm.get_particles(0), sm.get_particles(1)
    n_pca = 0
    for i in range(st.n_particles):
        p = to_oracle(cur, i)
        mv, q = R.propose_adaptive(p, st, i, stage, sweep, fits, scales)
        assert prop.move[i] == mv and bool(prop.valid[i]) == (q is not None), i
        if q is None:
            continue
        n_pca += mv == 5 and p.model(st) in fits
        got = R.theta_of(to_oracle(prop, i), st)
        ref = R.theta_of(q, st).astype(np.float32).astype(np.float64)
        assert (q.kappa, q.lam) == (int(prop.kappa[i]), int(prop.lam[i]))
        assert np.allclose(got, ref, rtol=4e-7, atol=1e-30), (i, mv, got, ref)
    assert n_pca > 10


def test_scale_bisection_matches_oracle(env):
    torch, L, S, gsys, s, y_true = env
    st = settings()
    data = I.noisy(y_true, seed=0)
    sm, gamma = staged(S, gsys, data, st)
    ad = sm.adaptation()
    fits, scales = gpu_fits(ad, st)
    p = sm.get_particles(0)
    parts = [to_oracle(p, i) for i in range(st.n_particles)]
    lmax = st.kappa_max + st.lambda_max + 1

    def gpu_loglik(ps):
        mb = R.merged_batch(ps, lmax)
        return L.loglik_f32(gsys, I.to_torch(mb, torch.float32), data, I.EPS_AN, I.EPS_MN).cpu().numpy()

    ref = R.pca_bisect_scales(parts, p.ll, fits, st, 1, gamma, gpu_loglik, a_prev={})
    same = [abs(np.log(scales[k]) - np.log(ref[k])) < 1e-9 for k in fits]
    print(f"\nscales (GPU): {np.round([scales[k] for k in fits], 3)}; equal to the oracle's for {sum(same)} of {len(same)}")
    assert sum(same) >= 0.9 * len(same)


def test_adaptive_perturb_acceptance_near_target(env):
    torch, L, S, gsys, s, y_true = env
    SN = 8
    data = np.stack([I.noisy(y_true, seed=k) for k in range(SN)])
    ll_true = O.loglik(np.tile(y_true, (SN, 1)), data, I.EPS_AN, I.EPS_MN)
    rate = {}
    for adaptive in (0, 1):
        sm = S.SMC(gsys, data, I.EPS_AN, I.EPS_MN, n_particles=256, n_soundings=SN, kappa_max=3, lambda_max=4,
                   seed=4, adaptive=adaptive)
        sm.init()
        stages = sm.run(max_stages=400, n_sweeps=20)
        info = sm.stats()
        rate[adaptive] = info["accepted"][:, 5].sum() / info["proposed"][:, 5].sum()
        p = sm.get_particles(0)
        llmax = np.array([p.ll[k * 256:(k + 1) * 256].max() for k in range(SN)])
        print(f"\nadaptive={adaptive}: {stages} stages, final-stage perturb acceptance {rate[adaptive]:.3f}, "
              f"{np.mean(llmax > ll_true - 50):.2f} of soundings within 50 of the truth's log-likelihood")
    assert abs(rate[1] - 0.44) < 0.12


def test_recycled_fit_matches_oracle(env):
    """Particle recycling (Section 3.2): at each of four stages the GPU's fit
    over the last three post-resample populations equals the oracle's
    weighted fit on the same populations, log-likelihoods, gammas and
    evidence estimates."""
    torch, L, S, gsys, s, y_true = env
    st = settings(n_particles=384, recycle=3)
    sm = S.SMC(gsys, I.noisy(y_true, seed=0), I.EPS_AN, I.EPS_MN, n_particles=st.n_particles,
               kappa_max=st.kappa_max, lambda_max=st.lambda_max, seed=st.seed, adaptive=1, recycle_stages=3)
    sm.init()

    def population():
        p = sm.get_particles(0)
        return [to_oracle(p, i) for i in range(st.n_particles)], p.ll.copy()

    parts, ll = population()
    history, gammas, log_z = [(0, parts, ll)], [0.0], [np.zeros(st.n_models)]
    n_checked = 0
    for t in range(1, 5):
        g = sm.reweight()
        sm.resample()
        parts, ll = population()
        _, _, lz = sm.model_odds()
        gammas.append(g[0])
        log_z.append(lz[0].copy())
        history = (history + [(t, parts, ll)])[-3:]
        sm.adapt()
        ad = sm.adaptation()
        ref = R.fit_model_gaussians_recycled(history, st, t, gammas, log_z)
        for k in range(st.n_models):
            assert bool(ad["ok"][0, k]) == (k in ref), (t, k)
            if k not in ref:
                continue
            mu, U, lam = ref[k]
            d = len(mu)
            C_ref = U @ np.diag(lam) @ U.T
            Ug, lg = ad["U"][0, k, :d, :d], ad["lam"][0, k, :d]
            scale = np.abs(C_ref).max()
            assert np.allclose(ad["mu"][0, k, :d], mu, rtol=1e-10, atol=1e-10 * np.abs(mu).max()), (t, k)
            assert np.allclose(Ug @ np.diag(lg) @ Ug.T, C_ref, atol=1e-9 * scale), (t, k)
            n_checked += 1
        sm.mutate(3)
    assert n_checked >= 20
    # the image carries the recycling history (resume is tested in test_gpu_checkpoint.py)
    assert len(sm.checkpoint()) > 3 * sm.P * 8


@pytest.mark.parametrize("zca", [1.0, 0.5])
def test_zca_moves_match_oracle(env, zca):
    """Appendix F's ZCA-coloured birth / death on the GPU: given the GPU's fit,
    every proposal of a sweep and its log factor equal the oracle's
    propose_adaptive (moves, support decisions, parameters to float32
    rounding, log factors to 1e-9)."""
    torch, L, S, gsys, s, y_true = env
    st = settings(zca=zca)
    sm, _ = staged(S, gsys, I.noisy(y_true, seed=0), st)
    fits, scales = gpu_fits(sm.adaptation(), st)
    n_zca = 0
    for sweep in (0, 3):
        sm.propose(1, sweep)
        cur, prop = sm.get_particles(0), sm.get_particles(1)
        lf = sm.log_factors()
        for i in range(st.n_particles):
            p = to_oracle(cur, i)
            res = R.propose_adaptive(p, st, i, 1, sweep, fits, scales)
            mv, q = res[:2]
            lf_ref = res[2] if len(res) > 2 else 0.0
            assert prop.move[i] == mv and bool(prop.valid[i]) == (q is not None), (i, mv)
            if len(res) > 2:
                n_zca += 1
                assert abs(lf[i] - lf_ref) <= 1e-9 * max(1.0, abs(lf_ref)), (i, lf[i], lf_ref)
            else:
                assert lf[i] == 0.0
            if q is None:
                continue
            assert (q.kappa, q.lam) == (int(prop.kappa[i]), int(prop.lam[i]))
            got = R.theta_of(to_oracle(prop, i), st)
            ref = R.theta_of(q, st).astype(np.float32).astype(np.float64)
            assert np.allclose(got, ref, rtol=4e-7, atol=1e-30), (i, mv, got, ref)
    assert n_zca > 50
