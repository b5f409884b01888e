"""Parity of the CUDA RJSMC stage (through the C ABI) with the serial oracle:
bit-exact Philox streams and resampling, reweighting to rounding, identical
prior draws and proposals given the same state, model odds consistent with the
particle counts (the decision-level and statistical parity of the mutation
and of the model odds are in test_gpu_rjsmc_parity.py)."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import rjsmc as R
from paper_2109_00661_gb300 import inputs as I
from parity_util import bound32, kappa, loglik_bound, oracle_system

pytestmark = pytest.mark.gpu

NAME = "sounding-g20-f40-k120"


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


@pytest.fixture(scope="module")
def L():
    import paper_2109_00661_gb300 as lib
    return lib


@pytest.fixture(scope="module")
def S():
    from paper_2109_00661_gb300 import smc
    return smc


@pytest.fixture(scope="module")
def gsys(L):
    return L.System(**I.system_kwargs(NAME))


@pytest.fixture(scope="module")
def data():
    s = oracle_system(NAME)
    y_true = O.forward(I.truth_3layer(), s, mode=O.HANKEL_RULE)[0]
    return I.noisy(y_true, seed=0)


def test_philox_bit_exact(torch, S):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, (1000, 4), dtype=np.uint64)
    ctr[:10] = 0
    for key in [(0, 0), (123456789, 987654321), (2 ** 32 - 1, 7)]:
        ref = R.philox4x32(ctr, key)
        got = S.philox4x32(torch.as_tensor(ctr.astype(np.uint32).view(np.int32), device="cuda"), *key)
        got = got.cpu().numpy().view(np.uint32).astype(np.uint64)
        assert np.array_equal(got, ref)


def population(seed, N, K, spread=15.0):
    rng = np.random.default_rng(seed)
    model = rng.integers(0, K, N)
    model[: K // 3] = 0  # some models may be empty, model 0 never is
    ll = rng.normal(-40.0, spread, N) - 3.0 * model
    return ll, model


@pytest.mark.parametrize("case", [(0, 256, 20, 0.0), (1, 4096, 100, 0.3), (2, 1000, 7, 0.9), (3, 64, 1, 0.0)])
def test_reweight_matches_oracle(torch, S, case):
    seed, N, K, g0 = case
    ll, model = population(seed, N, K)
    dg, done, inc, W = S.reweight(torch.as_tensor(ll, device="cuda"),
                                  torch.as_tensor(model.astype(np.int32), device="cuda"), K, g0, 0.5)
    dg_ref, done_ref, inc_ref, W_ref = R.reweight(ll, model, K, g0, 0.5)
    assert int(done.item()) == int(done_ref)
    assert abs(dg.item() - dg_ref) <= 1e-10 * max(dg_ref, 1e-300) + 1e-15
    present = np.bincount(model, minlength=K) > 0
    assert np.allclose(inc.cpu().numpy()[present], inc_ref[present], rtol=1e-9, atol=1e-9)
    assert np.allclose(W.cpu().numpy(), W_ref, rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("case", [(0, 300, 9), (1, 4096, 100), (2, 17, 3), (3, 1, 1)])
def test_resample_bit_exact(torch, S, case):
    seed, N, K = case
    rng = np.random.default_rng(seed)
    model = rng.integers(0, K, N)
    W = np.zeros(N)
    for k in range(K):
        idx = np.nonzero(model == k)[0]
        if idx.size:
            w = rng.exponential(1.0, idx.size) ** 4
            W[idx] = w / w.sum()
    u40 = rng.integers(0, 1 << 40, K, dtype=np.uint64)
    ref = R.resample_systematic(W, model, K, u40)
    got = S.resample_systematic(torch.as_tensor(W, device="cuda"), torch.as_tensor(model.astype(np.int32), device="cuda"),
                                K, torch.as_tensor(u40.astype(np.int64), device="cuda"))
    assert np.array_equal(got.cpu().numpy(), ref)


def test_out_of_range_model_ids_take_no_part(torch, S):
    """Standalone a7 / a8 with model ids outside [0, n_models) (negative, just
    past the range, past 255): those particles get ancestor -1 and weight 0,
    and the others are resampled exactly as without them."""
    rng = np.random.default_rng(9)
    N, K = 500, 7
    model = rng.integers(0, K, N)
    bad = rng.choice(N, 40, replace=False)
    model[bad[:10]] = -1
    model[bad[10:20]] = K
    model[bad[20:30]] = 300
    model[bad[30:]] = 256 + 3  # would alias model 3 in an 8-bit key
    good = np.ones(N, bool)
    good[bad] = False
    W = np.zeros(N)
    for k in range(K):
        idx = np.nonzero((model == k) & good)[0]
        w = rng.exponential(1.0, idx.size)
        W[idx] = w / w.sum()
    u40 = rng.integers(0, 1 << 40, K, dtype=np.uint64)
    mt = torch.as_tensor(model.astype(np.int32), device="cuda")
    got = S.resample_systematic(torch.as_tensor(W, device="cuda"), mt, K,
                                torch.as_tensor(u40.astype(np.int64), device="cuda")).cpu().numpy()
    keep = np.nonzero(good)[0]
    ref = R.resample_systematic(W[keep], model[keep], K, u40)
    assert np.all(got[bad] == -1)
    assert np.array_equal(got[keep], keep[ref])
    ll = rng.normal(-30.0, 5.0, N)
    _, _, _, Wr = S.reweight(torch.as_tensor(ll, device="cuda"), mt, K, 0.2, 0.5)
    _, _, _, W_ref = R.reweight(ll[keep], model[keep], K, 0.2, 0.5)
    Wr = Wr.cpu().numpy()
    assert np.all(Wr[bad] == 0.0) and np.allclose(Wr[keep], W_ref, rtol=1e-8, atol=1e-14)


def settings(**kw):
    base = dict(n_particles=128, kappa_max=3, lambda_max=4, n_sweeps=10, seed=11)
    base.update(kw)
    return R.SMCSettings(**base)


def gpu_smc(S, gsys, data, st: R.SMCSettings, soundings=1):
    return S.SMC(gsys, np.tile(data, (soundings, 1)), I.EPS_AN, I.EPS_MN, n_particles=st.n_particles,
                 n_soundings=soundings, kappa_max=st.kappa_max, lambda_max=st.lambda_max, zmax=st.zmax,
                 seed=st.seed, r_max=st.r_max)


def to_oracle(p, i):
    k, l = int(p.kappa[i]), int(p.lam[i])
    f = lambda v: float(np.float64(v))
    return R.Particle(k, l, f(p.phib[i]), [f(v) for v in p.zc[i, :k]], [f(v) for v in p.phic[i, :k]],
                      [f(v) for v in p.zm[i, :l]], [f(v) for v in p.mv[i, :l]], f(p.tau[i]), f(p.c[i]))


def test_prior_draws_match_oracle(S, gsys, data):
    st = settings()
    sm = gpu_smc(S, gsys, data, st)
    sm.init()
    p = sm.get_particles(0)
    for i in range(st.n_particles):
        ref = R.sample_prior(st, i)
        assert (int(p.kappa[i]), int(p.lam[i])) == (ref.kappa, ref.lam)
        f32 = lambda v: np.float32(v)
        assert p.phib[i] == f32(ref.phib) and p.tau[i] == f32(ref.tau) and p.c[i] == f32(ref.c)
        assert np.array_equal(p.zc[i, :ref.kappa], np.float32(ref.zc))
        assert np.array_equal(p.phic[i, :ref.kappa], np.float32(ref.phic))
        assert np.array_equal(p.zm[i, :ref.lam], np.float32(ref.zm))
        assert np.array_equal(p.mv[i, :ref.lam], np.float32(ref.mv))


def test_prior_loglik_matches_oracle(S, gsys, data):
    st = settings()
    sm = gpu_smc(S, gsys, data, st)
    sm.init()
    p = sm.get_particles(0)
    parts = [to_oracle(p, i) for i in range(st.n_particles)]
    mb = R.merged_batch(parts, st.kappa_max + st.lambda_max + 1)
    s = oracle_system(NAME)
    y, imh, absh = O.forward(mb, s, mode=O.HANKEL_RULE, want_imh=True, want_absh=True)
    ll_ref = O.loglik(y, data, I.EPS_AN, I.EPS_MN)
    bound = loglik_bound(y, data, bound32(kappa(imh, s["T"], y, absh), s["T"].shape[1]))
    assert np.all(np.abs(p.ll - ll_ref) <= bound + 1e-9 * np.abs(ll_ref))


@pytest.mark.parametrize("stage,sweep", [(1, 0), (3, 7), (12, 2)])
def test_proposals_match_oracle(S, gsys, data, stage, sweep):
    st = settings(n_particles=512)
    sm = gpu_smc(S, gsys, data, st)
    sm.init()
    sm.propose(stage, sweep)
    cur = sm.get_particles(0)
    prop = sm.get_particles(1)
    moves = np.zeros(6, dtype=int)
    for i in range(st.n_particles):
        mv, q = R.propose(to_oracle(cur, i), st, i, stage, sweep)
        moves[mv] += 1
        assert prop.move[i] == mv
        assert bool(prop.valid[i]) == (q is not None)
        if q is None:
            continue
        assert (int(prop.kappa[i]), int(prop.lam[i])) == (q.kappa, q.lam)
        got = np.concatenate([[prop.phib[i], prop.tau[i], prop.c[i]], prop.zc[i, :q.kappa], prop.phic[i, :q.kappa],
                              prop.zm[i, :q.lam], prop.mv[i, :q.lam]]).astype(np.float64)
        ref = np.concatenate([[q.phib, q.tau, q.c], q.zc, q.phic, q.zm, q.mv]).astype(np.float32).astype(np.float64)
        assert np.allclose(got, ref, rtol=2e-7, atol=1e-30), (i, mv, got, ref)
    assert np.all(moves > 0)


@pytest.mark.parametrize("N,km,lm,soundings", [(256, 3, 4, 1), (1024, 3, 4, 1), (4096, 9, 9, 3)])
def test_stage_reweight_through_state_api(S, gsys, data, N, km, lm, soundings):
    """smc_reweight on the sampler's own particles equals the oracle step on
    the same log-likelihoods and model ids, per sounding: with one CTA per
    sounding (N = 256) and with the cluster-split form that few, large
    soundings take (N >= 1024)."""
    st = settings(n_particles=N, kappa_max=km, lambda_max=lm)
    sm = gpu_smc(S, gsys, data, st, soundings=soundings)
    sm.init()
    p = sm.get_particles(0)
    g = sm.reweight()
    _, _, lz = sm.model_odds()
    for s_ in range(soundings):
        sl = slice(s_ * N, (s_ + 1) * N)
        model = p.kappa[sl] * (st.lambda_max + 1) + p.lam[sl]
        dg_ref, done_ref, inc_ref, _ = R.reweight(p.ll[sl], model, st.n_models, 0.0, 0.5)
        assert abs(g[s_] - (1.0 if done_ref else dg_ref)) <= 1e-10 * max(dg_ref, 1e-300)
        present = np.bincount(model, minlength=st.n_models) > 0
        assert np.allclose(lz[s_][present], inc_ref[present], rtol=1e-9, atol=1e-9)


def test_model_odds_consistent_with_counts(S, gsys, data):
    st = settings(n_particles=256)
    sm = gpu_smc(S, gsys, data, st, soundings=3)
    sm.init()
    post, lb, _ = sm.model_odds()
    p = sm.get_particles(0)
    for s in range(3):
        sl = slice(s * 256, (s + 1) * 256)
        model = p.kappa[sl] * (st.lambda_max + 1) + p.lam[sl]
        counts = np.bincount(model, minlength=st.n_models)
        assert np.allclose(post[s], counts / 256)
        ref_post, ref_lb = R.model_odds(counts, st.kappa_max, st.lambda_max)
        assert lb[s] == pytest.approx(ref_lb)
    # soundings draw from independent streams
    assert not np.array_equal(p.kappa[:256], p.kappa[256:512])


def run_gpu(S, gsys, data, seed, N=256):
    st = settings(n_particles=N, seed=seed)
    sm = gpu_smc(S, gsys, data, st)
    sm.init()
    stages = sm.run(max_stages=200, n_sweeps=10)
    post, lb, lz = sm.model_odds()
    info = sm.stats()
    return stages, post[0], lb[0], info


def test_full_rjsmc_reaches_gamma_one(S, gsys, data):
    stages, post, lb, info = run_gpu(S, gsys, data, seed=3)
    assert info["gamma"][0] == 1.0
    assert 1 < stages < 200
    assert abs(post.sum() - 1.0) < 1e-12
    assert info["proposed"][0].sum() == 256 * 10


def test_flight_line_ip_probability_follows_chargeability(torch, L, S):
    """All soundings of a synthetic line in one sampler: the chargeable-model
    probability is high where the second layer is chargeable (m = 0.5 at the
    centre) and the IP odds fall towards the ends where m -> 0 (Section 4.1:
    detectability grows with chargeability)."""
    truth, x = I.flight_line(9)
    sysg = L.System(**I.system_kwargs(NAME))
    y = L.forward_f32(sysg, I.to_torch(truth, torch.float32)).cpu().numpy().astype(np.float64)
    y_obs = np.stack([I.noisy(y[s], seed=50 + s) for s in range(9)])
    sm = S.SMC(sysg, y_obs, I.EPS_AN, I.EPS_MN, n_particles=512, n_soundings=9, kappa_max=3, lambda_max=4,
               seed=5, r_max=10)
    sm.init()
    sm.run(max_stages=200, n_sweeps=10)
    post, lb, _ = sm.model_odds()
    p_ip = post.reshape(9, 4, 5)[:, :, 1:].sum(axis=(1, 2))
    print("\nx", np.round(x, 2), "\nP(IP)", np.round(p_ip, 3), "\nlog BFIPD", np.round(lb, 2))
    assert p_ip[4] > 0.9
    assert lb[4] > max(lb[0], lb[8])
    assert np.all(np.isfinite(post))


def test_detectability_study_trends(torch, L, S):
    """Section 4.1's synthetic study in one sampler: chargeable layer tops at
    10 and 60 m with m = 0 and 0.5, over a resistive (0.001 S/m) and a
    conductive (0.1 S/m) basement, tau = 4.07e-4 s, c = 1, N = 2048 per
    sounding.  The paper's findings, as inequalities on log BFIPD (clipped
    at +-50, where every particle sits on one side): the IP odds grow with
    chargeability, fall with depth and are higher over the resistive
    basement; without chargeability they stay below 1.5, at most weak
    evidence (2 ln B < 3 on Kass and Raftery's scale; models with a little
    chargeability fit such data as well as the others).  The log-uniform tau prior (log10 tau ~ U(-6, -1)) is used: the
    truth's tau sits at 4e-4 of the uniform prior's range, where a
    2048-particle population places almost no mass."""
    depths, ms, bases = (10.0, 60.0), (0.0, 0.5), (0.001, 0.1)
    grids = [I.detectability_grid(depths, ms, b) for b in bases]
    truth = {k: np.concatenate([g[k] for g in grids]) for k in grids[0]}
    n = len(truth["nlayers"])
    sysg = L.System(**I.system_kwargs(NAME))
    y = L.forward_f32(sysg, I.to_torch(truth, torch.float32)).cpu().numpy().astype(np.float64)
    y_obs = np.stack([I.noisy(y[s], seed=70 + s) for s in range(n)])
    sm = S.SMC(sysg, y_obs, I.EPS_AN, I.EPS_MN, n_particles=2048, n_soundings=n, kappa_max=3, lambda_max=4,
               seed=9, r_max=10, tau_log_prior=1)
    sm.init()
    sm.run(max_stages=300, n_sweeps=10)
    _, lb, _ = sm.model_odds()
    lb = np.clip(lb, -50, 50).reshape(2, 2, 2)  # (basement, depth, m)
    print("\nlog BFIPD [basement][depth][m]\n", np.round(lb, 2))
    assert np.all(lb[:, :, 1] > lb[:, :, 0])      # grows with chargeability
    assert np.all(lb[:, 0, 1] >= lb[:, 1, 1])     # falls with depth
    assert lb[0, 1, 1] >= lb[1, 1, 1]             # higher over the resistive basement
    assert np.all(lb[:, :, 0] < 1.5)              # no chargeability: at most weak evidence


# sampler options of the graph test: the fixed-scale moves; the adaptive
# proposal with particle recycling and ZCA-coloured birth / death; Langevin
# sweeps with step adaptation
GRAPH_MODES = {"fixed": {}, "adaptive_recycling_zca": dict(adaptive=1, recycle_stages=3, zca=0.5),
               "langevin": dict(n_langevin=2), "app_b_sweeps": {}}


@pytest.mark.parametrize("mode", list(GRAPH_MODES))
def test_graph_captured_run_equals_host_loop(S, gsys, data, mode):
    """smc_run_graph (one captured stage repeated by a device-side WHILE
    condition) reproduces smc_run bit for bit: particles, log-likelihoods,
    gammas, evidence estimates and the stage count, on three soundings, for
    each sampler option, and with App. B's sweep count R_t (n_sweeps = 0),
    which the graph form decides on the device."""
    import time
    runs = []
    n_sweeps = {"fixed": 10, "app_b_sweeps": 0}.get(mode, 4)
    for graph in (False, True):
        st = settings(n_particles=256, seed=21)
        sm = S.SMC(gsys, np.tile(data, (3, 1)), I.EPS_AN, I.EPS_MN, n_particles=st.n_particles, n_soundings=3,
                   kappa_max=st.kappa_max, lambda_max=st.lambda_max, zmax=st.zmax, seed=st.seed, r_max=st.r_max,
                   **GRAPH_MODES[mode])
        sm.init()
        t0 = time.perf_counter()
        if graph:
            stages = sm.run_graph(max_stages=200, n_sweeps=n_sweeps)
        else:
            stages = sm.run(max_stages=200, n_sweeps=n_sweeps)
        dt = time.perf_counter() - t0
        p = sm.get_particles(0)
        post, lb, lz = sm.model_odds()
        extra = {"langevin": lambda: sm.langevin_stats()[2],
                 "adaptive_recycling_zca": lambda: sm.adaptation()["scale"],
                 "app_b_sweeps": lambda: sm.stats()["accepted"]}.get(mode, lambda: 0)()
        runs.append((stages, p, sm.stats()["gamma"], lz, dt, extra))
    (s0, p0, g0, z0, t0_, e0), (s1, p1, g1, z1, t1_, e1) = runs
    print(f"\n{mode}: host loop {t0_ * 1e3:.1f} ms, graph {t1_ * 1e3:.1f} ms, {s0} stages")
    assert s0 == s1 and np.all(g1 == 1.0)
    assert np.array_equal(g0, g1) and np.array_equal(z0, z1)
    assert np.array_equal(e0, e1)
    for name in ("kappa", "lam", "phib", "tau", "c", "zc", "phic", "zm", "mv", "ll"):
        assert np.array_equal(getattr(p0, name), getattr(p1, name)), name


def test_graph_equals_host_loop_with_cluster_reweight(S, gsys, data):
    """Few large soundings take the cluster-split reweight step: captured in
    the graph it gives the host loop's results bit for bit."""
    runs = []
    for graph in (False, True):
        st = settings(n_particles=2048, seed=31)
        sm = S.SMC(gsys, np.tile(data, (2, 1)), I.EPS_AN, I.EPS_MN, n_particles=st.n_particles, n_soundings=2,
                   kappa_max=st.kappa_max, lambda_max=st.lambda_max, zmax=st.zmax, seed=st.seed, r_max=st.r_max)
        sm.init()
        stages = sm.run_graph(max_stages=6, n_sweeps=2) if graph else sm.run(max_stages=6, n_sweeps=2)
        p = sm.get_particles(0)
        runs.append((stages, p, sm.stats()["gamma"], sm.model_odds()[2]))
    (s0, p0, g0, z0), (s1, p1, g1, z1) = runs
    assert s0 == s1 == 6
    assert np.array_equal(g0, g1) and np.array_equal(z0, z1)
    for name in ("kappa", "lam", "phib", "tau", "c", "zc", "phic", "zm", "mv", "ll"):
        assert np.array_equal(getattr(p0, name), getattr(p1, name)), name


def test_graph_capped_run(S, gsys, data):
    # a capped run stops after max_stages
    sm = gpu_smc(S, gsys, data, settings(n_particles=256, seed=21), soundings=3)
    sm.init()
    assert sm.run_graph(max_stages=3, n_sweeps=2) == 3
