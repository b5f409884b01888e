"""Failure handling through the C ABI, made on the host with no GPU fault:

* non-finite likelihoods: particles with NaN parameters evaluate to NaN, the
  sampler sets them to -inf (zero weight, rejected as proposals) and counts
  them per sounding, and the stage goes on;
* an unbracketable tempering step: more than (1 - alpha) N particles at
  ll = -inf, so no positive step keeps TESS >= alpha N: AEM_ERR_NO_BRACKET
  from smc_reweight, smc_run and smc_run_graph;
* a sounding with no finite likelihood at all: AEM_ERR_NONFINITE, gamma kept;
* the tensor-core transform's bounded wait: the diagnostic switch makes each
  CTA issue no MMA for its first tile and poll a few times, so the wait runs
  out with nothing in flight; the kernel records AEM_ERR_TIMEOUT in the
  status word, frees its tensor memory and returns, and later calls work."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import rjsmc as R
from paper_2109_00661_gb300 import inputs as I
from parity_util import oracle_system

pytestmark = pytest.mark.gpu

NAME = "sounding-g20-f40-k120"
ERR_NONFINITE, ERR_TIMEOUT, ERR_NO_BRACKET = -3, -4, -5


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2109_00661_gb300 as L
    from paper_2109_00661_gb300 import smc as S
    gsys = L.System(**I.system_kwargs(NAME))
    data = I.noisy(O.forward(I.truth_3layer(), oracle_system(NAME), mode=O.HANKEL_RULE)[0], seed=0)
    return torch, L, S, gsys, data


def sampler(S, gsys, data, N=256, soundings=1, **kw):
    return S.SMC(gsys, np.tile(data, (soundings, 1)), I.EPS_AN, I.EPS_MN, n_particles=N, n_soundings=soundings,
                 kappa_max=3, lambda_max=4, seed=3, r_max=10, **kw)


def test_nan_parameters_forward_and_loglik(env):
    """The standalone forward model passes NaN through (only that model's
    outputs), the other models' results are unchanged."""
    torch, L, S, gsys, data = env
    models = I.random_models(64, seed=4, layers_max=6)
    ref = L.loglik_f32(gsys, I.to_torch(models, torch.float32), data, I.EPS_AN, I.EPS_MN).cpu().numpy()
    bad = {k: np.array(v, copy=True) for k, v in models.items()}
    bad["logsig"][5, 0] = np.nan
    bad["m"][9, :] = np.nan
    got = L.loglik_f32(gsys, I.to_torch(bad, torch.float32), data, I.EPS_AN, I.EPS_MN).cpu().numpy()
    assert np.isnan(got[5]) and np.isnan(got[9])
    keep = np.ones(64, bool)
    keep[[5, 9]] = False
    assert np.array_equal(got[keep], ref[keep])


def test_sampler_maps_nonfinite_to_minus_inf(env):
    torch, L, S, gsys, data = env
    sm = sampler(S, gsys, data, N=256, soundings=2)
    sm.init()
    p = sm.get_particles(0)
    bad = [3, 17, 300]  # two in sounding 0, one in sounding 1
    p.phib[bad] = np.nan
    sm.set_particles(p)
    sm.loglik_current()
    q = sm.get_particles(0)
    assert np.all(q.ll[bad] == -np.inf)
    assert np.all(np.isfinite(np.delete(q.ll, bad)))
    status, nonfinite = sm.status()
    assert status == 0 and list(nonfinite) == [2, 1]
    # the stage goes on: the -inf particles get no weight and are resampled away
    g = sm.reweight()
    assert np.all(g > 0)
    sm.resample()
    r = sm.get_particles(0)
    assert np.all(np.isfinite(r.ll)) and not np.any(np.isnan(r.phib))
    sm.mutate(2)
    assert sm.status()[0] == 0


def minus_inf_population(S, gsys, data, frac, soundings=1, N=200):
    sm = sampler(S, gsys, data, N=N, soundings=soundings)
    sm.init()
    p = sm.get_particles(0)
    rng = np.random.default_rng(0)
    for s in range(soundings):
        idx = s * N + rng.choice(N, int(round(frac * N)), replace=False)
        p.ll[idx] = -np.inf
    sm.set_particles(p)
    return sm


# N = 200: one CTA per sounding; N = 2048: the cluster-split reweight step
@pytest.mark.parametrize("N", [200, 2048])
def test_unbracketable_step_reports_no_bracket(env, N):
    """60 % of the particles at ll = -inf: TESS(dgamma) <= 0.4 N < alpha N for
    every dgamma > 0."""
    torch, L, S, gsys, data = env
    sm = minus_inf_population(S, gsys, data, 0.6, N=N)
    with pytest.raises(L.AEMError) as ei:
        sm.reweight()
    assert ei.value.code == ERR_NO_BRACKET
    g = sm.stats()["gamma"][0]
    assert 0.0 < g < 1e-15  # the smallest probed step, (1 - gamma) 2^-60
    assert sm.status()[0] == 0  # reported once, then cleared
    # 40 % at -inf is still bracketable
    ok = minus_inf_population(S, gsys, data, 0.4, N=N)
    assert ok.reweight()[0] > 0.0


@pytest.mark.parametrize("graph", [False, True])
def test_run_stops_on_no_bracket(env, graph):
    torch, L, S, gsys, data = env
    sm = minus_inf_population(S, gsys, data, 0.6)
    with pytest.raises(L.AEMError) as ei:
        if graph:
            sm.run_graph(max_stages=50, n_sweeps=2)
        else:
            sm.run(max_stages=50, n_sweeps=2)
    assert ei.value.code == ERR_NO_BRACKET
    assert sm.stats()["stage"] == 1


@pytest.mark.parametrize("N", [200, 2048])
def test_sounding_without_finite_likelihood_reports_nonfinite(env, N):
    torch, L, S, gsys, data = env
    sm = minus_inf_population(S, gsys, data, 1.0, soundings=2, N=N)
    p = sm.get_particles(0)
    p.ll[N:] = np.random.default_rng(1).normal(-100.0, 5.0, N)  # sounding 1 is healthy
    sm.set_particles(p)
    with pytest.raises(L.AEMError) as ei:
        sm.reweight()
    assert ei.value.code == ERR_NONFINITE
    g = sm.stats()["gamma"]
    assert g[0] == 0.0 and g[1] > 0.0


def test_tensor_core_wait_timeout_is_reported(env):
    torch, L, S, gsys, data = env
    sysg = L.System(**I.system_kwargs("forward-g30-f60-k200"))
    models = I.random_models(1000, seed=2, layers_max=5)
    imh = L.spectrum_f32(sysg, I.to_torch(models, torch.float32))
    ref, _ = L.gates_from_spectrum(sysg, imh, L.GATES_TF32_SPLIT)
    assert L.system_status(sysg) == 0
    L.debug_bounded_wait(sysg, spins=16, skip_first_mma=True)
    try:
        L.gates_from_spectrum(sysg, imh, L.GATES_TF32_SPLIT)
        torch.cuda.synchronize()
        assert L.system_status(sysg) == ERR_TIMEOUT
        assert L.system_status(sysg) == 0  # read and cleared
    finally:
        L.debug_bounded_wait(sysg, spins=0, skip_first_mma=False)
    # the context is intact: the same call again gives the same gates
    again, _ = L.gates_from_spectrum(sysg, imh, L.GATES_TF32_SPLIT)
    assert torch.equal(again, ref)
    assert L.system_status(sysg) == 0
    with pytest.raises(L.AEMError):
        L.debug_bounded_wait(sysg, spins=0, skip_first_mma=2)
