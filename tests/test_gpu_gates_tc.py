"""The gate transform on the tensor cores (TF32 and BF16 high/low splits,
tcgen05) and on the CUDA cores (FP32), through the C ABI.

* arithmetic: on the GPU's own FP32 spectra, every gate is within the split's
  derived bound of the FP64 product with the same (float) transform table:
  |y - y64| <= c * sum_f |T_gf| |x_f| with, per term, the operand residual of
  the split and the dropped low x low product (3 u^2 for unit roundoff u of
  the input type: TF32 u = 2^-11, BF16 u = 2^-8) plus FP32 accumulation of
  3 F + 1 terms, or (F + 1) 2^-24 for the FP32 path; ragged and empty batches;
* likelihood: the epilogue's ll (FP32 terms, compensated sum) equals the
  oracle's FP64 likelihood of the returned gates within the terms' rounding;
* against the oracle on a 4096-model subset of the throughput workload: the
  forward bound of the FP32 path with the split's per-term coefficient."""
import numpy as np
import pytest

import oracle as O
from paper_2109_00661_gb300 import inputs as I
from parity_util import DELTA_S32, DELTA_T, ll_terms32_tol, oracle_ref, oracle_system

pytestmark = pytest.mark.gpu

NAME = "forward-g30-f60-k200"
MODES = {"fp32": 0, "tf32": 1, "bf16": 2}


def coef(mode, F):
    acc = (3 * F + 1) * 2.0 ** -24
    if mode == "fp32":
        return (F + 1) * 2.0 ** -24
    u = 2.0 ** -11 if mode == "tf32" else 2.0 ** -8
    return 3 * u * u + acc


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2109_00661_gb300 as L
    sysg = L.System(**I.system_kwargs(NAME))
    T32 = sysg.tables()[3].astype(np.float32).astype(np.float64)
    return torch, L, sysg, T32


def spectra(torch, L, sysg, P, seed):
    m = I.random_models(P, seed=seed, layers_max=6)
    for k in ("logsig", "logh", "m", "logtau", "c"):
        m[k] = m[k].astype(np.float32).astype(np.float64)
    return m, L.spectrum_f32(sysg, I.to_torch(m, torch.float32))


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("P", [1, 128, 129, 300])
def test_transform_arithmetic(env, mode, P):
    torch, L, sysg, T32 = env
    _, imh = spectra(torch, L, sysg, P, seed=P)
    gates, _ = L.gates_from_spectrum(sysg, imh, MODES[mode])
    x = imh.cpu().numpy().astype(np.float64)
    y64 = x @ T32.T
    scale = np.abs(x) @ np.abs(T32).T
    e = np.abs(gates.cpu().numpy().astype(np.float64) - y64)
    r = e / (coef(mode, sysg.F) * scale)
    print(f"\n{mode} P={P}: max error / bound {r.max():.3f}, max error / scale {np.max(e / scale):.2e}")
    assert r.max() <= 1.0
    assert L.system_status(sysg) == 0


def test_empty_batch(env):
    torch, L, sysg, _ = env
    imh = torch.empty((0, sysg.F), dtype=torch.float32, device="cuda")
    for mode in MODES.values():
        g, _ = L.gates_from_spectrum(sysg, imh, mode)
        assert g.shape == (0, sysg.G)


@pytest.mark.parametrize("mode", list(MODES))
def test_likelihood_epilogue(env, mode):
    torch, L, sysg, _ = env
    s = oracle_system(NAME)
    y_obs = I.noisy(O.forward(I.truth_3layer(), s, mode=O.HANKEL_RULE)[0], seed=0)
    _, imh = spectra(torch, L, sysg, 777, seed=5)
    g, ll = L.gates_from_spectrum(sysg, imh, MODES[mode], y_obs, I.EPS_AN, I.EPS_MN)
    yh = g.cpu().numpy().astype(np.float64)
    ref = O.loglik(yh, y_obs, I.EPS_AN, I.EPS_MN)
    # FP32 terms (r from the datum's float pair), summed by TwoSum
    tol = ll_terms32_tol(yh, y_obs)
    err = np.abs(ll.cpu().numpy() - ref)
    print(f"\n{mode}: ll error max {err.max():.2e}, max error / tolerance {np.max(err / tol):.3f}")
    assert np.all(err <= tol)


@pytest.mark.parametrize("mode", list(MODES))
def test_against_oracle_4096(env, mode):
    """Per-gate error of the FP32 forward model with each transform against
    the oracle (same discretisation) on 4096 models of the throughput
    workload, relative to max(|y|, eps_an): the FP32 path's bound with the
    transform's per-term coefficient, 1e-4 (TF32, FP32) or 1e-3 (BF16) floor."""
    torch, L, sysg, _ = env
    s = oracle_system(NAME)
    y_obs = I.noisy(O.forward(I.truth_3layer(), s, mode=O.HANKEL_RULE)[0], seed=0)
    models = I.random_models(4096, seed=31)
    for k in ("logsig", "logh", "m", "logtau", "c"):
        models[k] = models[k].astype(np.float32).astype(np.float64)
    ll, g = L.loglik_f32_tc(sysg, I.to_torch(models, torch.float32), y_obs, I.EPS_AN, I.EPS_MN, MODES[mode],
                            want_gates=True)
    y, _, _, kap = oracle_ref(models, NAME)
    e = np.abs(g.cpu().numpy().astype(np.float64) - y) / np.maximum(np.abs(y), I.EPS_AN)
    floor = 1e-3 if mode == "bf16" else 1e-4
    bound = floor + kap[2] * DELTA_S32 + kap[0] * coef(mode, sysg.F) + kap[1] * DELTA_T
    print(f"\n{mode}: per-gate error max {e.max():.2e} median {np.median(e):.2e}; "
          f"within {floor:g}: {np.mean(e <= floor):.4f}; max error / bound {np.max(e / bound):.3f}")
    assert np.all(e <= bound)


def test_benchmark_step_equals_loglik_tc(env):
    """The benchmark's step (spectra into a caller's buffer, then the TF32-split
    transform writing the likelihood into a caller's buffer) equals
    aem_loglik_f32_tc bit for bit."""
    torch, L, sysg, _ = env
    s = oracle_system(NAME)
    y_obs = I.noisy(O.forward(I.truth_3layer(), s, mode=O.HANKEL_RULE)[0], seed=0)
    models = I.to_torch(I.random_models(2000, seed=41), torch.float32)
    imh = torch.empty((2000, sysg.F), dtype=torch.float32, device="cuda")
    ll = torch.empty(2000, dtype=torch.float64, device="cuda")
    assert L.spectrum_f32(sysg, models, out=imh) is imh
    _, ll2 = L.gates_from_spectrum(sysg, imh, L.GATES_TF32_SPLIT, y_obs, I.EPS_AN, I.EPS_MN, want_gates=False,
                                   ll_out=ll)
    assert ll2 is ll
    ref = L.loglik_f32_tc(sysg, models, y_obs, I.EPS_AN, I.EPS_MN, L.GATES_TF32_SPLIT)
    assert torch.equal(ll, ref)
    with pytest.raises(L.AEMError):
        L.spectrum_f32(sysg, models, out=imh[:10])
