"""Posterior predictive summaries of the CUDA sampler (smc_ppd) against the
oracle's ppd_summary: the reductions themselves on the GPU's own
predictions (to rounding), and against the oracle's FP64 predictions of the
same particles within the FP32 forward bound propagated through the mean,
the variance and the standardised data."""
import numpy as np
import pytest

import oracle as O
from oracle import rjsmc as R
from paper_2109_00661_gb300 import inputs as I
from parity_util import bound32, kappa, oracle_system

pytestmark = pytest.mark.gpu

NAME = "sounding-g20-f40-k120"


def to_oracle(h, i):
    k, l = int(h.kappa[i]), int(h.lam[i])
    f = lambda v: float(np.float64(v))
    return R.Particle(k, l, f(h.phib[i]), [f(v) for v in h.zc[i, :k]], [f(v) for v in h.phic[i, :k]],
                      [f(v) for v in h.zm[i, :l]], [f(v) for v in h.mv[i, :l]], f(h.tau[i]), f(h.c[i]))


def test_ppd_after_a_run(tmp_path):
    import paper_2109_00661_gb300 as L
    from paper_2109_00661_gb300 import smc as S
    gsys = L.System(**I.system_kwargs(NAME))
    s = oracle_system(NAME)
    y_true = O.forward(I.truth_3layer(), s, mode=O.HANKEL_RULE)[0]
    data = np.stack([I.noisy(y_true, seed=0), I.noisy(y_true, seed=1)])
    N = 256
    sm = S.SMC(gsys, data, I.EPS_AN, I.EPS_MN, n_particles=N, n_soundings=2, kappa_max=3, lambda_max=4, seed=3)
    sm.init()
    sm.run(max_stages=200, n_sweeps=10)
    mean, var, z, gates = sm.ppd(want_gates=True)
    p = sm.get_particles(0)
    for snd in range(2):
        sl = slice(snd * N, (snd + 1) * N)
        yg = gates[sl].astype(np.float64)
        # 1) the reductions, on the GPU's own predictions
        m_ref, v_ref, z_ref = R.ppd_summary(yg, data[snd], I.EPS_AN, I.EPS_MN)
        assert np.allclose(mean[snd], m_ref, rtol=1e-12, atol=0)
        assert np.allclose(var[snd], v_ref, rtol=1e-12, atol=0)
        assert np.allclose(z[snd], z_ref, rtol=1e-10, atol=1e-12)
        # 2) against the oracle's predictions of the same particles
        parts = [to_oracle(p, i) for i in range(sl.start, sl.stop)]
        mb = R.merged_batch(parts, 8)
        y, imh, absh = O.forward(mb, s, mode=O.HANKEL_RULE, want_imh=True, want_absh=True)
        mo, vo, zo = R.ppd_summary(y, data[snd], I.EPS_AN, I.EPS_MN)
        d = bound32(kappa(imh, s["T"], y, absh), s["T"].shape[1]) * np.maximum(np.abs(y), I.EPS_AN)
        dm = d.mean(axis=0)
        dv = (2 * I.EPS_MN ** 2 * np.abs(y) * d + (I.EPS_MN * d) ** 2 + 2 * np.abs(y - mo) * (d + dm)
              + (d + dm) ** 2).mean(axis=0)
        assert np.all(np.abs(mean[snd] - mo) <= dm + 1e-12 * np.abs(mo))
        assert np.all(np.abs(var[snd] - vo) <= dv + 1e-12 * vo)
        dz = dm / np.sqrt(vo) + np.abs(data[snd] - mo) * dv / (2 * vo ** 1.5)
        assert np.all(np.abs(z[snd] - zo) <= 1.01 * dz + 1e-9)
        # how typical the data are of their own posterior predictive is a
        # property of the sampler's convergence, reported rather than asserted
        print(f"\nsounding {snd}: |z| max {np.abs(z[snd]).max():.2f}, median {np.median(np.abs(z[snd])):.2f}")
