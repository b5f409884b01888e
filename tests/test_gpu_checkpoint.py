"""smc_checkpoint / smc_restore: resuming from an image reproduces the
uninterrupted sampler exactly (counter-based random streams and
deterministic kernels), and damaged or mismatched images are refused."""
import numpy as np
import pytest

import oracle as O
from paper_2109_00661_gb300 import inputs as I
from parity_util import oracle_system

pytestmark = pytest.mark.gpu

NAME = "sounding-g20-f40-k120"


@pytest.fixture(scope="module")
def env():
    import paper_2109_00661_gb300 as L
    from paper_2109_00661_gb300 import smc as S
    gsys = L.System(**I.system_kwargs(NAME))
    s = oracle_system(NAME)
    data = I.noisy(O.forward(I.truth_3layer(), s, mode=O.HANKEL_RULE)[0], seed=0)
    return S, gsys, np.stack([data, I.noisy(O.forward(I.truth_3layer(), s, mode=O.HANKEL_RULE)[0], seed=1)])


def make(S, gsys, data, N=128, **extra):
    return S.SMC(gsys, data, I.EPS_AN, I.EPS_MN, n_particles=N, n_soundings=2, kappa_max=3, lambda_max=4, seed=21,
                 r_max=6, n_langevin=1, **extra)


# the fixed-scale sampler, and the adaptive proposal with particle recycling
# (3 history slots) and the ZCA-coloured birth / death: the image then carries
# the proposal scales and the recycling history as well
MODES = {"fixed": {}, "adaptive_recycling_zca": dict(adaptive=1, recycle_stages=3, zca=0.5)}


def stages(sm, n):
    for _ in range(n):
        sm.reweight()
        sm.resample()
        sm.mutate(0)  # adaptive R_t: uses the previous stage's acceptance counts


def snapshot(sm):
    p = sm.get_particles(0)
    post, lb, lz = sm.model_odds()
    st = sm.stats()
    acc, prop, h = sm.langevin_stats()
    return dict(kappa=p.kappa, lam=p.lam, phib=p.phib, tau=p.tau, c=p.c, zc=p.zc, phic=p.phic, zm=p.zm, mv=p.mv,
                ll=p.ll, lz=lz, gamma=st["gamma"], stage=st["stage"], acc=st["accepted"], h=h)


@pytest.mark.parametrize("mode", list(MODES))
def test_resume_reproduces_the_uninterrupted_run(env, mode):
    S, gsys, data = env
    a = make(S, gsys, data, **MODES[mode])
    a.init()
    stages(a, 3)
    image = a.checkpoint()
    stages(a, 4)
    ref = snapshot(a)
    if MODES[mode]:
        ref.update(a.adaptation())
    b = make(S, gsys, data, **MODES[mode])
    b.restore(image)
    stages(b, 4)
    got = snapshot(b)
    if MODES[mode]:
        got.update(b.adaptation())
    for k in ref:
        assert np.array_equal(np.asarray(got[k]), np.asarray(ref[k])), k
    assert ref["stage"] == 7


def test_restore_refuses_bad_images(env):
    S, gsys, data = env
    a = make(S, gsys, data)
    a.init()
    image = a.checkpoint()
    with pytest.raises(Exception):
        a.restore(b"XXXX" + image[4:])
    with pytest.raises(Exception):
        a.restore(image[:-8])
    other = make(S, gsys, data, N=64)
    with pytest.raises(Exception):
        other.restore(image)
    adaptive = make(S, gsys, data, adaptive=1, recycle_stages=3)
    with pytest.raises(Exception):  # a sampler with another proposal / history layout
        adaptive.restore(image)
    a.restore(image)  # the intact image still loads
