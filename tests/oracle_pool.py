"""Independent serial oracle RJSMC runs spread over host processes (a spawn
pool, started before any GPU work in the worker) for the statistical parity
tests: one single-threaded oracle sampler per seed on the same sounding."""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _one(args):
    name, truth_name, noise_seed, kw, seed = args
    import oracle as O
    from oracle import rjsmc as R
    from paper_2109_00661_gb300 import inputs as I
    s = I.oracle_system(name)
    s["T"] = O.tmatrix(s["freqs"], s["times"])
    y = O.forward(getattr(I, truth_name)(), s, mode=O.HANKEL_RULE, nthreads=1)[0]
    data = I.noisy(y, seed=noise_seed)
    st = R.SMCSettings(seed=seed, **kw)
    lik = R.ForwardLik(s, data, I.EPS_AN, I.EPS_MN, lmax=st.kappa_max + st.lambda_max + 1, nthreads=1)
    res = R.run(st, lik)
    post, lb = R.model_odds(res.counts, st.kappa_max, st.lambda_max)
    return post, lb, len(res.gammas)


def oracle_odds(name, truth_name, seeds, noise_seed=0, workers=None, **kw):
    """(post [n_seeds, M], log BFIPD [n_seeds], stages [n_seeds]) of the
    oracle sampler with settings kw, one run per seed."""
    workers = workers or min(len(seeds), os.cpu_count() or 1)
    jobs = [(name, truth_name, noise_seed, kw, int(sd)) for sd in seeds]
    with mp.get_context("spawn").Pool(workers) as pool:
        out = pool.map(_one, jobs)
    return (np.array([o[0] for o in out]), np.array([o[1] for o in out]), np.array([o[2] for o in out]))
