"""Seeded synthetic inputs shared by the tests, the benchmark and smoke().

This module holds only input recipes (shapes, sizes and value distributions of
the workloads); none of the method's arithmetic lives here.  The paper's VTEM ET
system and Colorado data are not available, so these synthetic soundings stand
in for them with the paper's shapes: off-time gates from 1e-5 to 1e-2 s
(Section 2.3.2), three-layer truths with a chargeable second layer (Section 4.1),
and log-uniform layer properties within the prior bounds of Section 2.3.1.
"""
from __future__ import annotations

import numpy as np

# Geometry of every workload: central loop, radius 13 m, at 30 m height.
LOOP_RADIUS = 13.0
HEIGHT = 30.0
F_MIN_HZ = 1.0
F_MAX_HZ = 1e7

# name: (gates G, frequencies F, Hankel points K)
CONFIGS = {
    "sounding-g20-f40-k120": dict(G=20, F=40, K=120),
    "forward-g30-f60-k200": dict(G=30, F=60, K=200),
}

EPS_MN = 0.03   # 3% multiplicative noise
EPS_AN = 1e-13  # additive floor, T/s for a 1 A transmitter


def gate_times(G):
    return np.logspace(-5, -2, G)


def system_kwargs(name):
    c = CONFIGS[name]
    return dict(loop_radius=LOOP_RADIUS, height=HEIGHT, current=1.0, n_freq=c["F"], f_min_hz=F_MIN_HZ,
                f_max_hz=F_MAX_HZ, gate_times=gate_times(c["G"]), n_hankel=c["K"])


def oracle_system(name, cc_form=0):
    """The same system as a plain dict for the oracle."""
    c = CONFIGS[name]
    freqs = np.exp(np.linspace(np.log(F_MIN_HZ), np.log(F_MAX_HZ), c["F"]))
    return dict(a=LOOP_RADIUS, h=HEIGHT, freqs=freqs, times=gate_times(c["G"]), K=c["K"], cc_form=cc_form,
                current=1.0)


def random_models(P, seed=0, lmax=10, lmin=1, layers_max=10):
    """Forward-throughput workload: layer counts uniform in lmin..layers_max,
    sigma log-uniform 1e-4..1 S/m, thickness log-uniform 2..200 m, m U(0,1),
    tau log-uniform 1e-6..1e-1 s, c U(0.1,1), drawn per layer (float64)."""
    rng = np.random.default_rng(seed)
    nl = rng.integers(lmin, layers_max + 1, size=P).astype(np.int8)
    shape = (P, lmax)
    return dict(
        nlayers=nl,
        logsig=rng.uniform(-4.0, 0.0, shape),
        logh=rng.uniform(np.log10(2.0), np.log10(200.0), shape),
        m=rng.uniform(0.0, 1.0, shape),
        logtau=rng.uniform(-6.0, -1.0, shape),
        c=rng.uniform(0.1, 1.0, shape),
    )


def contrast_models(P, seed=0, lmax=10):
    """Stacks that stress a depth cutoff: ten layers whose conductivities
    alternate between the prior's bounds (1e-4 and 1 S/m, the resistive one on
    top in half of them), thicknesses all at 2 m, all at 200 m or
    log-uniform, and chargeabilities 0 or up to 0.95 (float64)."""
    rng = np.random.default_rng(seed)
    n = np.arange(lmax)
    top = rng.integers(0, 2, size=P)
    logsig = np.where((n[None, :] + top[:, None]) % 2 == 0, -4.0, 0.0)
    kind = rng.integers(0, 3, size=P)
    logh = np.where(kind[:, None] == 0, np.log10(2.0),
                    np.where(kind[:, None] == 1, np.log10(200.0), rng.uniform(np.log10(2.0), np.log10(200.0), (P, lmax))))
    charge = rng.integers(0, 2, size=P)
    return dict(
        nlayers=np.full(P, lmax, dtype=np.int8),
        logsig=logsig,
        logh=logh,
        m=np.where(charge[:, None] == 1, rng.uniform(0.5, 0.95, (P, lmax)), 0.0),
        logtau=rng.uniform(-6.0, -1.0, (P, lmax)),
        c=rng.uniform(0.1, 1.0, (P, lmax)),
    )


def truth_3layer():
    """Single-sounding truth: sigma (0.01, 0.1, 0.01) S/m, thicknesses (20, 30) m,
    Cole-Cole IP in layer 2 with m = 0.3, tau = 1e-3 s, c = 0.5."""
    return dict(
        nlayers=np.array([3], dtype=np.int8),
        logsig=np.log10([[0.01, 0.1, 0.01]]),
        logh=np.log10([[20.0, 30.0, 1.0]]),
        m=np.array([[0.0, 0.3, 0.0]]),
        logtau=np.full((1, 3), -3.0),
        c=np.full((1, 3), 0.5),
    )


def truth_marginal():
    """Weakly chargeable sounding (the evidence for IP near even): the
    three-layer earth of truth_3layer with its second layer 30 m thick from
    50 m depth and chargeability m = 0.1 (tau = 1e-3 s, c = 0.5)."""
    return dict(
        nlayers=np.array([3], dtype=np.int8),
        logsig=np.log10([[0.01, 0.1, 0.01]]),
        logh=np.log10([[50.0, 30.0, 1.0]]),
        m=np.array([[0.0, 0.1, 0.0]]),
        logtau=np.full((1, 3), -3.0),
        c=np.full((1, 3), 0.5),
    )


def truth_5layer():
    """Larger truth: sigma (0.01, 0.1, 0.003, 0.03, 0.01) S/m, h (15, 20, 30, 40) m,
    chargeable layers 2 and 4 with m (0.4, 0.2), tau 4.07e-4 s, c 1.0."""
    return dict(
        nlayers=np.array([5], dtype=np.int8),
        logsig=np.log10([[0.01, 0.1, 0.003, 0.03, 0.01]]),
        logh=np.log10([[15.0, 20.0, 30.0, 40.0, 1.0]]),
        m=np.array([[0.0, 0.4, 0.0, 0.2, 0.0]]),
        logtau=np.full((1, 5), np.log10(4.07e-4)),
        c=np.ones((1, 5)),
    )


def noisy(y_true, seed=0, eps_an=EPS_AN, eps_mn=EPS_MN):
    """Observed data: the truth plus zero-mean Gaussian noise whose standard
    deviation adds eps_an and eps_mn * |y| in quadrature."""
    rng = np.random.default_rng(seed)
    y_true = np.asarray(y_true, dtype=np.float64)
    sd = np.sqrt(eps_an ** 2 + (eps_mn * y_true) ** 2)
    return y_true + sd * rng.standard_normal(y_true.shape)


def to_torch(models, dtype, device="cuda"):
    import torch
    out = {"nlayers": torch.as_tensor(np.asarray(models["nlayers"], dtype=np.int8), device=device)}
    for k in ("logsig", "logh", "m", "logtau", "c"):
        out[k] = torch.as_tensor(np.ascontiguousarray(models[k]), dtype=dtype, device=device).contiguous()
    return out


def subset(models, idx):
    return {k: np.asarray(v)[idx] for k, v in models.items()}


DETECT_BASEMENTS = (0.001, 0.01, 0.032, 0.1)  # S/m: igneous, hard sedimentary, moderate, conductive


def detectability_grid(depths, ms, basement_sigma, tau=4.07e-4, c=1.0):
    """The synthetic detectability study (Section 4.1): a 3-layer earth with
    sigma 0.01 S/m over a 20 m thick chargeable layer of 0.1 S/m whose top is at
    the given depth, over a basement of basement_sigma S/m; Cole-Cole tau and c
    fixed, chargeability m in the second layer only.  One sounding per
    (depth, m) pair, depth-major."""
    D, Mv = np.meshgrid(np.asarray(depths, dtype=np.float64), np.asarray(ms, dtype=np.float64), indexing="ij")
    D, Mv = D.ravel(), Mv.ravel()
    S = D.size
    return dict(
        nlayers=np.full(S, 3, dtype=np.int8),
        logsig=np.tile(np.log10([0.01, 0.1, basement_sigma]), (S, 1)),
        logh=np.stack([np.log10(D), np.full(S, np.log10(20.0)), np.zeros(S)], axis=1),
        m=np.stack([np.zeros(S), Mv, np.zeros(S)], axis=1),
        logtau=np.full((S, 3), np.log10(tau)),
        c=np.full((S, 3), c),
    )


def flight_line(n_soundings):
    """Synthetic flight line: sounding s at x = s / (S - 1) over a 3-layer earth
    (sigma 0.01, 0.1, 0.01 S/m) whose chargeable second layer (30 m thick,
    tau = 1e-3 s, c = 0.5) starts at depth 50 - 30 cos(2 pi x) m (20..80 m)
    with chargeability 0.25 (1 - cos(2 pi x)) (0..0.5)."""
    S = n_soundings
    x = np.arange(S) / max(S - 1, 1)
    depth = 50.0 - 30.0 * np.cos(2 * np.pi * x)
    m = 0.25 * (1.0 - np.cos(2 * np.pi * x))
    return dict(
        nlayers=np.full(S, 3, dtype=np.int8),
        logsig=np.tile(np.log10([0.01, 0.1, 0.01]), (S, 1)),
        logh=np.stack([np.log10(depth), np.full(S, np.log10(30.0)), np.zeros(S)], axis=1),
        m=np.stack([np.zeros(S), m, np.zeros(S)], axis=1),
        logtau=np.full((S, 3), -3.0),
        c=np.full((S, 3), 0.5),
    ), x
