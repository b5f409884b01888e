#!/usr/bin/env python3
"""Benchmark: forward + log-likelihood evaluations per second on the
forward-throughput workload (2^20 synthetic layered models per GPU, 1..10
layers, 30 gates, 60 frequencies, 200 Hankel points), FP32 path.

One step = the forward model over the whole batch (Cole-Cole, TE recursion,
Hankel sums: aem_forward_f32 writing the spectra) then the step-off gate
transform on the tensor cores (TF32 high/low split) with the Gaussian
log-likelihood in its epilogue (aem_gates_from_spectrum), inputs resident in
HBM; the 210 MB of model inputs exceed the 129 MB L2, so each step re-reads
them from HBM.  The fused form (gates and likelihood in the forward kernel's
own epilogue, aem_loglik_f32) is reported beside it.  `e2e` times the same
calls with the inputs copied from pinned host memory and the
log-likelihoods copied back inside the timed region.

--impl reference times the FP64 CPU oracle (the comparison arm for this
build) on a bounded sample of the same workload on the host cores.

Multi-GPU: every rank evaluates its own 2^20 models (weak scaling, no
collective on the data path); value = all ranks' models / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "forward-g30-f60-k200"
P_PER_GPU = 1 << 20
FLOPS_PER_LAYER_STEP = 60  # FP32 flops (FMA = 2) per layer-step of the recursion, counted from forward.cu
MUFU_PER_LAYER_STEP = 6    # sqrt(|w|), rsqrt, rcp, ex2, sin, cos
# the adjoint's FP32 flops per layer-step, counted from adjoint.cu: the
# bottom-up recomputation of the reflection coefficients (60) and the
# top-down reverse sweep (170: the wavenumber, interface coefficient and
# propagation factor again, the Moebius step's partial derivatives, the
# adjoint recursion and the per-layer accumulation)
ADJ_FLOPS_PER_LAYER_STEP = 230
ACCURACY_MODELS = 4096     # subset of the batch on which each variant's per-gate error is measured
DEPTH_CUTOFF = 20.0        # the forward kernel's default (aem_system_set_depth_cutoff)
K_PARAM_BYTES = 201        # per model in: 5 float parameters x 10 layers + the int8 layer count
# DRAM bytes (read 218.59 MB + write 210.84 MB) of one spectrum-writing
# forward launch of the 256 x 3 dynamic-scheduled shape on 1,048,576 models of
# this workload, from an ncu capture (dram__bytes_read.sum and
# dram__bytes_write.sum, one pass); spectra still dirty in L2 when the launch
# ends are written back after it and are not counted
SPECTRUM_LAUNCH_BYTES_1M = 219.61e6 + 210.86e6
METRIC = "forward+loglik evals/s"
UNIT = "evals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--models", type=int, default=P_PER_GPU)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-rjsmc", action="store_true")
    ap.add_argument("--no-flight-line", action="store_true",
                    help="skip the 1000-sounding flight line (about 25 s) of the default run")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the FP64 form, gate-transform variants, bucketed order and adjoint measurements")
    ap.add_argument("--rjsmc-only", nargs="?", const="fixed", choices=["fixed", "adaptive", "large", "fp64"],
                    help="run only one RJSMC measurement (profiling): 128 x 256 with the fixed-scale moves or the "
                         "adaptive proposal with recycling and ZCA moves; 4 x 4096 with kappa, lambda <= 9 and "
                         "20 sweeps (large); 16 x 256 with the plain FP64 forward model (fp64)")
    ap.add_argument("--convergence-study", action="store_true",
                    help="fraction of soundings whose best particle reaches the truth's likelihood level, per "
                         "sampler setting (8 soundings of the 3-layer data, 2 seeds)")
    ap.add_argument("--detectability", action="store_true",
                    help="run only the synthetic detectability study: log BFIPD over layer depth x chargeability "
                         "for the four basement conductivities, all soundings in one sampler")
    ap.add_argument("--flight-line", type=int, default=0, metavar="S",
                    help="run only the flight-line sampler: S soundings x 2048 particles in one sampler")
    ap.add_argument("--layer-sweep", default="", metavar="L1,L2,...",
                    help="run only the forward kernel's cost per layer count: 65,536 models of exactly L layers "
                         "each on the throughput system, in the autotuned launch shape, one log-likelihood "
                         "launch per count after warm-up (the intercept is the per-item and per-model work)")
    args = ap.parse_args()
    if args.layer_sweep:
        try:
            counts = [int(x) for x in args.layer_sweep.split(",") if x]
        except ValueError:
            counts = []
        if not counts or any(not 1 <= n <= 10 for n in counts):
            ap.error("--layer-sweep: comma-separated layer counts in 1..10 (the workload's row stride)")
    return args


def layer_sweep(torch, L, I, counts, steps):
    """ms per launch of loglik_f32 on 65,536 models of exactly n layers, for
    each n in counts, and the least-squares line through them."""
    import numpy as np
    sysg = L.System(**I.system_kwargs(WORKLOAD))
    y_obs = np.full(sysg.G, 1e-11)
    P = 1 << 16
    sysg.autotune(I.to_torch(I.random_models(P, seed=0), torch.float32), repeats=2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = []
    for n in counts:
        m = I.to_torch(I.random_models(P, seed=5, lmin=n, layers_max=n), torch.float32)
        for _ in range(3):
            L.loglik_f32(sysg, m, y_obs, I.EPS_AN, I.EPS_MN)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            L.loglik_f32(sysg, m, y_obs, I.EPS_AN, I.EPS_MN)
        e1.record()
        torch.cuda.synchronize()
        out.append({"layers": n, "ms_per_launch": e0.elapsed_time(e1) / steps})
    res = {"workload": WORKLOAD, "models": P, "per_layer_count": out}
    if len(out) > 1:
        slope, icpt = np.polyfit([o["layers"] for o in out], [o["ms_per_launch"] for o in out], 1)
        res["fit_ms"] = {"intercept": float(icpt), "per_layer": float(slope)}
    return res


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def layer_steps(nlayers, F, K):
    return float(np.sum(nlayers.astype(np.int64))) * F * K


def cpu_baseline(accuracy_models, y_obs_np, target_seconds=15.0):
    """The FP64 oracle (adaptive-quadrature Hankel integrals), as it stands, on
    a bounded sample of the workload on this host's cores; the oracle with the
    GPU's discretisation (K-point rule) on the accuracy subset of the batch,
    whose gates and spectra are returned as the reference the variants' per-gate
    errors are measured against; the serial oracle RJSMC of the single-sounding
    configuration."""
    import oracle as O
    from paper_2109_00661_gb300 import inputs as I
    so = I.oracle_system(WORKLOAD)
    so["T"] = O.tmatrix(so["freqs"], so["times"])
    cores = os.cpu_count() or 1
    n = 64
    done, elapsed = 0, 0.0
    while elapsed < target_seconds:
        models = I.random_models(n, seed=1000 + done)
        t0 = time.perf_counter()
        y = O.forward(models, so, nthreads=cores)
        O.loglik(y, y_obs_np, I.EPS_AN, I.EPS_MN)
        elapsed += time.perf_counter() - t0
        done += n
        n = min(n * 2, 4096)
    # the same discretisation as the GPU (the K-point Hankel rule) in FP64 on
    # the same cores, on the accuracy subset (the models rounded to float32,
    # as the FP32 path sees them): the fair CPU form of the forward model
    m32 = {k: (np.asarray(v, dtype=np.float32).astype(np.float64) if k != "nlayers" else v)
           for k, v in accuracy_models.items()}
    t0 = time.perf_counter()
    y_ref, imh_ref, absh = O.forward(m32, so, mode=O.HANKEL_RULE, nthreads=cores, want_imh=True, want_absh=True)
    O.loglik(y_ref, y_obs_np, I.EPS_AN, I.EPS_MN)
    el_r = time.perf_counter() - t0
    done_r = len(m32["nlayers"])
    # the serial oracle RJSMC of the single-sounding configuration (N = 256,
    # kappa <= 3, lambda <= 4, 10 sweeps per stage): prior draw plus one stage,
    # extrapolated to the stage count the GPU sampler takes on it (30)
    from oracle import rjsmc as R
    ss = I.oracle_system("sounding-g20-f40-k120")
    ss["T"] = O.tmatrix(ss["freqs"], ss["times"])
    y1 = I.noisy(O.forward(I.truth_3layer(), ss, mode=O.HANKEL_RULE)[0], seed=0)
    lik = R.ForwardLik(ss, y1, I.EPS_AN, I.EPS_MN, lmax=8)
    st = R.SMCSettings(n_particles=256, kappa_max=3, lambda_max=4, n_sweeps=10, seed=0)
    t0 = time.perf_counter()
    parts = [R.sample_prior(st, i) for i in range(st.n_particles)]
    lik(parts)
    t_init = time.perf_counter() - t0
    t0 = time.perf_counter()
    R.run(st, lik, max_stages=1)
    t_stage = time.perf_counter() - t0 - t_init
    out = {"value": done / elapsed, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{done} models of the {WORKLOAD} workload (adaptive-quadrature FP64 oracle, "
                     f"{cores} threads), {elapsed:.1f} s",
           "same_discretisation": {"value": done_r / el_r, "unit": UNIT, "cores": cores,
                                   "sample": f"the first {done_r} models of the batch, FP64 oracle with the GPU's "
                                             f"{WORKLOAD.split('-k')[-1]}-point Hankel rule, {el_r:.2f} s"},
           "rjsmc": {"value": 1.0 / (t_init + 30 * t_stage), "unit": "soundings/s", "cores": cores,
                     "sample": f"serial oracle RJSMC, 256 particles, kappa<=3, lambda<=4, 10 sweeps/stage: prior "
                               f"draw {t_init:.2f} s + one stage {t_stage:.2f} s, extrapolated to 30 stages"}}
    return out, (y_ref, imh_ref, absh, so["T"])


def gate_errors(gates, ref, floor):
    """Per-gate error statistics of one variant against the oracle's gates on
    the accuracy subset: e = |gpu - oracle| / max(|oracle|, eps_an); the
    well-conditioned gates are those whose unavoidable error is below the
    floor: FP32 rounding of the spectrum and the transform, kappa_g (F + 1)
    2^-24, plus the 1e-8 (of each row's largest entry) by which the two
    independently built transform tables differ, kappa_T 1e-8."""
    from paper_2109_00661_gb300 import inputs as I
    y_ref, imh_ref, _, T = ref
    den = np.maximum(np.abs(y_ref), I.EPS_AN)
    e = np.abs(np.asarray(gates, dtype=np.float64) - y_ref) / den
    kap = (np.abs(imh_ref) @ np.abs(T).T) / den
    kap_t = np.sum(np.abs(imh_ref), axis=1, keepdims=True) * np.max(np.abs(T), axis=1)[None, :] / den
    good = kap * (T.shape[1] + 1) * 2.0 ** -24 + kap_t * 1e-8 < floor
    return {"max": float(e.max()), "median": float(np.median(e)), "p99": float(np.quantile(e, 0.99)),
            "floor": floor, "frac_within_floor": float(np.mean(e <= floor)),
            "well_conditioned_frac": float(good.mean()),
            "well_conditioned_within_floor": float(np.mean(e[good] <= floor)),
            "models": int(y_ref.shape[0])}


def json_num(v):
    """A float for the JSON line: +-inf as the strings "inf" / "-inf"."""
    v = float(v)
    return v if np.isfinite(v) else ("inf" if v > 0 else "-inf")


def flight_line_measure(torch, L, I, n_soundings, rank=0, world=1, reduce=None):
    """Cfg 5: the synthetic flight line (chargeable layer at 20..80 m, m 0..0.5),
    2048 particles per sounding in one sampler per rank whose stage loop is one
    captured CUDA graph; with several ranks each takes its contiguous block of
    the line's soundings (shard_range).  Soundings/s of the whole job and the
    unclipped log BFIPD at up to 20 evenly spaced soundings of this rank's block."""
    from paper_2109_00661_gb300.shard import shard_range
    truth, x = I.flight_line(n_soundings)
    start, stop = shard_range(n_soundings, rank, world)
    block = I.subset(truth, np.arange(start, stop))
    out = rjsmc_measure(torch, L, I, stop - start, 2048, 3, 4, 10, block, graph=True, per_sounding=True,
                        reduce=reduce, seed=rank, sounding_offset=start)
    lbs = out.pop("log_bfipd_per_sounding")
    step = max(1, (stop - start) // 20)
    out["log_bfipd_along_line"] = {f"{x[start + i]:.3f}": json_num(round(float(lbs[i]), 2))
                                   for i in range(0, stop - start, step)}
    out["soundings_of_rank_0"] = [start, stop] if rank == 0 else None
    return out


def bfipd_summary(lb):
    """Unclipped log BFIPD over soundings: the finite values' median and how
    many soundings had every particle on one side (+-inf)."""
    lb = np.asarray(lb, dtype=np.float64)
    fin = np.isfinite(lb)
    return {"median_finite": float(np.median(lb[fin])) if fin.any() else None, "n_finite": int(fin.sum()),
            "n_all_chargeable": int(np.sum(lb == np.inf)), "n_none_chargeable": int(np.sum(lb == -np.inf))}


def rjsmc_measure(torch, L, I, n_soundings, n_particles, kappa_max, lambda_max, sweeps, truth, seed=0,
                  reduce=None, n_langevin=0, graph=False, adaptive=None, per_sounding=False, precision=0,
                  sounding_offset=0):
    """Whole RJSMC runs (prior draw, then reweight / resample / mutate until
    gamma = 1) for a batch of independent soundings on the sounding system
    (20 gates, 40 frequencies, 120 Hankel points); returns soundings/s.  With
    n_langevin > 0 every stage ends with that many adjoint-driven Langevin
    sweeps (adapted step); adaptive: smc_desc fields of the adaptive proposal
    (fit and scale bisection, recycling window, ZCA mixture); precision 1:
    the plain FP64 forward model in every evaluation."""
    from paper_2109_00661_gb300 import smc as S
    sysg = L.System(**I.system_kwargs("sounding-g20-f40-k120"))
    lms = kappa_max + lambda_max + 1
    sample = I.random_models(min(n_soundings * n_particles, 1 << 15), seed=9, lmax=lms, layers_max=lms)
    shape, _ = sysg.autotune(I.to_torch(sample, torch.float32))
    y_true = L.forward_f32(sysg, I.to_torch(truth, torch.float32)).cpu().numpy().astype(np.float64)
    if y_true.shape[0] == 1:  # one truth for every sounding, independent noise draws
        y_true = np.repeat(y_true, n_soundings, axis=0)
    y_obs = np.stack([I.noisy(y_true[s], seed=1000 + sounding_offset + s) for s in range(n_soundings)])
    sm = S.SMC(sysg, y_obs, I.EPS_AN, I.EPS_MN, n_particles=n_particles, n_soundings=n_soundings,
               kappa_max=kappa_max, lambda_max=lambda_max, seed=seed, r_max=sweeps, n_langevin=n_langevin,
               precision=precision, **(adaptive or {}))
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sm.init()
    stages = sm.run_graph(max_stages=500, n_sweeps=sweeps) if graph else sm.run(max_stages=500, n_sweeps=sweeps)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3
    post, lb, _ = sm.model_odds()
    # every particle at the prior draw and every proposal of every sweep,
    # including the proposals that made no move (an impossible move, about
    # 16 % of them), whose evaluation the forward kernel skips
    evals = n_soundings * n_particles * (1 + stages * sweeps)
    lang = None
    if n_langevin:
        acc, prop, h = sm.langevin_stats()
        lang = {"sweeps_per_stage": n_langevin, "gradient_evals": n_soundings * n_particles * stages * (n_langevin + 1),
                "last_stage_acceptance": float(acc.sum() / max(prop.sum(), 1)), "median_step_h": float(np.median(h))}
    world_soundings = n_soundings
    if reduce is not None:  # ranks run disjoint soundings: sum the work, take the slowest time
        sec, world_soundings, evals = reduce(sec, n_soundings, evals)
    out = {"value": world_soundings / sec, "unit": "soundings/s", "seconds": sec, "stages": stages,
           "ms_per_stage": sec / stages * 1e3, "forward_evals_per_s": evals / sec,
           "config": f"{n_soundings} soundings x {n_particles} particles, kappa<={kappa_max}, lambda<={lambda_max}, "
                     f"{sweeps} sweeps/stage" + (f" + {n_langevin} Langevin sweeps/stage" if n_langevin else "") +
                     (", stages in one CUDA graph with a device-side loop condition" if graph else "") +
                     (", adaptive proposal " + ", ".join(f"{k}={v}" for k, v in adaptive.items()) if adaptive else "") +
                     (", plain FP64 forward model" if precision else "") +
                     ", alpha=0.5, sounding system G=20 F=40 K=120",
           "log_bfipd": bfipd_summary(lb),
           "p_ip_per_model_mean": post.mean(axis=0).round(4).tolist(),
           "forward_launch_shape": shape,
           "langevin": lang,
           "mean_p_ip": float(np.mean(post.reshape(n_soundings, kappa_max + 1, lambda_max + 1)[:, :, 1:].sum(axis=(1, 2))))}
    if per_sounding:  # unclipped; +-inf where every particle sits on one side
        out["log_bfipd_per_sounding"] = lb.tolist()
    sm.close()
    sysg.close()
    return out


def combine_runs(runs):
    """Runs of one RJSMC configuration with different seeds: soundings/s over
    the summed time, with each run's stage count (the number of tempering
    stages follows the path the sampler takes: 23 to 43 over five seeds of the
    4 x 4096 Langevin configuration)."""
    sec = sum(r["seconds"] for r in runs)
    stages = [r["stages"] for r in runs]
    out = dict(runs[0])
    out.update(value=sum(r["value"] * r["seconds"] for r in runs) / sec, seconds=sec, stages=stages,
               ms_per_stage=sec / sum(stages) * 1e3, seeds=len(runs),
               forward_evals_per_s=sum(r["forward_evals_per_s"] * r["seconds"] for r in runs) / sec,
               log_bfipd=[r["log_bfipd"] for r in runs],
               mean_p_ip=float(np.mean([r["mean_p_ip"] for r in runs])))
    if runs[0]["langevin"]:
        out["langevin"] = dict(runs[-1]["langevin"],
                               gradient_evals=sum(r["langevin"]["gradient_evals"] for r in runs))
    return out


def detectability_study(torch, L, I, n_particles=2048):
    """Section 4.1's synthetic study: the 3-layer earth with its chargeable
    second layer (20 m, 0.1 S/m, tau = 4.07e-4 s, c = 1) at 6 depths x 6
    chargeabilities over each of the four basements, 144 soundings in one
    sampler (N per sounding, kappa <= 3, lambda <= 4, 10 sweeps per stage,
    log-uniform tau prior); returns the log BFIPD grid and the timing."""
    from paper_2109_00661_gb300 import smc as S
    depths, ms = [10.0, 20.0, 30.0, 40.0, 60.0, 80.0], [0.0, 0.1, 0.2, 0.3, 0.5, 0.8]
    grids = [I.detectability_grid(depths, ms, b) for b in I.DETECT_BASEMENTS]
    truth = {k: np.concatenate([g[k] for g in grids]) for k in grids[0]}
    n = len(truth["nlayers"])
    sysg = L.System(**I.system_kwargs("sounding-g20-f40-k120"))
    lms = 3 + 4 + 1
    sysg.autotune(I.to_torch(I.random_models(1 << 15, seed=9, lmax=lms, layers_max=lms), torch.float32))
    y = L.forward_f32(sysg, I.to_torch(truth, torch.float32)).cpu().numpy().astype(np.float64)
    y_obs = np.stack([I.noisy(y[s], seed=3000 + s) for s in range(n)])
    sm = S.SMC(sysg, y_obs, I.EPS_AN, I.EPS_MN, n_particles=n_particles, n_soundings=n, kappa_max=3, lambda_max=4,
               seed=0, r_max=10, tau_log_prior=1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    sm.init()
    stages = sm.run(max_stages=500, n_sweeps=10)
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3
    _, lb, _ = sm.model_odds()
    grid = np.clip(lb, -50, 50).reshape(len(I.DETECT_BASEMENTS), len(depths), len(ms))
    return {"depths_m": depths, "chargeability": ms, "basement_S_per_m": list(I.DETECT_BASEMENTS),
            "log_bfipd": np.round(grid, 2).tolist(), "soundings": n, "particles_per_sounding": n_particles,
            "stages": stages, "seconds": sec, "soundings_per_s": n / sec}


def convergence_study(torch, L, I):
    """8 noisy copies of the 3-layer sounding, N = 256, kappa <= 3, lambda <= 4:
    for each sampler setting and seed, the fraction of soundings whose best
    final particle is within 50 of the truth's log-likelihood (both from the
    GPU's FP64 forward model) and the median |z| of the data against the
    posterior predictive."""
    from paper_2109_00661_gb300 import smc as S
    sysg = L.System(**I.system_kwargs("sounding-g20-f40-k120"))
    truth = I.truth_3layer()
    y_true = L.forward_f64(sysg, I.to_torch(truth, torch.float64)).cpu().numpy()[0]
    SN, N = 8, 256
    data = np.stack([I.noisy(y_true, seed=k) for k in range(SN)])
    ll_true = np.array([L.loglik_f64(sysg, I.to_torch(truth, torch.float64), data[k], I.EPS_AN,
                                     I.EPS_MN).cpu().numpy()[0] for k in range(SN)])
    rows = []
    for label, kw, sweeps in (("walk, 10 sweeps", {}, 10), ("adaptive, 10 sweeps", {"adaptive": 1}, 10),
                              ("walk, 20 sweeps", {}, 20), ("adaptive, 20 sweeps", {"adaptive": 1}, 20),
                              ("walk, 40 sweeps", {}, 40), ("adaptive, 40 sweeps", {"adaptive": 1}, 40),
                              ("walk, 10 sweeps, alpha 0.9", {"alpha": 0.9}, 10),
                              ("adaptive, 10 sweeps, alpha 0.9", {"adaptive": 1, "alpha": 0.9}, 10),
                              ("adaptive, 10 sweeps + 2 Langevin", {"adaptive": 1, "n_langevin": 2}, 10),
                              ("adaptive + recycling (8 stages), 10 sweeps", {"adaptive": 1, "recycle_stages": 8}, 10),
                              ("adaptive + recycling (8 stages), 20 sweeps", {"adaptive": 1, "recycle_stages": 8}, 20),
                              ("adaptive + ZCA birth/death (p 0.5), 20 sweeps", {"adaptive": 1, "zca": 0.5}, 20)):
        for seed in (3, 4):
            args = dict(n_particles=N, n_soundings=SN, kappa_max=3, lambda_max=4, seed=seed)
            args.update(kw)
            sm = S.SMC(sysg, data, I.EPS_AN, I.EPS_MN, **args)
            sm.init()
            stages = sm.run(max_stages=400, n_sweeps=sweeps)
            _, _, z = sm.ppd()
            ll = sm.get_particles(0).ll.reshape(SN, N)
            rows.append({"setting": label, "seed": seed, "stages": stages,
                         "converged": float(np.mean(ll.max(axis=1) > ll_true - 50)),
                         "median_abs_z": float(np.median(np.abs(z)))})
            sm.close()
    sysg.close()
    return rows


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    from paper_2109_00661_gb300 import inputs as I
    so = I.oracle_system(WORKLOAD)
    so["T"] = O.tmatrix(so["freqs"], so["times"])
    y_obs = I.noisy(O.forward(I.truth_3layer(), so)[0], seed=0)
    cores = os.cpu_count() or 1
    per_step = 256
    for w in range(args.warmup):
        O.forward(I.random_models(per_step, seed=w), so, nthreads=cores)
    t0 = time.perf_counter()
    for s in range(args.steps):
        y = O.forward(I.random_models(per_step, seed=100 + s), so, nthreads=cores)
        O.loglik(y, y_obs, I.EPS_AN, I.EPS_MN)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: {per_step}-model sample per step of the 2^20-model batch",
                       "models_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} models per step, {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_2109_00661_gb300 as L
    from paper_2109_00661_gb300 import inputs as I
    from paper_2109_00661_gb300.shard import job_throughput

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    if args.detectability:
        print(json.dumps({"detectability": detectability_study(torch, L, I)}), flush=True)
        return
    if args.flight_line:
        print(json.dumps({"flight_line": flight_line_measure(torch, L, I, args.flight_line)}), flush=True)
        return
    if args.convergence_study:
        print(json.dumps({"convergence_study": convergence_study(torch, L, I)}), flush=True)
        return
    if args.layer_sweep:
        counts = [int(x) for x in args.layer_sweep.split(",") if x]
        print(json.dumps({"layer_sweep": layer_sweep(torch, L, I, counts, max(1, args.steps))}), flush=True)
        return
    if args.rjsmc_only:
        if args.rjsmc_only == "large":
            out = rjsmc_measure(torch, L, I, 4, 4096, 9, 9, 20, I.truth_5layer())
        elif args.rjsmc_only == "fp64":
            out = rjsmc_measure(torch, L, I, 16, 256, 3, 4, 10, I.truth_3layer(), precision=1)
        else:
            ad = dict(adaptive=1, recycle_stages=3, zca=0.5) if args.rjsmc_only == "adaptive" else None
            out = rjsmc_measure(torch, L, I, 128, 256, 3, 4, 10, I.truth_3layer(), adaptive=ad)
        print(json.dumps({"rjsmc": out}), flush=True)
        return
    sysg = L.System(**I.system_kwargs(WORKLOAD))
    F, K, G = sysg.F, sysg.K, sysg.G
    P = args.models
    models_np = I.random_models(P, seed=rank)
    models = I.to_torch(models_np, torch.float32)
    # the data every model is scored against: the single-sounding truth (three
    # layers, chargeable second layer) through the FP64 forward model on this
    # system's 30 gates, with 3 % + 1e-13 T/s noise
    y_true = L.forward_f64(sysg, I.to_torch(I.truth_3layer(), torch.float64)).cpu().numpy()[0]
    y_obs_np = I.noisy(y_true, seed=0)
    y_obs = torch.as_tensor(y_obs_np, dtype=torch.float64, device="cuda")
    eps_an = torch.full((G,), I.EPS_AN, dtype=torch.float64, device="cuda")
    ll = torch.empty(P, dtype=torch.float64, device="cuda")
    steps_work = layer_steps(models_np["nlayers"], F, K)
    peaks = L.probe_peaks()
    # launch shape of the forward kernel, picked by the project's autotuner
    # on a 65,536-model sample of the workload before any timing
    shape, shape_ms = sysg.autotune(I.to_torch(I.subset(models_np, np.arange(min(P, 1 << 16))), torch.float32))
    # the share of the whole stack's layer-steps the recursion runs on this
    # batch with the depth cutoff (counted by the kernel, one untimed launch)
    _, kept_frac = L.forward_layer_steps(sysg, models)

    stream = torch.cuda.current_stream()
    # One step: the forward model (Cole-Cole, TE recursion, Hankel sums) writes
    # the spectra of every model, then the gate transform runs on the tensor
    # cores (TF32 high/low split) with the Gaussian log-likelihood in its
    # epilogue: a5 + a6 on tcgen05.  The forward kernel, the dominant one, is
    # timed on its own with events around its launch inside the timed region.
    imh_buf = torch.empty((P, F), dtype=torch.float32, device="cuda")
    ll_buf = torch.empty(P, dtype=torch.float64, device="cuda")
    fwd_events = []

    def step(record=False):
        if record:
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[0].record(stream)
        L.spectrum_f32(sysg, models, stream=stream, out=imh_buf)
        if record:
            ev[1].record(stream)
            fwd_events.append(ev)
        L.gates_from_spectrum(sysg, imh_buf, L.GATES_TF32_SPLIT, y_obs, eps_an, I.EPS_MN, want_gates=False,
                              stream=stream, ll_out=ll_buf)
        return ll_buf

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(record=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    fwd_ms = float(np.mean([a.elapsed_time(b) for a, b in fwd_events]))
    if L.system_status(sysg) != 0:
        raise RuntimeError("the tensor-core transform reported a timeout")
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = job_throughput([P] * world, [ms_max * 1e-3] * world)

    # end to end through the public API: pinned host inputs -> device ->
    # forward + transform -> host, every step.  The inputs are double-buffered
    # on the device: the host-to-device copy of the next step's inputs (its
    # own stream) overlaps this step's kernels, and the first step's copy is
    # inside the timed region like every other; each step's log-likelihoods
    # are copied back to pinned host memory.
    e2e = None
    if not args.no_e2e:
        host = {k: torch.as_tensor(np.ascontiguousarray(v, dtype=np.int8 if k == "nlayers" else np.float32)).pin_memory()
                for k, v in models_np.items()}
        ll_host = torch.empty(P, dtype=torch.float64).pin_memory()
        bufs = [{k: torch.empty_like(v, device="cuda") for k, v in host.items()} for _ in range(2)]
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        d2h = ll_host.numel() * ll_host.element_size()
        copy_stream = torch.cuda.Stream()

        def h2d_copy(buf):
            # the copy may start once the kernels that last read this buffer are done
            copy_stream.wait_stream(stream)
            with torch.cuda.stream(copy_stream):
                for k in host:
                    buf[k].copy_(host[k], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(copy_stream)
            return ev

        def e2e_run(n_steps):
            ready = h2d_copy(bufs[0])
            for i in range(n_steps):
                nxt = h2d_copy(bufs[(i + 1) % 2]) if i + 1 < n_steps else None
                stream.wait_event(ready)
                L.spectrum_f32(sysg, bufs[i % 2], stream=stream, out=imh_buf)
                L.gates_from_spectrum(sysg, imh_buf, L.GATES_TF32_SPLIT, y_obs, eps_an, I.EPS_MN,
                                      want_gates=False, stream=stream, ll_out=ll_buf)
                ll_host.copy_(ll_buf, non_blocking=True)
                ready = nxt

        e2e_run(2)
        torch.cuda.synchronize()
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        e2e_run(args.steps)
        f1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ems = f0.elapsed_time(f1) / args.steps
        te = torch.tensor([ems], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": world * P / (float(te.item()) * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "overlap": "double-buffered inputs: the next step's copy runs "
                                                         "during this step's kernels"}

    # the plain double-precision form of the same kernel on a 65,536-model block
    fp64 = None
    if rank == 0 and not args.no_variants:
        m64 = I.to_torch(I.subset(models_np, np.arange(1 << 16)), torch.float64)
        L.loglik_f64(sysg, m64, y_obs, eps_an, I.EPS_MN)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        L.loglik_f64(sysg, m64, y_obs, eps_an, I.EPS_MN)
        g1.record(stream)
        torch.cuda.synchronize()
        fp64 = {"value": (1 << 16) / (g0.elapsed_time(g1) * 1e-3), "unit": UNIT, "models": 1 << 16,
                "dtype": "f64"}

    # the gate-transform variants of the same step on the same models: the
    # forward kernel writes the spectra, then the transform + likelihood
    # kernel runs on the tensor cores (TF32 / BF16 high-low splits) or the
    # CUDA cores (FP32); both the whole step and the transform kernel alone
    transforms = None
    if rank == 0 and not args.no_variants:
        transforms = {}
        # the fused form: gates and likelihood in the forward kernel's own
        # epilogue (FP32 CUDA cores), one launch per step (aem_loglik_f32)
        for _ in range(2):
            L.loglik_f32(sysg, models, y_obs, eps_an, I.EPS_MN, stream=stream)
        torch.cuda.synchronize()
        t0_ = torch.cuda.Event(enable_timing=True)
        t1_ = torch.cuda.Event(enable_timing=True)
        t0_.record(stream)
        for _ in range(args.steps):
            L.loglik_f32(sysg, models, y_obs, eps_an, I.EPS_MN, stream=stream)
        t1_.record(stream)
        torch.cuda.synchronize()
        fused_ms = t0_.elapsed_time(t1_) / args.steps
        transforms["fp32_fused_epilogue"] = {"evals_per_s": P / (fused_ms * 1e-3), "ms_per_step": fused_ms,
                                             "roofline_frac": steps_work * FLOPS_PER_LAYER_STEP / (fused_ms * 1e-3)
                                             / (2.0 * peaks["fp32_fma_per_s"])}
        # the benchmark's step with the depth cutoff off: the recursion runs
        # every layer of every model (the paper's form of the recursion)
        sysg.set_depth_cutoff(0.0)
        try:
            for _ in range(2):
                step()
            torch.cuda.synchronize()
            t0_ = torch.cuda.Event(enable_timing=True)
            t1_ = torch.cuda.Event(enable_timing=True)
            fwd_events.clear()
            t0_.record(stream)
            for _ in range(args.steps):
                step(record=True)
            t1_.record(stream)
            torch.cuda.synchronize()
            ws_ms = t0_.elapsed_time(t1_) / args.steps
            ws_fwd = sum(a.elapsed_time(b) for a, b in fwd_events) / len(fwd_events)
        finally:
            sysg.set_depth_cutoff(DEPTH_CUTOFF)
        transforms["tf32_split_whole_stack"] = {
            "evals_per_s": P / (ws_ms * 1e-3), "ms_per_step": ws_ms, "forward_kernel_ms": ws_fwd,
            "roofline_frac": steps_work * FLOPS_PER_LAYER_STEP / (ws_fwd * 1e-3) / (2.0 * peaks["fp32_fma_per_s"]),
            "mufu_frac": steps_work * MUFU_PER_LAYER_STEP / (ws_fwd * 1e-3) / peaks["mufu_mix_per_s"]}
        imh = imh_buf
        for name, mode in (("fp32", L.GATES_FP32), ("tf32_split", L.GATES_TF32_SPLIT),
                           ("bf16_split", L.GATES_BF16_SPLIT)):
            for _ in range(2):
                L.loglik_f32_tc(sysg, models, y_obs, eps_an, I.EPS_MN, mode, stream=stream)
            torch.cuda.synchronize()
            t0_ = torch.cuda.Event(enable_timing=True)
            t1_ = torch.cuda.Event(enable_timing=True)
            t0_.record(stream)
            for _ in range(args.steps):
                L.loglik_f32_tc(sysg, models, y_obs, eps_an, I.EPS_MN, mode, stream=stream)
            t1_.record(stream)
            torch.cuda.synchronize()
            step_ms = t0_.elapsed_time(t1_) / args.steps
            for _ in range(2):
                L.gates_from_spectrum(sysg, imh, mode, y_obs, eps_an, I.EPS_MN, want_gates=False, stream=stream)
            torch.cuda.synchronize()
            t0_.record(stream)
            for _ in range(args.steps):
                L.gates_from_spectrum(sysg, imh, mode, y_obs, eps_an, I.EPS_MN, want_gates=False, stream=stream)
            t1_.record(stream)
            torch.cuda.synchronize()
            kms = t0_.elapsed_time(t1_) / args.steps
            transforms[name] = {"evals_per_s": P / (step_ms * 1e-3), "ms_per_step": step_ms,
                                "transform_kernel_ms": kms,
                                "transform_tflops": 2.0 * P * F * G * (3 if "split" in name else 1) / (kms * 1e-3) / 1e12}
        # the fused step with the models reordered by layer count (one CTA per
        # model already keeps every warp on one model, so this only changes
        # the order in which CTAs meet short and long models)
        order = torch.argsort(models["nlayers"].to(torch.int32), stable=True)
        mb = {k: v[order].contiguous() for k, v in models.items()}
        for _ in range(2):
            L.loglik_f32(sysg, mb, y_obs, eps_an, I.EPS_MN, stream=stream)
        torch.cuda.synchronize()
        t0_.record(stream)
        for _ in range(args.steps):
            L.loglik_f32(sysg, mb, y_obs, eps_an, I.EPS_MN, stream=stream)
        t1_.record(stream)
        torch.cuda.synchronize()
        transforms["fp32_epilogue_bucketed_by_L"] = {"evals_per_s": P / (t0_.elapsed_time(t1_) / args.steps * 1e-3)}
        del mb
        if L.system_status(sysg) != 0:
            raise RuntimeError("a transform kernel reported a timeout")

    # the adjoint: log-likelihood and its gradient with respect to every
    # layer's (log10 sigma, log10 h, m, log10 tau, c) for 65,536 of the same
    # random models (1..10 layers), one aem_loglik_grad_f32 launch per step
    adjoint = None
    if rank == 0 and not args.no_variants:
        na = 1 << 16
        ma = I.to_torch(I.subset(models_np, np.arange(na)), torch.float32)
        for _ in range(3):
            L.loglik_grad_f32(sysg, ma, y_obs, eps_an, I.EPS_MN, stream=stream)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.steps):
            L.loglik_grad_f32(sysg, ma, y_obs, eps_an, I.EPS_MN, stream=stream)
        a1.record(stream)
        torch.cuda.synchronize()
        ams = a0.elapsed_time(a1) / args.steps
        a_steps = layer_steps(models_np["nlayers"][:na], F, K)
        a_ach = a_steps * ADJ_FLOPS_PER_LAYER_STEP / (ams * 1e-3) / 1e12
        a_peak = 2.0 * peaks["fp32_fma_per_s"] / 1e12
        adjoint = {"value": na / (ams * 1e-3), "unit": "gradient evals/s", "models": na, "ms_per_launch": ams,
                   "dtype": "f32", "relative_cost_vs_loglik": (ams / na) / (ms / P),
                   "roofline": {"bound": "alu", "achieved": a_ach, "peak": a_peak, "unit": "TFLOP/s",
                                "frac": a_ach / a_peak, "flops_per_layer_step": ADJ_FLOPS_PER_LAYER_STEP,
                                "peak_source": "FP32 FMA rate measured live by aem_probe_peaks (x2 flops)",
                                "note": "the launch includes the forward kernel's pass for the gates "
                                        "(60 flops per layer-step, not counted in the adjoint's figure)"},
                   "config": f"{WORKLOAD}: {na} random models, 1..10 layers, 5 parameters per layer"}

    # RJSMC soundings/s: the single-sounding configuration (N = 256, kappa <= 3,
    # lambda <= 4, 10 sweeps per stage, 3-layer IP truth) batched over 128
    # soundings per GPU, and the large one (N = 4096, kappa, lambda <= 9, 20
    # sweeps, 5-layer truth) over 4 soundings per GPU; ranks run disjoint
    # soundings (weak scaling by sounding)
    def reduce(sec, n, evals):
        if world == 1:
            return sec, n, evals
        t_ = torch.tensor([sec], dtype=torch.float64, device="cuda")
        w_ = torch.tensor([float(n), float(evals)], dtype=torch.float64, device="cuda")
        dist.all_reduce(t_, op=dist.ReduceOp.MAX)
        dist.all_reduce(w_, op=dist.ReduceOp.SUM)
        return float(t_.item()), float(w_[0].item()), float(w_[1].item())

    rjsmc = None
    if not args.no_rjsmc:
        # the 4-sounding configurations run three seeds each: their stage
        # counts vary more from one sampler path to another
        seeds = [rank + world * i for i in range(3)]
        rjsmc = {
            "rjsmc": rjsmc_measure(torch, L, I, 128, 256, 3, 4, 10, I.truth_3layer(), seed=rank, reduce=reduce),
            # the same single-sounding configuration with the plain FP64 forward
            # model in every evaluation (Algorithm 1 unchanged), on 16 soundings
            "rjsmc_fp64": rjsmc_measure(torch, L, I, 16, 256, 3, 4, 10, I.truth_3layer(), seed=rank,
                                        reduce=reduce, precision=1),
            "rjsmc_large": combine_runs([rjsmc_measure(torch, L, I, 4, 4096, 9, 9, 20, I.truth_5layer(), seed=sd,
                                                       reduce=reduce) for sd in seeds]),
            "rjsmc_langevin": combine_runs([rjsmc_measure(torch, L, I, 4, 4096, 9, 9, 20, I.truth_5layer(), seed=sd,
                                                          reduce=reduce, n_langevin=2) for sd in seeds]),
            "rjsmc_graph": rjsmc_measure(torch, L, I, 128, 256, 3, 4, 10, I.truth_3layer(), seed=rank,
                                         reduce=reduce, graph=True),
            # Section 3.2's adaptive within-model proposal with particle
            # recycling over 3 stages and Appendix F's ZCA-coloured birth /
            # death in half the trans-dimensional moves
            "rjsmc_adaptive": rjsmc_measure(torch, L, I, 128, 256, 3, 4, 10, I.truth_3layer(), seed=rank,
                                            reduce=reduce, adaptive=dict(adaptive=1, recycle_stages=3, zca=0.5)),
        }
        if not args.no_flight_line:
            # the 1000-sounding flight line in one graph-captured sampler (per rank: its block of soundings)
            rjsmc["flight_line"] = flight_line_measure(torch, L, I, 1000, rank, world, reduce)

    # per-gate error of every variant against the oracle on the first
    # ACCURACY_MODELS models of the batch (outside every timed region; the
    # oracle's reference comes from the cpu_baseline leg)
    base = None
    accuracy = None
    if rank == 0 and not args.no_cpu_baseline:
        na_ = min(ACCURACY_MODELS, P)
        # the subset rounded to float32 once: every variant and the oracle see the same inputs
        sub = {k: (np.asarray(v, dtype=np.float32).astype(np.float64) if k != "nlayers" else v)
               for k, v in I.subset(models_np, np.arange(na_)).items()}
        base, ref = cpu_baseline(sub, y_obs_np)
        if not args.no_variants:
            ms32 = I.to_torch(sub, torch.float32)
            accuracy = {"fp64_plain": gate_errors(
                            L.forward_f64(sysg, I.to_torch(sub, torch.float64)).cpu().numpy(), ref, 1e-4),
                        "fp32": gate_errors(L.forward_f32(sysg, ms32).cpu().numpy(), ref, 1e-4)}
            for name, mode, floor in (("fp32_separate_transform", L.GATES_FP32, 1e-4),
                                      ("tf32_split", L.GATES_TF32_SPLIT, 1e-4),
                                      ("bf16_split", L.GATES_BF16_SPLIT, 1e-3)):
                _, g_ = L.loglik_f32_tc(sysg, ms32, y_obs, eps_an, I.EPS_MN, mode, want_gates=True)
                accuracy[name] = gate_errors(g_.cpu().numpy(), ref, floor)

    if rank == 0:
        # the dominant kernel (the forward model, 99 % of the step): its
        # algorithmic flops per launch (F K L layer-steps per model, the whole
        # stack) over its own event-timed duration
        flops = steps_work * FLOPS_PER_LAYER_STEP
        achieved = flops / (fwd_ms * 1e-3) / 1e12
        peak = 2.0 * peaks["fp32_fma_per_s"] / 1e12
        # the special-function unit: layer-steps x 6 MUFU ops against the
        # measured rate of the same mix (rsqrt, rsqrt, rcp, ex2, sin, cos)
        mufu_frac = steps_work * MUFU_PER_LAYER_STEP / (fwd_ms * 1e-3) / peaks["mufu_mix_per_s"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: {P} random layered models per GPU, 1..10 layers, "
                                   f"{G} gates, {F} freqs, {K} Hankel points, a=13 m, h=30 m",
                       "step": "forward model to spectra (forward_f32_kernel), then gate transform + likelihood "
                               "on the tensor cores (gates_tc_kernel, TF32 high/low split)",
                       "models_per_gpu": P, "gates": G, "freqs": F, "hankel": K,
                       "forward_launch_shape": {"index": shape, "sample_ms_per_shape": shape_ms},
                       "l2": "inputs larger than L2 (210 MB of model parameters per step)"},
            "roofline": {"bound": "alu", "kernel": "forward_f32_kernel", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "kernel_ms": fwd_ms,
                         # DRAM bytes of one spectrum-writing launch from an ncu
                         # capture of the dynamic-scheduled 256 x 3 shape on 2^20
                         # models of this workload, scaled by the model count; null
                         # when the autotuner picks another shape
                         "traffic": (SPECTRUM_LAUNCH_BYTES_1M / 1048576 * P) if shape == 8 else None,
                         "traffic_unit": "bytes per launch",
                         "algorithmic_bytes": float(P) * (K_PARAM_BYTES + 4 * F),
                         "peak_source": "FP32 FMA rate measured live by aem_probe_peaks (x2 flops)",
                         "mufu_frac": mufu_frac,
                         # the two-pipe roofline: the batch cannot take less than
                         # max(FP32 ops / FP32 peak, MUFU ops / MUFU peak); the
                         # fraction of that bound the launch reaches, and its pipe
                         "roofline_time_frac": max(achieved / peak, mufu_frac),
                         "binding_pipe": "mufu" if mufu_frac > achieved / peak else "fp32",
                         "layer_steps_per_s": steps_work / (ms * 1e-3),
                         # the depth cutoff (aem_system_set_depth_cutoff): the
                         # kernel runs only this share of the whole stack's
                         # layer-steps (counted by the kernel on the batch), so
                         # its pipes' efficiency on the steps it runs is
                         # frac_executed and mufu_frac_executed
                         "depth_cutoff": DEPTH_CUTOFF, "layer_steps_kept_frac": kept_frac,
                         "frac_executed": achieved / peak * kept_frac,
                         "mufu_frac_executed": mufu_frac * kept_frac},
            "gpu_launches": 2 * args.steps,
            "clocks": clocks,
            "peaks_measured": peaks,
            "e2e": e2e,
        }
        if fp64 is not None:
            line["fp64_plain"] = fp64
        if rjsmc is not None:
            line.update(rjsmc)
        if adjoint is not None:
            line["adjoint"] = adjoint
        if transforms is not None:
            line["gate_transform_variants"] = transforms
        if accuracy is not None:
            line["accuracy_vs_oracle"] = accuracy
        if base is not None:
            line["cpu_baseline"] = base
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
