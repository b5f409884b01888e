/*
 * aem_rjsmc.h -- C ABI of the GB300 (sm_103a) hot path of reversible jump
 * sequential Monte Carlo (RJSMC) for airborne-EM induced-polarisation
 * detectability, after Davies, Ley-Cooper, Sutton & Drovandi,
 * arXiv 2109.00661.
 *
 * Conventions for every entry point:
 *   - Pointers marked [device] are CUDA device pointers on the current device;
 *     [host] pointers are ordinary host memory.  The caller owns every buffer
 *     passed in; the library owns only the handles it creates and the tables
 *     inside them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream are asynchronous on it unless the
 *     comment says otherwise.
 *   - Return value: AEM_OK (0) or a negative aem_status.  Nothing throws across
 *     the ABI.  aem_last_error() returns a thread-local message for the last
 *     failure on the calling thread.
 *   - Units: SI throughout.  Gate values are -dBz/dt in T/s for the system's
 *     transmitter current (the sign makes a conductive earth positive, as the
 *     paper says of its data in Section 2.3.2).
 */
#ifndef AEM_RJSMC_H
#define AEM_RJSMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AEM_OK = 0,
    AEM_ERR_INVALID_ARG = -1, /* a size, pointer or value is out of range */
    AEM_ERR_CUDA = -2,        /* a CUDA runtime call failed */
    AEM_ERR_NONFINITE = -3,   /* a reduction produced NaN/Inf */
    AEM_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
    AEM_ERR_NO_BRACKET = -5,  /* tempering bisection could not bracket alpha*N */
    AEM_ERR_UNSUPPORTED = -6  /* configuration not built into this library */
} aem_status;

/* Cole-Cole forms.  Section 2 writes sigma(w) = sigma_inf (1 - m / (1 + (i w tau)^c))
 * and notes Pelton's form is a bijective reparameterisation of it. */
typedef enum {
    AEM_CC_PAPER = 0, /* log10 sigma parameter is log10 sigma_inf (high-frequency) */
    AEM_CC_PELTON = 1 /* 1/rho, rho = rho_0 (1 - m (1 - 1/(1 + (i w tau)^c))); parameter is log10 sigma_0 (DC) */
} aem_cc_form;

/* Limits compiled into the kernels. */
#define AEM_MAX_LAYERS 20  /* merged layers per model (<= kappa_max + lambda_max + 1) */
#define AEM_MAX_FREQ 128
#define AEM_MAX_GATES 64
#define AEM_MAX_HANKEL 512

const char *aem_last_error(void);

/* ------------------------------------------------------------------------
 * System: central-loop AEM geometry and the precomputed tables.
 *
 * Section 2 (the forward model is the 1-D layered-earth Hankel-transform
 * model the paper takes from Ward & Hohmann 1988) and Section 2.3.2 (off-time
 * dB/dt gates).  The library builds, in double precision on the host:
 *   - n_freq frequencies log-spaced on [f_min_hz, f_max_hz];
 *   - an n_hankel-point log-spaced Hankel rule: lambda_k = exp(x0 + k dx) with
 *     x0 = ln(1e-5/(2h+a)), x_{K-1} = ln(20/h), weights dx (halved at both
 *     ends) times (I a / 2) lambda^2 J1(lambda a) e^{-2 lambda h}, so that
 *     Hz_s(w) = sum_k w_k R_0(lambda_k, w);
 *   - the G x F step-off transform matrix T with y(t_g) = sum_f T[g,f] Im Hz_s(w_f),
 *     y = -dBz/dt = -(2 mu0/pi) Int Im Hz_s(w) sin(w t) dw, Im Hz_s
 *     interpolated by a cubic spline in ln w clamped to a tail ~ w below the
 *     first node and ~ w^-1/2 above the last node.
 * Gates are point samples at gate_times (an ideal step-off waveform).
 * ---------------------------------------------------------------------- */
typedef struct aem_system aem_system;

typedef struct {
    double loop_radius;       /* a [m], > 0 */
    double height;            /* h [m], transmitter and receiver height, > 0 */
    double current;           /* I [A], > 0 */
    int n_freq;               /* F, 2..AEM_MAX_FREQ */
    double f_min_hz;          /* first frequency node [Hz], > 0 */
    double f_max_hz;          /* last frequency node [Hz], > f_min_hz */
    int n_gates;              /* G, 1..AEM_MAX_GATES */
    const double *gate_times; /* [host] G gate centre times [s], ascending, > 0 */
    int n_hankel;             /* K, 8..AEM_MAX_HANKEL */
    int cc_form;              /* aem_cc_form */
} aem_system_desc;

/* Synchronous.  Builds the tables and uploads them to the current device. */
int aem_system_create(const aem_system_desc *desc, aem_system **out);
int aem_system_destroy(aem_system *sys);

/* Synchronous.  Copies the host tables out (any pointer may be NULL):
 * freqs_hz [F], lambda [K], hankel_w [K], T [G*F] row-major by gate. */
int aem_system_tables(const aem_system *sys, double *freqs_hz, double *lambda, double *hankel_w, double *T);

/* ------------------------------------------------------------------------
 * Merged layered models (the forward model's input after the direct-sum
 * merge of Section 2.1): structure of arrays, row-major [n_models][lmax].
 * Layer 0 is the top layer; layer nlayers-1 is the basement half-space, whose
 * thickness entry is ignored.  All parameters are per layer.
 * ---------------------------------------------------------------------- */
typedef struct {
    int n_models;          /* P >= 0 */
    int lmax;              /* row stride, 1..AEM_MAX_LAYERS */
    const int8_t *nlayers; /* [device] P, each in 1..lmax */
    const float *logsig;   /* [device] P*lmax, log10 conductivity [S/m] (see aem_cc_form) */
    const float *logh;     /* [device] P*lmax, log10 thickness [m] */
    const float *m;        /* [device] P*lmax, intrinsic chargeability in [0,1) */
    const float *logtau;   /* [device] P*lmax, log10 time constant [s] */
    const float *c;        /* [device] P*lmax, frequency exponent in (0,1] */
} aem_models_f32;

typedef struct {
    int n_models;
    int lmax;
    const int8_t *nlayers;
    const double *logsig, *logh, *m, *logtau, *c;
} aem_models_f64;

/* Forward model (Section 2): gates [device, P*G] row-major by model, and
 * optionally Im Hz_s at the frequency nodes (imh [device, P*F], may be NULL;
 * gates may be NULL if only imh is wanted).  The f32 entry computes the
 * layer recursion, Hankel sum and gate transform in FP32; the f64 entry is
 * the plain double-precision form of the same arithmetic. */
int aem_forward_f32(const aem_system *sys, const aem_models_f32 *models, float *gates, float *imh, void *stream);
int aem_forward_f64(const aem_system *sys, const aem_models_f64 *models, double *gates, double *imh,
                    void *stream);

/* Gaussian log-likelihood (Section 2.3.2):
 *   ll_p = -1/2 sum_g [ (y_g - yhat_g)^2 / v_g + ln(2 pi v_g) ],
 *   v_g = eps_an[g]^2 + (eps_mn * yhat_g)^2   (variance from the model prediction).
 * y_obs, eps_an: [device] G doubles.  ll: [device] P doubles, summed in FP64.
 * gates: optional [device] P*G copy of the predictions (may be NULL). */
int aem_loglik_f32(const aem_system *sys, const aem_models_f32 *models, const double *y_obs,
                   const double *eps_an, double eps_mn, double *ll, float *gates, void *stream);
int aem_loglik_f64(const aem_system *sys, const aem_models_f64 *models, const double *y_obs,
                   const double *eps_an, double eps_mn, double *ll, double *gates, void *stream);

/* ------------------------------------------------------------------------
 * Device throughput probes used for the roofline denominators: FP32 FMA and
 * MUFU (ex2/sin/cos/rsqrt/rcp) operation rates measured by dependency-free
 * loops on every SM.  Synchronous.  Results in operations per second.
 * ---------------------------------------------------------------------- */
int aem_probe_peaks(double *fp32_fma_per_s, double *mufu_per_s, double *fp64_fma_per_s, double *sm_clock_hz);

#ifdef __cplusplus
}
#endif
#endif /* AEM_RJSMC_H */
