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
    AEM_CC_PELTON = 1, /* 1/rho, rho = rho_0 (1 - m (1 - 1/(1 + (i w tau)^c))); parameter is log10 sigma_0 (DC) */
    AEM_CC_LITERAL = 2 /* sigma_0 (1 - m (1 - 1/(1 + (i w tau)^c))) taken as a conductivity: sigma_0 at DC,
                          sigma_0 (1 - m) at high frequency (the paper's form with sigma_inf = sigma_0 (1 - m) and
                          chargeability -m / (1 - m)) */
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
/* aem_forward_f32 that also adds to *layer_steps ([device] unsigned long
 * long, caller-initialised) the number of (layer, abscissa pair) steps its
 * recursion ran: with the depth cutoff off this is P x F x ceil(K/2) x the
 * mean layer count; the ratio is the fraction of the stack the cutoff kept
 * (aem_system_set_depth_cutoff).  A diagnostic for the throughput figures. */
int aem_forward_f32_count(const aem_system *sys, const aem_models_f32 *models, float *gates, float *imh,
                          unsigned long long *layer_steps, void *stream);
int aem_forward_f64(const aem_system *sys, const aem_models_f64 *models, double *gates, double *imh,
                    void *stream);

/* Gaussian log-likelihood (Section 2.3.2):
 *   ll_p = -1/2 sum_g [ (y_g - yhat_g)^2 / v_g + ln(2 pi v_g) ],
 *   v_g = eps_an[g]^2 + (eps_mn * yhat_g)^2   (variance from the model prediction).
 * y_obs, eps_an: [device] G doubles.  ll: [device] P doubles, summed in FP64;
 * the f32 entry forms each term in FP32 (the residual y_g - yhat_g from an FP64
 * difference), so eps_an^2 must be a normal float (eps_an >= 1e-18), the f64
 * entry in FP64.  A NaN parameter gives NaN for that model only.
 * gates: optional [device] P*G copy of the predictions (may be NULL). */
int aem_loglik_f32(const aem_system *sys, const aem_models_f32 *models, const double *y_obs,
                   const double *eps_an, double eps_mn, double *ll, float *gates, void *stream);
int aem_loglik_f64(const aem_system *sys, const aem_models_f64 *models, const double *y_obs,
                   const double *eps_an, double eps_mn, double *ll, double *gates, void *stream);

/* Launch-shape autotuner of the FP32 forward kernel (aem_forward_f32,
 * aem_loglik_f32 and every sampler call that evaluates the forward model).
 * Shapes: 0 = 256 threads per CTA with 4 resident CTAs per SM (the default),
 * 1 = 128 x 8, 2 = 512 x 2, 3 = 256 x 3, 4 = 128 x 6 (the register budget per
 * thread follows from the pair), each with a fixed grid-stride order of
 * models; 5..9 = the same five with dynamic scheduling (a CTA claims its
 * next model from a counter in stream-ordered scratch when it finishes one).  aem_autotune_forward times every shape that
 * fits on an SM on the caller's sample batch (one untimed launch, then
 * `repeats` launches timed with CUDA events on `stream`; synchronous), and
 * records the fastest for the sample's lmax in the system: later launches
 * with that lmax use it.  shape_out (may be NULL) receives the choice; ms_out
 * (may be NULL, AEM_F32_SHAPES floats) the mean time per launch of each shape, -1 for a
 * shape that does not fit.  It takes P x G floats of stream-ordered scratch
 * (cudaMallocAsync) for the duration of the call.  aem_forward_shape sets the
 * shape for an lmax directly.  Not thread-safe against concurrent launches on
 * the same system. */
#define AEM_F32_SHAPES 10
int aem_autotune_forward(aem_system *sys, const aem_models_f32 *sample, int repeats, void *stream, int *shape_out,
                         float *ms_out);
int aem_forward_shape(aem_system *sys, int lmax, int shape);

/* Depth cutoff of the FP32 forward kernel (aem_forward_f32, aem_loglik_f32,
 * the tensor-core and gradient entries' forward pass and every sampler call
 * that evaluates the FP32 forward model) and of the FP32 adjoint
 * (aem_loglik_grad_f32, where each abscissa runs the layers it needs); the
 * FP64 form always takes the whole stack.  The TE recursion of Section 2 (Ward & Hohmann's reflection form)
 * runs bottom-up through every layer, but a layer below a depth where the
 * round-trip attenuation exp(-2 sum Re(u_i) h_i) of the layers above is under
 * exp(-a) changes R_0 by less than exp(-a) times the largest reflection
 * coefficient below it; the kernel then treats that layer as the half-space.
 * a = attenuation + ln(max_n |s_n| / |s_0|) per model and frequency (s_n =
 * i omega mu0 sigma_n), so a large conductivity contrast below a resistive top
 * keeps more layers.  The depth is found from a lower bound of the attenuation
 * (Re u_i >= Re sqrt(s_i) and Re u_i >= sqrt(lambda^2 - max_n(-Re s_n))) and
 * taken per group of 32 (frequency, abscissa-pair) items as the largest any of
 * them needs, so the results do not depend on the launch shape.  attenuation:
 * >= 0 and finite; 0 turns the cutoff off (every layer always).  Default 20
 * (exp(-20) = 2.1e-9, under FP32 resolution).  Synchronous; applies to later
 * launches. */
int aem_system_set_depth_cutoff(aem_system *sys, double attenuation);

/* Gate transform and likelihood from a batch of spectra (the a5 + a6 steps on
 * their own; Section 2.3.2).  imh: [device] n_models x F Im Hz_s at the
 * system's frequency nodes (as aem_forward_f32 writes it).  mode selects the
 * arithmetic of y = T Im H:
 *   AEM_GATES_FP32        FP32 dot products on the CUDA cores;
 *   AEM_GATES_TF32_SPLIT  tensor cores (tcgen05, kind::tf32), each operand
 *                         split into TF32 high + low parts, three products
 *                         accumulated in FP32 (relative residual ~2^-22 per term);
 *   AEM_GATES_BF16_SPLIT  the same with BF16 parts (kind::f16, ~2^-17 per term).
 * gates: [device] n_models x G (may be NULL); ll: [device] n_models doubles
 * (may be NULL; then y_obs and eps_an may be NULL too), with y_obs [device] G
 * and eps_an [device] G as for aem_loglik_f32.  Asynchronous.  A bounded
 * wait inside the tensor-core kernel that gives up records AEM_ERR_TIMEOUT in
 * the system's status word (aem_system_status). */
#define AEM_GATES_FP32 0
#define AEM_GATES_TF32_SPLIT 1
#define AEM_GATES_BF16_SPLIT 2
int aem_gates_from_spectrum(const aem_system *sys, const float *imh, int n_models, int mode, const double *y_obs,
                            const double *eps_an, double eps_mn, float *gates, double *ll, void *stream);

/* aem_loglik_f32 with the gate transform of `mode` (above): the forward
 * kernel writes the spectra into imh_work ([device] P x F floats, caller's
 * scratch), then aem_gates_from_spectrum forms gates (may be NULL) and ll. */
int aem_loglik_f32_tc(const aem_system *sys, const aem_models_f32 *models, const double *y_obs,
                      const double *eps_an, double eps_mn, int mode, float *imh_work, double *ll, float *gates,
                      void *stream);

/* Synchronous.  Reads and clears the system's device status word: 0, or the
 * AEM_ERR_TIMEOUT a kernel recorded since the last call. */
int aem_system_status(const aem_system *sys, int *status);

/* Diagnostics of the bounded device wait (for tests; no counterpart in the
 * paper).  spins > 0 sets the iteration limit of the tensor-core transform's
 * completion wait (0 restores the default, 2^22 polls); skip_first_mma = 1
 * makes each CTA of that kernel issue no MMA and no commit for its first
 * tile, so its wait runs out with no tensor-core work in flight: the CTA then
 * records AEM_ERR_TIMEOUT in the status word, frees its tensor memory and
 * returns, leaving the outputs of its tiles unwritten.  The limit applies to
 * the first wait only; the wait for a CTA's own MMAs after a timeout keeps the
 * full limit (should that one also run out, the MMAs may still be in flight
 * when the tensor memory is freed, which is undefined: treat a context that
 * reported a timeout as unreliable).  Not thread-safe against launches on the
 * same system.  skip_first_mma must be 0 or 1 (AEM_ERR_INVALID_ARG). */
int aem_debug_bounded_wait(aem_system *sys, unsigned int spins, int skip_first_mma);

/* Gradient of the log-likelihood above (FP32 forward model) with respect to
 * every merged layer's parameters, by reverse-mode differentiation of the
 * forward model of Section 2 and the likelihood of Section 2.3.2.
 * grad: [device] P*lmax*5 floats, row-major [model][layer][parameter] with
 * parameters (log10 sigma, log10 thickness, m, log10 tau, c); the basement's
 * thickness entry and layers >= nlayers are 0.  ll: [device] P doubles (may
 * be NULL).  Every aem_cc_form is differentiated (log10 sigma is the form's
 * conductivity parameter). */
int aem_loglik_grad_f32(const aem_system *sys, const aem_models_f32 *models, const double *y_obs,
                        const double *eps_an, double eps_mn, double *ll, float *grad, void *stream);

/* ------------------------------------------------------------------------
 * RJSMC stage (Algorithm 1 with the adaptive choices of Section 3.2 and
 * Appendices B-E).
 *
 * Particle state (decoupled model of Section 2.1, priors of Section 2.3.1):
 * kappa conductive interfaces (depths zc, log10 sigma of the layer below each,
 * phic) under a background log10 sigma phib; lambda chargeable interfaces
 * (depths zm, chargeability of the layer below each, mv) under m = 0; global
 * Cole-Cole tau [s] and c.  Model index k = kappa * (lambda_max + 1) + lambda.
 * Priors: kappa ~ U{0..kappa_max}, lambda ~ U{0..lambda_max}, depths sorted
 * uniforms on (0, zmax), log10 sigma ~ U(phi_lo, phi_hi), m ~ U(0,1),
 * tau ~ U(0,1) (or log10 tau ~ U(logtau_lo, logtau_hi)), c ~ U(0,1).
 * Random numbers: Philox4x32-10 with key (seed low 32 bits, seed high 32 bits
 * xor sounding) and counter (particle, purpose, stage, sweep).
 * ---------------------------------------------------------------------- */
#define AEM_SMC_SLOTS 10           /* interface slots per profile: kappa_max, lambda_max <= 9 */
#define AEM_SMC_MAX_MODELS 100     /* (kappa_max + 1) (lambda_max + 1) */
#define AEM_SMC_MAX_PARTICLES 16384 /* particles per sounding */
/* Particle-space gradient row: phi_b, phi_c[SLOTS], z_c[SLOTS], z_m[SLOTS],
 * m[SLOTS], tau coordinate, c (slots past kappa / lambda are 0). */
#define AEM_SMC_GRAD_DIM (3 + 4 * AEM_SMC_SLOTS)

typedef struct {
    int n_particles;   /* N per sounding, 2..AEM_SMC_MAX_PARTICLES */
    int n_soundings;   /* S >= 1; soundings are independent samplers */
    int kappa_max;     /* 0..9 */
    int lambda_max;    /* 0..9, kappa_max + lambda_max + 1 <= AEM_MAX_LAYERS */
    double zmax;       /* maximum interface depth [m] */
    double alpha;      /* TESS threshold proportion, 0 < alpha < 1 */
    double c_mut;      /* c of App. B: R_t = ceil(log c / log(1 - p_acc_min)) */
    int r_max;         /* upper bound on R_t */
    double step_phi, step_m, step_tau, step_c, step_z; /* random-walk scales */
    double phi_lo, phi_hi;                 /* log10 sigma prior bounds */
    int tau_log_prior;                     /* 0: tau ~ U(0,1) s; 1: log10 tau ~ U(lo, hi) */
    double logtau_lo, logtau_hi;
    unsigned long long seed;
    int bisect_iters;                      /* bisection iterations for gamma_t (1..200) */
    int n_langevin;                        /* Langevin sweeps per stage after the random walks (0..1000; 0: off) */
    double langevin_h;                     /* initial Langevin step h in units of the random-walk scales (> 0) */
    int langevin_adapt;                    /* 1: after each stage h <- h exp(2 (rate - 0.574)), in [1e-6, 10] */
    int adaptive;                          /* 1: the adaptive within-model proposal of Section 3.2 (below) */
    double pca_target;                     /* its target acceptance rate (0.44) */
    int pca_bisect_iters;                  /* bisection steps on trial proposals per stage (1..60) */
    double pca_ridge;                      /* covariance ridge, fraction of the random-walk steps (>= 0) */
    int recycle_stages;                    /* 0..32; > 0 (with adaptive): particle recycling over that many stages */
    double zca;                            /* 0..1 (with adaptive): probability of the ZCA-coloured birth / death */
    int precision;                         /* AEM_SMC_FP32 (default): every forward evaluation by the FP32 kernel;
                                              AEM_SMC_FP64: the plain FP64 forward model (Algorithm 1 unchanged; the
                                              Langevin moves, FP32 adjoint, are then unsupported) */
} smc_desc;

#define AEM_SMC_FP32 0
#define AEM_SMC_FP64 1

typedef struct smc_state smc_state;

/* Host mirror of the particle arrays (P = S * N particles, sounding-major;
 * zc/phic/zm/mv are [P][AEM_SMC_SLOTS], entries past kappa / lambda are 0).
 * move / valid may be NULL; they are filled only for the proposal set. */
typedef struct {
    int *kappa, *lam;
    float *phib, *tau, *c, *zc, *phic, *zm, *mv;
    double *ll;
    int8_t *move, *valid;
} smc_particles_host;

/* Fills *d with the defaults (N = 256, kappa_max = 3, lambda_max = 4,
 * zmax = 500 m, alpha = 0.5, c_mut = 0.01, r_max = 10, log10 sigma in (-4, 2),
 * no Langevin sweeps, langevin_h = 0.1, langevin_adapt = 1, adaptive = 0,
 * pca_target = 0.44, pca_bisect_iters = 6, pca_ridge = 0.01, recycle_stages = 0,
 * zca = 0). */
int smc_desc_defaults(smc_desc *d);

/* Synchronous.  y_obs [host, S x G] observed gates per sounding; eps_an [host, G];
 * eps_mn multiplicative noise.  All later calls run on `stream`. */
int smc_create(const aem_system *sys, const smc_desc *desc, const double *y_obs, const double *eps_an,
               double eps_mn, void *stream, smc_state **out);
int smc_destroy(smc_state *st);

/* Draws every particle from the prior and evaluates its log-likelihood
 * (Alg. 1 initialisation; gamma_0 = 0, Z_0 = 1). */
int smc_init(smc_state *st);

/* Re-weight (a7): gamma_t by bisection so that TESS = sum_k ESS_k ~ alpha N
 * (the whole remaining step when that keeps TESS >= alpha N), log Z_k +=
 * log(mean_i L_i^(gamma_t - gamma_{t-1})) over model k, normalised weights
 * within each model.  FP64 throughout.  Advances the stage counter.  If
 * gamma_out is not NULL the new gamma of every sounding is copied to it
 * (synchronising the stream). */
int smc_reweight(smc_state *st, double *gamma_out);

/* Resample (a8): within-model systematic resampling (N_k kept fixed) on an
 * integer CDF (q = round(W 2^40), last entry forced to 2^40), one uniform
 * per model and stage. */
int smc_resample(smc_state *st);

/* Mutate (a9): n_sweeps sweeps (n_sweeps <= 0: R_t of App. B from the
 * previous stage's lowest move-type acceptance rate, r_max on the first
 * stage).  Each sweep proposes one move per particle, chosen uniformly among
 * conductive birth, conductive death, chargeable birth, chargeable death,
 * depth move and Gaussian random walk (impossible moves count as rejected),
 * evaluates the proposals through the FP32 forward model and accepts with
 * probability min(1, exp(gamma_t (l' - l))).  Then desc.n_langevin
 * within-model Langevin (MALA) sweeps, a move the paper does not use: with
 * theta the particle's continuous parameters (phi_b, phi_c, z_c, z_m, m, the
 * tau coordinate, c), D = diag(s_j^2) of the random-walk steps and h the
 * sounding's current step (desc.langevin_h after smc_init; with
 * desc.langevin_adapt, updated after each call from that call's Langevin
 * acceptance rate towards 0.574, Roberts & Rosenthal 1998), the proposal is
 *   theta' = theta + (h^2 / 2) D gamma_t grad l(theta) + h D^(1/2) xi,
 * the gradient coming from the adjoint kernel (aem_loglik_grad_f32) mapped
 * through the direct sum; it is accepted when
 *   ln u < gamma_t (l' - l) + log q(theta | theta') - log q(theta' | theta)
 * and rejected outside the prior support or the interface order.  The
 * Langevin tests compare likelihoods from the adjoint kernel on both sides.
 * Synchronises at the end. */
int smc_mutate(smc_state *st, int n_sweeps);

/* Proposal step only (for inspection): proposals for (stage, sweep) from the
 * current particles into the proposal set, without likelihood evaluation. */
int smc_propose(smc_state *st, int stage, int sweep);

/* Re-evaluates the log-likelihood of the current particles. */
int smc_loglik_current(smc_state *st);

/* Log-likelihood (into the current particles' ll) and the gradient of the
 * log-likelihood with respect to each current particle's parameters, by the
 * adjoint kernel and the chain rule through the direct sum (Section 2.1).
 * grad_host: [host] P x AEM_SMC_GRAD_DIM floats (may be NULL: the gradient is
 * then only kept on the device for smc_langevin_propose); the tau slot is
 * d l / d tau [s] with the uniform tau prior and d l / d log10 tau with the
 * log-uniform one.  Synchronous when grad_host is not NULL. */
int smc_grad_current(smc_state *st, float *grad_host);

/* Langevin proposal step only (for inspection): proposals for (stage, sweep)
 * from the current particles and the gradient of the last smc_grad_current
 * into the proposal set (valid flags as for smc_propose), at each sounding's
 * current gamma and step.  AEM_ERR_INVALID_ARG when no gradient of the current
 * particles is held (none computed, or the particles changed since). */
int smc_langevin_propose(smc_state *st, int stage, int sweep);

/* n_sweeps (0..1000) Langevin sweeps alone, at the current stage and each
 * sounding's current gamma and step (sweep counters 0..n_sweeps-1, as
 * smc_mutate uses them after its random-walk sweeps; the step is not
 * adapted).  Synchronises at the end. */
int smc_langevin(smc_state *st, int n_sweeps);

/* Synchronous.  accepted / proposed [S]: Langevin counts of the last
 * smc_mutate or smc_langevin call; h [S]: each sounding's current step.  Any
 * pointer may be NULL. */
int smc_langevin_stats(const smc_state *st, int *accepted, int *proposed, double *h);

/* Runs reweight / resample / mutate until gamma = 1 for every sounding or
 * max_stages stages (Alg. 1).  stages_out may be NULL. */
int smc_run(smc_state *st, int max_stages, int n_sweeps, int *stages_out);

/* smc_run with the stage loop on the device: one stage (reweight,
 * resample, n_sweeps >= 1 sweeps of the moves; with the descriptor's options
 * also the recycling record, the adaptive fit and scale bisection and the
 * Langevin sweeps with their step adaptation) is captured once into a CUDA
 * graph as the body of a conditional WHILE node.  A kernel at the end of the
 * body advances nothing on the host; it sets the loop condition from the new
 * gammas (another stage while any sounding's gamma < 1 and fewer than
 * max_stages stages have run), and the stage number lives in device memory.
 * No host synchronisation or allocation happens between stages.  Same results
 * as smc_run(st, max_stages, n_sweeps) bit for bit.  n_sweeps <= 0 takes App.
 * B's R_t as smc_mutate does, decided on the device each stage from the
 * previous stage's acceptance counts: the graph then holds r_max sweeps whose
 * kernels return at once beyond R_t (R_t's double-precision logarithm is the
 * device's, which may differ from the host's in its last bit).  With
 * recycling the stage counter must stay below 1024 (AEM_ERR_INVALID_ARG
 * otherwise).  Synchronous; stages_out may be NULL. */
int smc_run_graph(smc_state *st, int max_stages, int n_sweeps, int *stages_out);

/* Synchronous (a10).  post_k [S x M]: N_k / N; log_bfipd [S]: log of the
 * BFIPD statistic of Section 2.3.3, the grouped Bayes factor
 * |M_kappa| sum_{k chargeable} (pi_k / p_k) / (|M_lambda| sum_{k not} (pi_k / p_k))
 * with the sampler's uniform p(k), i.e. log(N_IP / (lambda_max N_nonIP)):
 * +inf when no particle is non-chargeable, -inf when none is chargeable
 * (never clipped); log_z_k [S x M]: accumulated log Z_k.  The counts, the
 * posterior probabilities and log BFIPD are formed on the device in FP64.  Any
 * pointer may be NULL. */
int smc_model_odds(const smc_state *st, double *post_k, double *log_bfipd, double *log_z_k);

/* Failure reporting (synchronous).  status: AEM_OK, or the first failure a
 * reweight step recorded since the last call (read and cleared):
 * AEM_ERR_NONFINITE when a sounding had no particle with a finite
 * log-likelihood (its gamma and log Z are left unchanged and its weights
 * uniform within each model), AEM_ERR_NO_BRACKET when no probed tempering
 * step kept TESS >= alpha N (more than (1 - alpha) N particles with ll = -inf;
 * the smallest probed step is taken).  smc_reweight with gamma_out != NULL,
 * smc_run and smc_run_graph return these codes themselves (smc_run stops at
 * that stage; smc_run_graph finishes it, then stops).  nonfinite [S] (may be
 * NULL): per sounding, how many log-likelihoods came out NaN or +inf since
 * smc_init; the sampler sets each such value to -inf, so that particle has no
 * weight and a proposal that produced one is rejected. */
int smc_status(smc_state *st, int *status, int *nonfinite);

/* Synchronous.  gamma [S], stage, accepted / proposed [S x 6] counts of the
 * last smc_mutate call by move type.  Any pointer may be NULL. */
int smc_stats(const smc_state *st, double *gamma, int *stage, int *accepted, int *proposed);

/* Synchronous copies of the particle arrays: which = 0 current, 1 proposals. */
int smc_get_particles(const smc_state *st, int which, smc_particles_host *h);
/* Synchronous.  Replaces the current particles (and, when not NULL / >= 0,
 * gamma [S], log_z [S x M] and the stage counter). */
int smc_set_particles(smc_state *st, const smc_particles_host *h, const double *gamma, const double *log_z,
                      int stage);

/* The adaptive within-model proposal of Section 3.2, for the current stage
 * (smc_mutate calls it before its sweeps when desc.adaptive is set): per
 * sounding and model k with at least two particles, the mean mu_k and
 * covariance Sigma_k of the continuous vector theta (phi_b, phi_c, z_c, z_m,
 * m, the tau coordinate, c) over the model's particles, plus (pca_ridge s_j)^2
 * on the diagonal (s_j the random-walk step of component j), decomposed as
 * U Lambda U^T by Jacobi rotations in FP64; then desc.pca_bisect_iters steps of
 * bisection on log a_k within +-3 of the previous stage's value, each a forward
 * pass over trial proposals theta + a sqrt(Lambda_r) xi U_r (r uniform, xi
 * normal, the same draws at every step), comparing the model's mean
 * min(1, (L'/L)^gamma) with desc.pca_target.  The perturb move of smc_mutate
 * then steps along U_r with standard deviation a_k sqrt(Lambda_r); models
 * without a fit keep the fixed-scale component-wise walk.
 * With desc.recycle_stages = H > 0 the fit recycles particles (Section 3.2,
 * particle impoverishment): mu_k and Sigma_k are weighted over the model's
 * particles of the last H post-resample populations (stage 0 = the prior
 * draw), particle i from any stage carrying
 *   log nu = gamma_t l_i - log( (1/(t+1)) sum_{l=0}^{t} exp(gamma_l l_i - log Z_{l,k}) )
 * over every stage's gamma and log Z (at most 1024 stages); a model is
 * fitted when its current population holds at least two particles.  The
 * history takes H x P particle records of device memory; a checkpoint
 * carries it.
 * With desc.zca = p > 0 a birth or death uses, with probability p (a draw
 * independent of the state) and when the target model (birth) or the current
 * model (death) has a fit, Appendix F's ZCA-coloured move: the new layer's
 * value starts as the split layer's (0 for a chargeable layer above every
 * chargeable interface), then every component but the new depth moves by
 * u Z[i, j], u ~ N(0, 1), Z = U Lambda^(1/2) U^T of model k+1's fit, i the new
 * value's component; the Metropolis-Hastings test adds log(|J| / (width phi(u)))
 * with J = Z[i, i] - Z[i, h] (the reciprocal for a death, u solved from the two
 * values).  p = 1 is the paper's form. */
int smc_adapt(smc_state *st);
/* Synchronous.  lf [host, P]: the log factor each particle's last proposal
 * (smc_propose or a sweep of smc_mutate) adds to gamma_t (l' - l) in its
 * Metropolis-Hastings test: log(|J| / (width phi(u))) for a ZCA-coloured birth,
 * its reciprocal for a death, 0 for every other move. */
int smc_get_log_factors(const smc_state *st, double *lf);

/* Synchronous copies of the fitted proposal, D = 3 + 2 kappa_max + 2 lambda_max:
 * mu [S][M][D], U [S][M][D][D] (row j, column r = direction r), lam [S][M][D],
 * scale [S][M], ok [S][M] (entries past a model's own dimension are unused).
 * Any pointer may be NULL. */
int smc_get_adaptation(const smc_state *st, double *mu, double *U, double *lam, double *scale, int *ok);

/* Posterior predictive summaries (the goodness of fit of Section 4.1) over
 * each sounding's current particles, which after smc_run are equally weighted
 * draws from the posterior (models mixed by their counts): the forward model
 * of every particle, then per gate, in FP64,
 *   mean = (1/N) sum_i yhat_i,  var = (1/N) sum_i [v(yhat_i) + (yhat_i - mean)^2],
 *   z = (y - mean) / sqrt(var),  v(yhat) = eps_an^2 + (eps_mn yhat)^2,
 * the moments of p(y~ | y) = int p(y~ | theta) pi(theta | y) d theta and the
 * data standardised to it.  mean, var, z: [host] S x G (any may be NULL);
 * gates_host: [host] P x G predictions (may be NULL).  The first call
 * allocates P x G floats of device scratch held by the sampler.  Synchronous. */
int smc_ppd(smc_state *st, double *mean, double *var, double *z, float *gates_host);

/* Checkpoint / resume.  smc_checkpoint writes a self-describing image of the
 * sampler's dynamic state (current particles with their log-likelihoods,
 * gamma, log Z_k, stage counter, Langevin steps, the previous stage's
 * acceptance counts that set R_t; with desc.adaptive the proposal scale of
 * every (sounding, model), on which the next stage's bisection is centred;
 * with desc.recycle_stages = H the H history slots and the gamma and log Z_k
 * of every stage so far) into the caller's host buffer: with buf == NULL it
 * only stores the image size in *size; otherwise *size is the buffer's
 * capacity on entry (AEM_ERR_INVALID_ARG if too small) and the image's size
 * on return.  Take it between stages (after smc_mutate or smc_run returns):
 * the adaptive fit itself is rebuilt at the start of the next stage's
 * sweeps.  Synchronous.  smc_restore loads such an image into a sampler
 * created with the same n_soundings, n_particles, kappa_max, lambda_max,
 * adaptive flag and recycling window (AEM_ERR_INVALID_ARG otherwise, or for a
 * damaged or truncated image); the random streams are counter-based, so
 * resuming reproduces the uninterrupted run exactly when the descriptors
 * match. */
int smc_checkpoint(const smc_state *st, void *buf, size_t *size);
int smc_restore(smc_state *st, const void *buf, size_t size);

/* Standalone single-sounding forms of a7 and a8 on caller buffers
 * ([device] pointers; `work` is a [device] scratch buffer of at least
 * aem_smc_workspace_bytes(n, n_models) bytes, 64-byte aligned, owned by the
 * caller and overwritten). */
size_t aem_smc_workspace_bytes(int n, int n_models);
/* ll [n], model [n] (0..n_models-1): outputs dgamma [1], reached_one [1],
 * logz_inc [n_models] (0 for empty models) and W [n] normalised within each
 * model, for the step from gamma_prev.  A particle whose model id is outside
 * [0, n_models) takes no part (its W is 0).  ll must not hold NaN (the
 * sampler maps NaN to -inf before its reweight step); particles at -inf get
 * weight 0, and when no probed step keeps TESS >= alpha N the smallest probed
 * step, (1 - gamma_prev) 2^-bisect_iters, is returned (the sampler reports
 * that case as AEM_ERR_NO_BRACKET, see smc_status). */
int aem_reweight(const double *ll, const int *model, int n, int n_models, double gamma_prev, double alpha,
                 int bisect_iters, double *dgamma, int *reached_one, double *logz_inc, double *W, void *work,
                 size_t work_bytes, void *stream);
/* W [n] normalised within each model, model [n], u40 [n_models] integers in
 * [0, 2^40): ancestor [n] of every particle (bit-exact integer arithmetic).
 * A particle whose model id is outside [0, n_models) takes no part: its
 * ancestor is -1 and it is never chosen as one. */
int aem_resample_systematic(const double *W, const int *model, int n, int n_models, const unsigned long long *u40,
                            int *ancestor, void *work, size_t work_bytes, void *stream);
/* Resampling without any allocation.  The paper has no counterpart: this is
 * for callers that cannot call cudaMalloc or pass a workspace, e.g. code that
 * runs inside a host framework which owns all device memory through its own
 * pre-planned pool, or a latency-critical loop where an allocation (and the
 * device synchronisation it can cause) is not allowed.  Same inputs, outputs
 * and bit-exact result as aem_resample_systematic, but the scratch lives in a
 * fixed static device array of 512 KiB that every GPU loading the library
 * holds until the process exits.  Limits: n <= AEM_NOALLOC_MAX_PARTICLES,
 * n_models <= AEM_NOALLOC_MAX_MODELS; larger problems return
 * AEM_ERR_INVALID_ARG.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress, which allocates nothing); make that
 * first call before any stream capture.  All calls share the one array:
 * calls that may overlap on the GPU (different streams, or different host
 * threads on one device) race and must be serialised by the caller.  The
 * array keeps the last call's contents; every word a call reads is written
 * earlier in the same call, so no clearing is needed.  Calls no cudaMalloc,
 * cudaFree or allocating library routine. */
#define AEM_NOALLOC_MAX_PARTICLES 16384
#define AEM_NOALLOC_MAX_MODELS 100
int aem_resample_systematic_noalloc(const double *W, const int *model, int n, int n_models,
                                    const unsigned long long *u40, int *ancestor, void *stream);
/* Philox4x32-10 of n counters [device, n x 4] under key (key0, key1). */
int aem_philox4x32(const unsigned int *counters, unsigned int key0, unsigned int key1, unsigned int *out, int n,
                   void *stream);

/* ------------------------------------------------------------------------
 * Device throughput probes used for the roofline denominators: FP32 FMA,
 * MUFU ex2, FP64 FMA and the forward recursion's special-function mix (two
 * rsqrt, rcp, ex2, sin, cos per layer-step) measured by independent
 * dependency chains on every SM.  Synchronous.  Operations per second.
 * ---------------------------------------------------------------------- */
int aem_probe_peaks(double *fp32_fma_per_s, double *mufu_ex2_per_s, double *fp64_fma_per_s, double *mufu_mix_per_s);

#ifdef __cplusplus
}
#endif
#endif /* AEM_RJSMC_H */
