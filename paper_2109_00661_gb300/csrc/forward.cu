// Batched forward model and Gaussian log-likelihood on sm_103a.
//
// One CTA works on one model at a time (grid-stride over models).  For that
// model it stages, in shared memory, s_n(w_f) = i w_f mu0 sigma_n(w_f) for every
// frequency node and merged layer (Cole-Cole, Section 2), then its threads
// sweep the flattened (frequency, Hankel abscissa) index space.  Each item runs
// the bottom-up TE reflection recursion over the layers (the hot loop: F*K*L
// layer-steps per model), weights Im R_0 by the folded Hankel weight and
// reduces over the abscissae of a frequency with a segmented warp sum into
// shared memory.  The epilogue applies the G x F step-off transform and, for
// the likelihood entry points, the Gaussian log-likelihood of Section 2.3.2
// with its sum in double precision.
//
// Recursion used (quasi-static TE mode, exp(+i w t)):
//   u_n = sqrt(lambda^2 + s_n), Re u_n > 0
//   r   = (s_n - s_{n+1}) / (u_n + u_{n+1})^2       (= (u_n - u_{n+1})/(u_n + u_{n+1}))
//   R_n = (r + R_{n+1} E) / (1 + r R_{n+1} E),  E = exp(-2 u_{n+1} h_{n+1})
// carried projectively as R = N / D so the Moebius step needs no division:
//   N' = r D + N E,  D' = D + r N E.  |D| grows by at most 2x per layer.
#include <cuda_runtime.h>

#include <cstdint>

#include "aem_internal.h"

namespace aem {
namespace {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

template <class R>
struct C2 {
    R x, y;
};

template <class R>
__device__ __forceinline__ C2<R> cmul(C2<R> a, C2<R> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// ---- precision-specific primitives ------------------------------------
struct FP32Ops {
    using R = float;
    // Hardware approximations (MUFU): rsqrt, rcp and sqrt(v) = v * rsqrt(v)
    // for v > 0 (every argument here is strictly positive).
    static __device__ __forceinline__ float rsq(float v) { return rsqrtf(v); }
    static __device__ __forceinline__ float sq(float v) { return v * rsqrtf(v); }
    static __device__ __forceinline__ float rcp(float v) { return __fdividef(1.0f, v); }
    static __device__ __forceinline__ void expsincos(float re, float im, float *e, float *s, float *c) {
        *e = __expf(re);
        __sincosf(im, s, c);
    }
};

struct FP64Ops {
    using R = double;
    static __device__ __forceinline__ double rsq(double v) { return rsqrt(v); }
    static __device__ __forceinline__ double sq(double v) { return sqrt(v); }
    static __device__ __forceinline__ double rcp(double v) { return 1.0 / v; }
    static __device__ __forceinline__ void expsincos(double re, double im, double *e, double *s, double *c) {
        *e = exp(re);
        sincos(im, s, c);
    }
};

// Principal square root of (x, y) with y >= 0 (Im s_n >= 0 for a passive
// medium): q = sqrt((|w| + |x|)/2); the other component is y / (2 q).
template <class Ops>
__device__ __forceinline__ C2<typename Ops::R> csqrt_upper(typename Ops::R x, typename Ops::R y) {
    using R = typename Ops::R;
    R mod = Ops::sq(x * x + y * y);
    R t = R(0.5) * (mod + fabs(x));
    R rq = Ops::rsq(t);
    R q = t * rq;
    R o = R(0.5) * y * rq;
    C2<R> u;
    u.x = (x >= R(0)) ? q : o;
    u.y = (x >= R(0)) ? o : q;
    return u;
}

// Im R_0 for one (lambda, frequency) pair; s points at this frequency's L
// layer values, thick at the L-1 finite thicknesses.
template <class Ops>
__device__ __forceinline__ typename Ops::R im_r0(typename Ops::R lam, typename Ops::R lam2,
                                                 const C2<typename Ops::R> *__restrict__ s,
                                                 const typename Ops::R *__restrict__ thick, int L) {
    using R = typename Ops::R;
    C2<R> sb = s[L - 1];
    C2<R> ub = csqrt_upper<Ops>(lam2 + sb.x, sb.y);
    C2<R> N = {R(0), R(0)}, D = {R(1), R(0)};
    bool first = true;
    for (int n = L - 2; n >= -1; --n) {
        C2<R> sn, un;
        if (n >= 0) {
            sn = s[n];
            un = csqrt_upper<Ops>(lam2 + sn.x, sn.y);
        } else {
            sn = {R(0), R(0)};
            un = {lam, R(0)};
        }
        // r = (s_n - s_below) / (u_n + u_below)^2
        C2<R> q = {un.x + ub.x, un.y + ub.y};
        R q2 = q.x * q.x + q.y * q.y;
        R iq2 = Ops::rcp(q2);
        R iq4 = iq2 * iq2;
        C2<R> qq = {q.x * q.x - q.y * q.y, R(-2) * q.x * q.y};  // conj(q^2)
        C2<R> A = {sn.x - sb.x, sn.y - sb.y};
        C2<R> r = cmul(A, qq);
        r.x *= iq4;
        r.y *= iq4;
        if (first) {
            N = r;
            first = false;
        } else {
            // E = exp(-2 u_below h_below)
            R hb = thick[n + 1];
            R e, sn_, cs_;
            Ops::expsincos(R(-2) * ub.x * hb, R(-2) * ub.y * hb, &e, &sn_, &cs_);
            C2<R> E = {e * cs_, e * sn_};
            C2<R> P = cmul(N, E);
            C2<R> rD = cmul(r, D);
            C2<R> rP = cmul(r, P);
            N = {rD.x + P.x, rD.y + P.y};
            D = {D.x + rP.x, D.y + rP.y};
        }
        sb = sn;
        ub = un;
    }
    R dd = D.x * D.x + D.y * D.y;
    return (N.y * D.x - N.x * D.y) * Ops::rcp(dd);
}

template <class R>
__device__ __forceinline__ R pow10r(R v);
template <>
__device__ __forceinline__ float pow10r<float>(float v) { return exp10f(v); }
template <>
__device__ __forceinline__ double pow10r<double>(double v) { return exp10(v); }

__device__ __forceinline__ void sincospi_r(float v, float *s, float *c) { sincospif(v, s, c); }
__device__ __forceinline__ void sincospi_r(double v, double *s, double *c) { sincospi(v, s, c); }

template <class R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

template <class Ops>
struct ModelsView {
    using R = typename Ops::R;
    int n, lmax;
    const int8_t *nlayers;
    const R *logsig, *logh, *m, *logtau, *c;
};

constexpr int kWarps = kThreads / 32;

// Shared memory layout (dynamic): s_tab[F * LMAX] complex, thick[LMAX],
// imh[F], T[G * F], lam[K], lam2[K], hw[K], imh_w[kWarps * F].
// Each warp owns one row of imh_w, so the Hankel sums are formed in a fixed
// order (no atomics) and the result does not depend on scheduling.
template <class Ops>
__global__ void __launch_bounds__(kThreads) forward_kernel(ModelsView<Ops> mv, int F, int G, int K, int cc_form,
                                                           const typename Ops::R *__restrict__ g_omega,
                                                           const typename Ops::R *__restrict__ g_lam,
                                                           const typename Ops::R *__restrict__ g_hw,
                                                           const typename Ops::R *__restrict__ g_T,
                                                           typename Ops::R *__restrict__ gates_out,
                                                           typename Ops::R *__restrict__ imh_out,
                                                           const double *__restrict__ y_obs, int obs_per,
                                                           const double *__restrict__ eps_an, double eps_mn,
                                                           double *__restrict__ ll_out) {
    using R = typename Ops::R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int LM = AEM_MAX_LAYERS;
    C2<R> *s_tab = reinterpret_cast<C2<R> *>(smem_raw);
    R *thick = reinterpret_cast<R *>(s_tab + (size_t)F * LM);
    R *imh = thick + LM;
    R *Ts = imh + F;
    R *lam_s = Ts + (size_t)G * F;
    R *lam2_s = lam_s + K;
    R *hw_s = lam2_s + K;
    R *imh_w = hw_s + K;
    __shared__ R lsig[AEM_MAX_LAYERS], lm[AEM_MAX_LAYERS], ltau[AEM_MAX_LAYERS], lc[AEM_MAX_LAYERS];
    __shared__ double ll_part[kThreads / 32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < G * F; i += blockDim.x) Ts[i] = g_T[i];
    for (int k = tid; k < K; k += blockDim.x) {
        R l = g_lam[k];
        lam_s[k] = l;
        lam2_s[k] = l * l;
        hw_s[k] = g_hw[k];
    }
    const R mu0 = R(kMu0);
    const int FK = F * K;

    for (int p = blockIdx.x; p < mv.n; p += gridDim.x) {
        const int L = mv.nlayers[p];
        __syncthreads();  // previous model's epilogue is done with imh / s_tab
        if (tid < L) {
            size_t o = (size_t)p * mv.lmax + tid;
            lsig[tid] = pow10r<R>(mv.logsig[o]);
            thick[tid] = pow10r<R>(mv.logh[o]);
            lm[tid] = mv.m[o];
            ltau[tid] = pow10r<R>(mv.logtau[o]);
            lc[tid] = mv.c[o];
        }
        for (int i = tid; i < kWarps * F; i += blockDim.x) imh_w[i] = R(0);
        __syncthreads();
        // Cole-Cole per (frequency, layer): x = (w tau)^c e^{i pi c / 2}
        for (int i = tid; i < F * L; i += blockDim.x) {
            int f = i / L, n = i - f * L;
            R w = g_omega[f];
            R sig = lsig[n], mm = lm[n];
            R sr = sig, si = R(0);
            if (mm != R(0)) {
                R cc = lc[n];
                R mag = exp(cc * log(w * ltau[n]));
                R sp, cp;
                sincospi_r(R(0.5) * cc, &sp, &cp);
                R xr = R(1) + mag * cp, xi = mag * sp;  // 1 + x
                R den = xr * xr + xi * xi;
                if (cc_form == AEM_CC_PAPER) {
                    // sigma_inf (1 - m / (1 + x))
                    sr = sig * (R(1) - mm * xr / den);
                    si = sig * (mm * xi / den);
                } else {
                    // sigma_0 (1 + x) / (1 + (1 - m) x)
                    R br = R(1) + (R(1) - mm) * mag * cp, bi = (R(1) - mm) * mag * sp;
                    R bd = br * br + bi * bi;
                    sr = sig * (xr * br + xi * bi) / bd;
                    si = sig * (xi * br - xr * bi) / bd;
                }
            }
            // s = i w mu0 sigma
            s_tab[(size_t)f * LM + n] = {-w * mu0 * si, w * mu0 * sr};
        }
        __syncthreads();

        // Hot loop over (frequency, abscissa) items.
        int f = tid / K, k = tid - (tid / K) * K;
        for (int base = 0; base < FK; base += blockDim.x) {
            const int item = base + tid;
            R val = R(0);
            int fl = -1;
            if (item < FK) {
                fl = f;
                val = hw_s[k] * im_r0<Ops>(lam_s[k], lam2_s[k], s_tab + (size_t)f * LM, thick, L);
            }
            // segmented warp reduction over lanes that share a frequency
            unsigned pending = __ballot_sync(kFull, fl >= 0);
            while (pending) {
                int leader = __ffs(pending) - 1;
                int fsel = __shfl_sync(kFull, fl, leader);
                R part = warp_sum<R>(fl == fsel ? val : R(0));
                if (lane == leader) imh_w[warp * F + fsel] += part;
                pending &= ~__ballot_sync(kFull, fl == fsel);
            }
            k += blockDim.x;
            while (k >= K) {
                k -= K;
                ++f;
            }
        }
        __syncthreads();
        for (int j = tid; j < F; j += blockDim.x) {
            R acc = R(0);
#pragma unroll
            for (int w = 0; w < kWarps; ++w) acc += imh_w[w * F + j];
            imh[j] = acc;
        }
        __syncthreads();

        // Epilogue: gates, optional Im H, optional log-likelihood.
        double term = 0.0;
        if (tid < G) {
            R acc = R(0);
            for (int j = 0; j < F; ++j) acc += Ts[tid * F + j] * imh[j];
            if (gates_out) gates_out[(size_t)p * G + tid] = acc;
            if (ll_out) {
                double yh = (double)acc;
                double ea = eps_an[tid];
                double v = ea * ea + (eps_mn * yh) * (eps_mn * yh);
                // models [s*obs_per, (s+1)*obs_per) share sounding s's data
                const double *yo = y_obs + (obs_per > 0 ? (size_t)(p / obs_per) * G : 0);
                double rr = yo[tid] - yh;
                term = rr * rr / v + log(2.0 * kPi * v);
            }
        }
        if (imh_out)
            for (int j = tid; j < F; j += blockDim.x) imh_out[(size_t)p * F + j] = imh[j];
        if (ll_out) {
            if (warp * 32 < G) {
                double t = warp_sum<double>(term);
                if (lane == 0) ll_part[warp] = t;
            }
            __syncthreads();
            if (tid == 0) {
                double acc = 0.0;
                for (int w = 0; w * 32 < G; ++w) acc += ll_part[w];
                ll_out[p] = -0.5 * acc;
            }
        }
    }
}

template <class Ops>
size_t smem_bytes(int F, int G, int K) {
    using R = typename Ops::R;
    return sizeof(C2<R>) * (size_t)F * AEM_MAX_LAYERS +
           sizeof(R) * (AEM_MAX_LAYERS + F + (size_t)G * F + 3 * (size_t)K + (size_t)kWarps * F);
}

template <class Ops, class Models>
int launch_forward(const aem_system *sys, const Models *models, typename Ops::R *gates, typename Ops::R *imh,
                   const double *y_obs, int obs_per, const double *eps_an, double eps_mn, double *ll, void *stream,
                   const typename Ops::R *omega, const typename Ops::R *lam, const typename Ops::R *hw,
                   const typename Ops::R *T, const char *name) {
    if (!sys || !models) return fail(AEM_ERR_INVALID_ARG, std::string(name) + ": NULL system or models");
    if (models->n_models < 0 || models->lmax < 1 || models->lmax > AEM_MAX_LAYERS)
        return fail(AEM_ERR_INVALID_ARG, std::string(name) + ": n_models < 0 or lmax outside 1..AEM_MAX_LAYERS");
    if (models->n_models == 0) return AEM_OK;
    if (!gates && !imh && !ll) return fail(AEM_ERR_INVALID_ARG, std::string(name) + ": no output requested");
    if (!models->nlayers || !models->logsig || !models->logh || !models->m || !models->logtau || !models->c)
        return fail(AEM_ERR_INVALID_ARG, std::string(name) + ": NULL model array");
    if (ll && (!y_obs || !eps_an)) return fail(AEM_ERR_INVALID_ARG, std::string(name) + ": NULL y_obs or eps_an");
    const SystemTables &h = sys->host;
    ModelsView<Ops> mv{models->n_models, models->lmax, models->nlayers, models->logsig, models->logh,
                       models->m, models->logtau, models->c};
    size_t smem = smem_bytes<Ops>(h.F, h.G, h.K);
    auto kern = forward_kernel<Ops>;
    if (smem > 48 * 1024) AEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    AEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)sys->num_sms * per_sm;
    if (grid > models->n_models) grid = models->n_models;
    kern<<<(unsigned)grid, kThreads, smem, (cudaStream_t)stream>>>(mv, h.F, h.G, h.K, h.cc_form, omega, lam, hw, T,
                                                                   gates, imh, y_obs, obs_per, eps_an, eps_mn, ll);
    AEM_CUDA_TRY(cudaGetLastError());
    return AEM_OK;
}

}  // namespace
}  // namespace aem

namespace aem {
int loglik_f32_soundings(const aem_system *sys, const aem_models_f32 *models, const double *y_obs,
                         int models_per_sounding, const double *eps_an, double eps_mn, double *ll,
                         cudaStream_t stream) {
    return launch_forward<FP32Ops>(sys, models, (float *)nullptr, (float *)nullptr, y_obs, models_per_sounding,
                                   eps_an, eps_mn, ll, (void *)stream, sys->d_omega_f, sys->d_lam_f, sys->d_hw_f,
                                   sys->d_T_f, "loglik (SMC)");
}
}  // namespace aem

using namespace aem;

extern "C" int aem_forward_f32(const aem_system *sys, const aem_models_f32 *models, float *gates, float *imh,
                               void *stream) {
    return launch_forward<FP32Ops>(sys, models, gates, imh, nullptr, 0, nullptr, 0.0, nullptr, stream,
                                   sys ? sys->d_omega_f : nullptr, sys ? sys->d_lam_f : nullptr,
                                   sys ? sys->d_hw_f : nullptr, sys ? sys->d_T_f : nullptr, "aem_forward_f32");
}

extern "C" int aem_forward_f64(const aem_system *sys, const aem_models_f64 *models, double *gates, double *imh,
                               void *stream) {
    return launch_forward<FP64Ops>(sys, models, gates, imh, nullptr, 0, nullptr, 0.0, nullptr, stream,
                                   sys ? sys->d_omega_d : nullptr, sys ? sys->d_lam_d : nullptr,
                                   sys ? sys->d_hw_d : nullptr, sys ? sys->d_T_d : nullptr, "aem_forward_f64");
}

extern "C" int aem_loglik_f32(const aem_system *sys, const aem_models_f32 *models, const double *y_obs,
                              const double *eps_an, double eps_mn, double *ll, float *gates, void *stream) {
    if (!ll && models && models->n_models > 0) return fail(AEM_ERR_INVALID_ARG, "aem_loglik_f32: ll is NULL");
    return launch_forward<FP32Ops>(sys, models, gates, nullptr, y_obs, 0, eps_an, eps_mn, ll, stream,
                                   sys ? sys->d_omega_f : nullptr, sys ? sys->d_lam_f : nullptr,
                                   sys ? sys->d_hw_f : nullptr, sys ? sys->d_T_f : nullptr, "aem_loglik_f32");
}

extern "C" int aem_loglik_f64(const aem_system *sys, const aem_models_f64 *models, const double *y_obs,
                              const double *eps_an, double eps_mn, double *ll, double *gates, void *stream) {
    if (!ll && models && models->n_models > 0) return fail(AEM_ERR_INVALID_ARG, "aem_loglik_f64: ll is NULL");
    return launch_forward<FP64Ops>(sys, models, gates, nullptr, y_obs, 0, eps_an, eps_mn, ll, stream,
                                   sys ? sys->d_omega_d : nullptr, sys ? sys->d_lam_d : nullptr,
                                   sys ? sys->d_hw_d : nullptr, sys ? sys->d_T_d : nullptr, "aem_loglik_f64");
}
