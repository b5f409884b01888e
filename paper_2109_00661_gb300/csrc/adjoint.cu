// Gradient of the Gaussian log-likelihood with respect to every merged
// layer's (log10 sigma, log10 h, m, log10 tau, c), by reverse-mode
// differentiation of the forward model (Section 2: Cole-Cole conductivity,
// TE recursion, Hankel sum; Section 2.3.2: gate transform and likelihood).
//
// The FP32 forward kernel (forward.cu) first writes every model's gates and
// log-likelihood.  Then one CTA per model (models claimed from a counter)
// forms the adjoint seeds from those gates,
//   a_f = sum_g T[g,f] dl/dyhat_g,  dl/dyhat = r/v + (e_mn^2 yhat / v)(r^2/v - 1),
// and visits every (frequency, abscissa) item with weight a_f w_k: the
// recursion is run bottom-up storing the reflection coefficients Gamma_j, then
// top-down propagating dGamma_0/dGamma_j through the Moebius steps
//   Gamma_j = (rho_j + Gamma_{j+1} E_j) / (1 + rho_j Gamma_{j+1} E_j),
//   rho_j = (s_{j-1} - s_j) / (u_{j-1} + u_j)^2,  E_j = exp(-2 u_j h_j),
//   u_j = sqrt(lambda^2 + s_j),
// and emitting, for each layer, Im(dGamma_0/ds_n ds_n/dp) and Im(dGamma_0/dh_n)
// into per-thread accumulators, reduced over the CTA at the end of the model.
// R_0 is holomorphic in every s_n, so d Im R_0 / dp = Im(dR_0/ds_n ds_n/dp)
// for the real parameters p.
#include <cuda_runtime.h>

#include <cstdint>

#include "aem_internal.h"

namespace aem {
namespace {

constexpr int kGT = 256;
constexpr int kGW = kGT / 32;
constexpr int kNP = 5;  // parameters per layer: log10 sigma, log10 h, m, log10 tau, c
constexpr unsigned kMask = 0xffffffffu;

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 crcp(float2 a) {
    const float d = 1.0f / fmaf(a.x, a.x, a.y * a.y);
    return make_float2(a.x * d, -a.y * d);
}
// The per-item passes use the hardware approximations of rcp, rsqrt, ex2,
// sin and cos (relative error about 2^-22; the FP32 forward kernel uses the
// same ones), the per-(frequency, layer) Cole-Cole setup the rounded library
// functions.
__device__ __forceinline__ float rcp_a(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float rsqrt_a(float v) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float2 crcp_a(float2 a) {
    const float d = rcp_a(fmaf(a.x, a.x, a.y * a.y));
    return make_float2(a.x * d, -a.y * d);
}
// principal root of x + i y, y > 0: with t = (|z| + |x|) / 2 the pair
// (sqrt t, y / (2 sqrt t)) is (Re, Im) for x >= 0 and (Im, Re) otherwise
__device__ __forceinline__ float2 csqrt_a(float x, float y) {
    const float v = fmaf(x, x, y * y);
    const float t = 0.5f * fmaf(v, rsqrt_a(v), fabsf(x));
    const float rr = rsqrt_a(t);
    const float p = t * rr, o = 0.5f * y * rr;
    return x >= 0.f ? make_float2(p, o) : make_float2(o, p);
}
__device__ __forceinline__ float2 cexp_a(float2 z) {
    float s, c, e;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(z.y));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(z.y));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(z.x * 1.44269504088896341f));
    return make_float2(e * c, e * s);
}

template <class T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kMask, v, o);
    return v;
}

struct GradModels {
    int n, lmax;
    const int8_t *nlayers;
    const float *logsig, *logh, *m, *logtau, *c;
};

// Shared memory (dynamic): S[F*LS] (float2 s), DS[F*LS*4] (float2 ds/dp for
// log10 sigma, m, log10 tau, c), lamhw[K] (float2 {lambda, weight}),
// af[F], T[G*F], part[kGW * LS * kNP] (float).
// MAXL: the largest layer count the per-thread arrays hold (10 or
// AEM_MAX_LAYERS), so the common lmax <= 10 keeps them half as large.
template <int MAXL>
__global__ void __launch_bounds__(kGT) loglik_grad_kernel(GradModels mv, int F, int G, int K, int LS,
                                                          const float *__restrict__ g_omega,
                                                          const float *__restrict__ g_lam,
                                                          const float *__restrict__ g_hw,
                                                          const float *__restrict__ g_T,
                                                          const double *__restrict__ y_obs, int obs_per,
                                                          const double *__restrict__ eps_an, double eps_mn,
                                                          const float *__restrict__ g_gates, float *__restrict__ grad,
                                                          int *__restrict__ work_counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *S = reinterpret_cast<float2 *>(smem_raw);
    float2 *DS = S + (size_t)F * LS;
    float2 *lamhw = DS + (size_t)F * LS * 4;
    float *af = reinterpret_cast<float *>(lamhw + K);
    float *Ts = af + F;
    float *part = Ts + (size_t)G * F;
    __shared__ float thick[AEM_MAX_LAYERS];
    __shared__ float sig_s[AEM_MAX_LAYERS], m_s[AEM_MAX_LAYERS], tau_s[AEM_MAX_LAYERS], c_s[AEM_MAX_LAYERS];
    __shared__ double dldy[AEM_MAX_GATES];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float mu0 = (float)kMu0, ln10 = 2.302585092994046f;
    for (int i = tid; i < G * F; i += blockDim.x) Ts[i] = g_T[i];
    for (int k = tid; k < K; k += blockDim.x) lamhw[k] = make_float2(g_lam[k], g_hw[k]);
    const int FK = F * K;

    // models are claimed from a counter as CTAs finish them (model costs vary
    // with the layer count, so a fixed stride would leave SMs idle at the end)
    __shared__ int next_model;
    for (int p = blockIdx.x; p < mv.n; p = next_model) {
        const int L = mv.nlayers[p];
        __syncthreads();
        if (tid == 0) next_model = (int)gridDim.x + atomicAdd(work_counter, 1);
        if (tid < L) {
            const size_t o = (size_t)p * mv.lmax + tid;
            sig_s[tid] = exp10f(mv.logsig[o]);
            thick[tid] = exp10f(mv.logh[o]);
            m_s[tid] = mv.m[o];
            tau_s[tid] = exp10f(mv.logtau[o]);
            c_s[tid] = mv.c[o];
        }
        __syncthreads();
        // Cole-Cole (paper form) and its derivatives, per (frequency, layer):
        // sig = s_inf (1 - m / (1 + x)), x = (w tau)^c e^{i pi c / 2}, s = i w mu0 sig
        for (int i = tid; i < F * L; i += blockDim.x) {
            const int f = i / L, n = i - f * L;
            const float w = g_omega[f];
            const float si = sig_s[n], mm = m_s[n], cc = c_s[n];
            const float lwt = logf(w * tau_s[n]);
            const float mag = expf(cc * lwt);
            float sp, cp;
            sincospif(0.5f * cc, &sp, &cp);
            const float2 x = make_float2(mag * cp, mag * sp);
            const float2 ix1 = crcp(make_float2(1.f + x.x, x.y));  // 1 / (1 + x)
            const float2 sg = make_float2(si * (1.f - mm * ix1.x), -si * mm * ix1.y);
            const float2 dsg_dm = cscale(ix1, -si);
            const float2 ix1sq = cmul(ix1, ix1);
            const float2 dsg_dx = cscale(ix1sq, si * mm);                 // s_inf m / (1 + x)^2
            const float2 dx_dlt = cscale(x, cc * ln10);                   // d x / d log10 tau
            const float2 dx_dc = cmul(x, make_float2(lwt, 1.57079632679489662f));
            const float2 iwm = make_float2(0.f, w * mu0);                 // i w mu0
            S[(size_t)f * LS + n] = cmul(iwm, sg);
            float2 *d = DS + ((size_t)f * LS + n) * 4;
            d[0] = cmul(iwm, cscale(sg, ln10));
            d[1] = cmul(iwm, dsg_dm);
            d[2] = cmul(iwm, cmul(dsg_dx, dx_dlt));
            d[3] = cmul(iwm, cmul(dsg_dx, dx_dc));
        }
        __syncthreads();

        // ---- dl/dyhat from the forward kernel's gates of this model
        if (tid < G) {
            const double yh = (double)g_gates[(size_t)p * G + tid];
            const double ea = eps_an[tid];
            const double v = ea * ea + (eps_mn * yh) * (eps_mn * yh);
            const double r = y_obs[(size_t)(p / obs_per) * G + tid] - yh;
            dldy[tid] = r / v + (eps_mn * eps_mn * yh / v) * (r * r / v - 1.0);
        }
        __syncthreads();
        for (int j = tid; j < F; j += blockDim.x) {
            double a = 0.0;
            for (int g = 0; g < G; ++g) a += (double)Ts[g * F + j] * dldy[g];
            af[j] = (float)a;
        }
        __syncthreads();

        // ---- pass 2: reverse sweep per item, per-thread accumulators
        float acc[MAXL * kNP];
        for (int v = 0; v < L * kNP; ++v) acc[v] = 0.f;
        // reflection coefficients of the bottom-up pass; with MAXL <= 10 also
        // its vertical wavenumbers and propagation factors, which the top-down
        // pass then reuses (for 20 layers the larger stack costs more than the
        // recomputation saves)
        constexpr bool kKeep = MAXL <= 10;
        constexpr int MK = kKeep ? MAXL : 1;
        float2 Gam[MAXL], Us[MK], Es[MK];
        int f = tid / K, k = tid - (tid / K) * K;
        for (int item = tid; item < FK; item += blockDim.x) {
            const float2 lh = lamhw[k];
            const float wgt = af[f] * lh.y;
            const float lam = lh.x, lam2 = lam * lam;
            const float2 *Sf = S + (size_t)f * LS;
            const float2 *Df = DS + (size_t)f * LS * 4;
            // bottom-up: Gamma_j for every interface j
            {
                float2 sb = Sf[L - 1];
                float2 ub = csqrt_a(lam2 + sb.x, sb.y);
                for (int j = L - 1; j >= 0; --j) {
                    if constexpr (kKeep) Us[j] = ub;
                    const float2 sa = j > 0 ? Sf[j - 1] : make_float2(0.f, 0.f);
                    const float2 ua = j > 0 ? csqrt_a(lam2 + sa.x, sa.y) : make_float2(lam, 0.f);
                    const float2 q = cadd(ua, ub);
                    const float2 rho = cmul(csub(sa, Sf[j]), crcp_a(cmul(q, q)));
                    if (j == L - 1) {
                        Gam[j] = rho;
                    } else {
                        const float2 E = cexp_a(cscale(ub, -2.f * thick[j]));
                        if constexpr (kKeep) Es[j] = E;
                        const float2 b = cmul(Gam[j + 1], E);
                        Gam[j] = cmul(cadd(rho, b), crcp_a(cadd(make_float2(1.f, 0.f), cmul(rho, b))));
                    }
                    ub = ua;
                }
            }
            // top-down: adjoints
            float2 gbar = make_float2(1.f, 0.f);
            float2 up = make_float2(lam, 0.f), sp = make_float2(0.f, 0.f);
            float2 ubar_p = make_float2(0.f, 0.f), sbar_p = make_float2(0.f, 0.f);
            for (int j = 0; j < L; ++j) {
                const float2 sj = Sf[j];
                float2 uj;
                if constexpr (kKeep)
                    uj = Us[j];
                else
                    uj = csqrt_a(lam2 + sj.x, sj.y);
                const float2 q = cadd(up, uj);
                const float2 iq = crcp_a(q);
                const float2 iq2 = cmul(iq, iq);
                const float2 rho = cmul(csub(sp, sj), iq2);
                float2 rbar, ubar_j = make_float2(0.f, 0.f), gnext = make_float2(0.f, 0.f);
                if (j < L - 1) {
                    const float h = thick[j];
                    float2 E;
                    if constexpr (kKeep)
                        E = Es[j];
                    else
                        E = cexp_a(cscale(uj, -2.f * h));
                    const float2 Gn = Gam[j + 1];
                    const float2 b = cmul(Gn, E);
                    const float2 iden = crcp_a(cadd(make_float2(1.f, 0.f), cmul(rho, b)));
                    const float2 iden2 = cmul(iden, iden);
                    rbar = cmul(gbar, cmul(csub(make_float2(1.f, 0.f), cmul(b, b)), iden2));
                    const float2 tbar = cmul(gbar, cmul(csub(make_float2(1.f, 0.f), cmul(rho, rho)), iden2));
                    const float2 Ebar = cmul(tbar, Gn);
                    gnext = cmul(tbar, E);
                    // d Gamma_0 / d h_j = Ebar (-2 u_j E);  d / d log10 h = h ln10 d / d h
                    const float2 hbar = cmul(Ebar, cscale(cmul(uj, E), -2.f));
                    acc[j * kNP + 1] += wgt * hbar.y * h * ln10;
                    ubar_j = cmul(Ebar, cscale(E, -2.f * h));
                } else {
                    rbar = gbar;
                }
                const float2 dq = cmul(rbar, cmul(cscale(rho, -2.f), iq));  // d rho / d u_{j-1} = d rho / d u_j
                if (j > 0) {
                    sbar_p = cadd(sbar_p, cmul(rbar, iq2));
                    ubar_p = cadd(ubar_p, dq);
                    // layer j-1 complete: s enters through u as well (du/ds = 1 / (2 u))
                    sbar_p = cadd(sbar_p, cmul(ubar_p, cscale(crcp_a(up), 0.5f)));
                    const float2 *d = Df + (size_t)(j - 1) * 4;
                    acc[(j - 1) * kNP + 0] += wgt * cmul(sbar_p, d[0]).y;
                    acc[(j - 1) * kNP + 2] += wgt * cmul(sbar_p, d[1]).y;
                    acc[(j - 1) * kNP + 3] += wgt * cmul(sbar_p, d[2]).y;
                    acc[(j - 1) * kNP + 4] += wgt * cmul(sbar_p, d[3]).y;
                }
                sbar_p = cscale(cmul(rbar, iq2), -1.f);
                ubar_p = cadd(ubar_j, dq);
                up = uj;
                sp = sj;
                gbar = gnext;
            }
            sbar_p = cadd(sbar_p, cmul(ubar_p, cscale(crcp_a(up), 0.5f)));
            {
                const float2 *d = Df + (size_t)(L - 1) * 4;
                acc[(L - 1) * kNP + 0] += wgt * cmul(sbar_p, d[0]).y;
                acc[(L - 1) * kNP + 2] += wgt * cmul(sbar_p, d[1]).y;
                acc[(L - 1) * kNP + 3] += wgt * cmul(sbar_p, d[2]).y;
                acc[(L - 1) * kNP + 4] += wgt * cmul(sbar_p, d[3]).y;
            }
            k += blockDim.x;
            while (k >= K) {
                k -= K;
                ++f;
            }
        }
        // CTA reduction of the per-thread accumulators (fixed order)
        for (int v = 0; v < L * kNP; ++v) {
            const float s = wsum<float>(acc[v]);
            if (lane == 0) part[warp * LS * kNP + v] = s;
        }
        __syncthreads();
        for (int v = tid; v < mv.lmax * kNP; v += blockDim.x) {
            float s = 0.f;
            if (v < L * kNP)
                for (int w = 0; w < kGW; ++w) s += part[w * LS * kNP + v];
            grad[(size_t)p * mv.lmax * kNP + v] = s;
        }
    }
}

}  // namespace
}  // namespace aem

using namespace aem;

namespace aem {

int loglik_grad_f32_soundings(const aem_system *sys, const aem_models_f32 *models, const double *y_obs,
                              int models_per_sounding, const double *eps_an, double eps_mn, double *ll, float *grad,
                              cudaStream_t stream) {
    const SystemTables &h = sys->host;
    if (h.cc_form != AEM_CC_PAPER)
        return fail(AEM_ERR_UNSUPPORTED, "aem_loglik_grad_f32: only the paper's Cole-Cole form is differentiated");
    const int LS = models->lmax;
    const size_t smem = sizeof(float2) * ((size_t)h.F * LS * 5 + h.K) +
                        sizeof(float) * ((size_t)h.F + (size_t)h.G * h.F + (size_t)kGW * LS * kNP);
    auto kern = LS <= 10 ? loglik_grad_kernel<10> : loglik_grad_kernel<AEM_MAX_LAYERS>;
    if (smem > 48 * 1024) AEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    AEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGT, smem));
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)sys->num_sms * per_sm;
    if (grid > models->n_models) grid = models->n_models;
    GradModels gm{models->n_models, models->lmax, models->nlayers, models->logsig, models->logh,
                  models->m, models->logtau, models->c};
    // stream-ordered scratch: the model count for the claim counter, then the gates
    void *work = nullptr;
    const size_t gate_off = 256;
    AEM_CUDA_TRY(cudaMallocAsync(&work, gate_off + sizeof(float) * (size_t)models->n_models * h.G, stream));
    int *counter = static_cast<int *>(work);
    float *gates = reinterpret_cast<float *>(static_cast<char *>(work) + gate_off);
    int rc = loglik_gates_f32_soundings(sys, models, y_obs, models_per_sounding, eps_an, eps_mn, ll, gates, stream);
    cudaError_t e = cudaSuccess;
    if (rc == AEM_OK) {
        e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
        if (e == cudaSuccess) {
            kern<<<(unsigned)grid, kGT, smem, stream>>>(gm, h.F, h.G, h.K, LS, sys->d_omega_f, sys->d_lam_f,
                                                        sys->d_hw_f, sys->d_T_f, y_obs, models_per_sounding, eps_an,
                                                        eps_mn, gates, grad, counter);
            e = cudaGetLastError();
        }
    }
    cudaFreeAsync(work, stream);
    if (rc) return rc;
    AEM_CUDA_TRY(e);
    return AEM_OK;
}

}  // namespace aem

extern "C" int aem_loglik_grad_f32(const aem_system *sys, const aem_models_f32 *models, const double *y_obs,
                                   const double *eps_an, double eps_mn, double *ll, float *grad, void *stream) {
    if (!sys || !models) return fail(AEM_ERR_INVALID_ARG, "aem_loglik_grad_f32: NULL system or models");
    if (models->n_models < 0 || models->lmax < 1 || models->lmax > AEM_MAX_LAYERS)
        return fail(AEM_ERR_INVALID_ARG, "aem_loglik_grad_f32: n_models < 0 or lmax outside 1..AEM_MAX_LAYERS");
    if (models->n_models == 0) return AEM_OK;
    if (!grad || !y_obs || !eps_an || !models->nlayers || !models->logsig || !models->logh || !models->m ||
        !models->logtau || !models->c)
        return fail(AEM_ERR_INVALID_ARG, "aem_loglik_grad_f32: NULL pointer");
    return loglik_grad_f32_soundings(sys, models, y_obs, models->n_models, eps_an, eps_mn, ll, grad,
                                     (cudaStream_t)stream);
}
