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
//
// Like the forward kernel, each thread carries two abscissae of one frequency
// (k and k + K/2) through both passes in 64-bit register pairs on the paired
// FP32 instructions (f32x2.h); the two abscissae's weighted adjoints are added
// before they meet the per-(frequency, layer) derivatives ds_n/dp, which do
// not depend on the abscissa.
#include <cuda_runtime.h>

#include <cstdint>

#include "aem_internal.h"
#include "depth_cutoff.h"
#include "f32x2.h"

namespace aem {
namespace {

using namespace f32x2;

constexpr int kGT = 256;
constexpr int kGW = kGT / 32;
constexpr int kNP = 5;  // parameters per layer: log10 sigma, log10 h, m, log10 tau, c
constexpr unsigned kMask = 0xffffffffu;

// scalar complex helpers of the per-(frequency, layer) Cole-Cole setup
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 crcp(float2 a) {
    const float d = 1.0f / fmaf(a.x, a.x, a.y * a.y);
    return make_float2(a.x * d, -a.y * d);
}

// paired complex helpers: two abscissae per operation
__device__ __forceinline__ C2x2 c2(u64 re, u64 im) {
    C2x2 r;
    r.re = re;
    r.im = im;
    return r;
}
__device__ __forceinline__ C2x2 c2add(C2x2 a, C2x2 b) { return c2(add2(a.re, b.re), add2(a.im, b.im)); }
__device__ __forceinline__ C2x2 c2neg(C2x2 a) { return c2(sub2(kZero2, a.re), sub2(kZero2, a.im)); }
__device__ __forceinline__ C2x2 c2add1(C2x2 a) { return c2(add2(kOne2, a.re), a.im); }         // 1 + a
__device__ __forceinline__ C2x2 c2mul(C2x2 a, C2x2 b) {
    return c2(sub2(mul2(a.re, b.re), mul2(a.im, b.im)), fma2(a.re, b.im, mul2(a.im, b.re)));
}
__device__ __forceinline__ C2x2 c2mulc(C2x2 a, C2x2 b) {  // a conj(b)
    return c2(fma2(a.re, b.re, mul2(a.im, b.im)), sub2(mul2(a.im, b.re), mul2(a.re, b.im)));
}
__device__ __forceinline__ C2x2 c2sq(C2x2 a) {
    const u64 t = mul2(a.re, a.im);
    return c2(mul2(sub2(a.re, a.im), add2(a.re, a.im)), add2(t, t));
}
__device__ __forceinline__ C2x2 c2scale(C2x2 a, u64 s) { return c2(mul2(a.re, s), mul2(a.im, s)); }
constexpr u64 kMinus2 = 0xc0000000c0000000ull;  // (-2, -2)
__device__ __forceinline__ C2x2 c2one_minus_sq(C2x2 a) {  // 1 - a^2
    return c2(fma2(a.im, a.im, sub2(kOne2, mul2(a.re, a.re))), mul2(mul2(a.re, a.im), kMinus2));
}
__device__ __forceinline__ u64 c2inorm(C2x2 a) {  // 1 / |a|^2
    float m0, m1;
    up2(fma2(a.re, a.re, mul2(a.im, a.im)), m0, m1);
    return pk2(rcp_approx(m0), rcp_approx(m1));
}
__device__ __forceinline__ C2x2 c2div(C2x2 x, C2x2 a) { return c2scale(c2mulc(x, a), c2inorm(a)); }

// Principal root u of z = lambda^2 + s (Im s > 0) for both abscissae, and
// 1 / (2 |z|) (= 1 / (2 |u|^2), for du/ds = 1 / (2 u) = conj(u) / (2 |z|)).  With t = (|z| + |x|) / 2 the pair
// (sqrt t, Im s / (2 sqrt t)) is (Re u, Im u) when x = Re z >= 0 and
// (Im u, Re u) otherwise.  s = ((Re s, Re s), (Im s, Im s)), y2 = (Im s)^2.
__device__ __forceinline__ C2x2 c2root(u64 lam2, ulonglong2 s, u64 y2, u64 &inv_mod) {
    const u64 x = add2(lam2, s.x);
    const u64 v = fma2(x, x, y2);
    float v0, v1, x0, x1;
    up2(v, v0, v1);
    up2(x, x0, x1);
    const u64 rv = pk2(rsqrt_approx(v0), rsqrt_approx(v1));  // v = |z|^2
    inv_mod = mul2(rv, kHalf2);
    const u64 t = mul2(add2(mul2(v, rv), pk2(fabsf(x0), fabsf(x1))), kHalf2);
    float t0, t1;
    up2(t, t0, t1);
    const u64 rr = pk2(rsqrt_approx(t0), rsqrt_approx(t1));
    float p0, p1, o0, o1;
    up2(mul2(t, rr), p0, p1);
    up2(mul2(mul2(s.y, kHalf2), rr), o0, o1);
    return c2(pk2(x0 >= 0.f ? p0 : o0, x1 >= 0.f ? p1 : o1), pk2(x0 >= 0.f ? o0 : p0, x1 >= 0.f ? o1 : p1));
}

// E = exp(-2 h u) for both abscissae; he = ((-2 h log2 e) x 2, (-2 h) x 2)
__device__ __forceinline__ C2x2 c2expm(ulonglong2 he, C2x2 u) {
    float a0, a1, f0, f1, s0, c0, s1, c1;
    up2(mul2(he.x, u.re), a0, a1);
    up2(reduce_2pi2(mul2(he.y, u.im)), f0, f1);
    sincos_approx(f0, &s0, &c0);
    sincos_approx(f1, &s1, &c1);
    const u64 e = pk2(ex2_approx(a0), ex2_approx(a1));
    return c2(mul2(e, pk2(c0, c1)), mul2(e, pk2(s0, s1)));
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

// Shared memory (dynamic), in order: RS[F*LS] (ulonglong2: (Re s, Re s),
// (Im s, Im s)), lamp[K2] (ulonglong2: (lam_a^2, lam_b^2), (lam_a, lam_b)),
// DS[F*LS*4] (float2 ds/dp for log10 sigma, m, log10 tau, c), RY2[F*LS] (u64:
// (Im s)^2 twice), hwp[K2] (float2 weights of the pair), af[F], T[G*F],
// part[kGW * LS * kNP], TH[F*LS] (float: the depth cutoff's thresholds).
size_t grad_smem_bytes(int F, int G, int K, int LS) {
    const size_t K2 = (size_t)(K + 1) / 2, FL = (size_t)F * LS;
    return sizeof(ulonglong2) * (FL + K2) + sizeof(float2) * (FL * 4) + sizeof(u64) * FL + sizeof(float2) * K2 +
           sizeof(float) * ((size_t)F + (size_t)G * F + (size_t)kGW * LS * kNP + FL);
}

// MAXL: the largest layer count the per-thread arrays hold (10 or
// AEM_MAX_LAYERS), so the common lmax <= 10 keeps them half as large.  Three
// resident CTAs per SM (80 registers) measured faster than two (128
// registers, no spills) and four (64 registers, 200 bytes spilled).
template <int MAXL>
__global__ void __launch_bounds__(kGT, 3) loglik_grad_kernel(GradModels mv, int F, int G, int K, int LS, int cc_form,
                                                          const float *__restrict__ g_omega,
                                                          const float *__restrict__ g_lam,
                                                          const float *__restrict__ g_hw,
                                                          const float *__restrict__ g_T,
                                                          const double *__restrict__ y_obs, int obs_per,
                                                          const double *__restrict__ eps_an, double eps_mn,
                                                          const float *__restrict__ g_gates, float *__restrict__ grad,
                                                          int *__restrict__ work_counter, float att0,
                                                          const int8_t *__restrict__ valid) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K2 = (K + 1) / 2;
    const size_t FL = (size_t)F * LS;
    ulonglong2 *RS = reinterpret_cast<ulonglong2 *>(smem_raw);
    ulonglong2 *lamp = RS + FL;
    float2 *DS = reinterpret_cast<float2 *>(lamp + K2);
    u64 *RY2 = reinterpret_cast<u64 *>(DS + FL * 4);
    float2 *hwp = reinterpret_cast<float2 *>(RY2 + FL);
    float *af = reinterpret_cast<float *>(hwp + K2);
    float *Ts = af + F;
    float *part = Ts + (size_t)G * F;
    float *TH = part + (size_t)kGW * LS * kNP;
    __shared__ ulonglong2 HE[AEM_MAX_LAYERS];
    __shared__ float thick[AEM_MAX_LAYERS];
    __shared__ float sig_s[AEM_MAX_LAYERS], m_s[AEM_MAX_LAYERS], tau_s[AEM_MAX_LAYERS], c_s[AEM_MAX_LAYERS];
    __shared__ double dldy[AEM_MAX_GATES];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float mu0 = (float)kMu0, ln10 = 2.302585092994046f;
    for (int i = tid; i < G * F; i += blockDim.x) Ts[i] = g_T[i];
    // abscissa pairs (k, k + K2); an odd K pads the last pair with a zero weight
    for (int k = tid; k < K2; k += blockDim.x) {
        const int kb = k + K2 < K ? k + K2 : K - 1;
        const float la = g_lam[k], lb = g_lam[kb];
        lamp[k] = make_ulonglong2(pk2(la * la, lb * lb), pk2(la, lb));
        hwp[k] = make_float2(g_hw[k], k + K2 < K ? g_hw[kb] : 0.f);
    }
    const int FK2 = F * K2;

    // models are claimed from a counter as CTAs finish them (model costs vary
    // with the layer count, so a fixed stride would leave SMs idle at the end)
    __shared__ int next_model;
    for (int p = blockIdx.x; p < mv.n; p = next_model) {
        const int L = mv.nlayers[p];
        __syncthreads();
        if (tid == 0) next_model = (int)gridDim.x + atomicAdd(work_counter, 1);
        if (valid && !valid[p]) {  // a proposal the caller will not use (CTA-uniform)
            __syncthreads();       // next_model visible to every thread
            continue;
        }
        if (tid < L) {
            const size_t o = (size_t)p * mv.lmax + tid;
            sig_s[tid] = exp10f(mv.logsig[o]);
            const float h = exp10f(mv.logh[o]);
            thick[tid] = h;
            const float a = -2.f * 1.44269504088896341f * h, b = -2.f * h;
            HE[tid] = make_ulonglong2(pk2(a, a), pk2(b, b));
            m_s[tid] = mv.m[o];
            tau_s[tid] = exp10f(mv.logtau[o]);
            c_s[tid] = mv.c[o];
        }
        __syncthreads();
        // Cole-Cole and its derivatives, per (frequency, layer), with
        // x = (w tau)^c e^{i pi c / 2} and s = i w mu0 sig:
        //   paper   sig = s_inf (1 - m / (1 + x))
        //   Pelton  sig = s_0 (1 + x) / (1 + (1 - m) x)
        //   literal sig = s_0 (1 + (1 - m) x) / (1 + x)
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
            float2 sg, dsg_dm, dsg_dx;
            // sig itself without cancellation, as the forward kernel forms it:
            // real parts as sums of non-negative terms (Re x >= 0), imaginary
            // parts as the single product m Im x / |.|^2
            if (cc_form == AEM_CC_PAPER) {
                // s_inf ((1 - m) + x) / (1 + x); ix1.y <= 0
                sg = make_float2(si * fmaf((1.f - mm) + x.x, ix1.x, -x.y * ix1.y), -si * mm * ix1.y);
                dsg_dm = cscale(ix1, -si);
                dsg_dx = cscale(cmul(ix1, ix1), si * mm);                // s_inf m / (1 + x)^2
            } else {
                const float2 b = make_float2(1.f + (1.f - mm) * x.x, (1.f - mm) * x.y);  // 1 + (1 - m) x
                if (cc_form == AEM_CC_PELTON) {
                    const float2 ib = crcp(b);                           // conj(b) / |b|^2
                    sg = make_float2(si * fmaf(1.f + x.x, ib.x, -x.y * ib.y), si * mm * x.y / (b.x * b.x + b.y * b.y));
                    dsg_dm = cmul(sg, cmul(x, ib));                      // sig x / (1 + (1 - m) x)
                    dsg_dx = cscale(cmul(ib, ib), si * mm);              // s_0 m / (1 + (1 - m) x)^2
                } else {
                    sg = make_float2(si * fmaf(b.x, ix1.x, -b.y * ix1.y), si * mm * ix1.y);
                    dsg_dm = cscale(cmul(x, ix1), -si);                  // -s_0 x / (1 + x)
                    dsg_dx = cscale(cmul(ix1, ix1), -si * mm);           // -s_0 m / (1 + x)^2
                }
            }
            const float2 dx_dlt = cscale(x, cc * ln10);                   // d x / d log10 tau
            const float2 dx_dc = cmul(x, make_float2(lwt, 1.57079632679489662f));
            const float2 iwm = make_float2(0.f, w * mu0);                 // i w mu0
            const float2 sv = cmul(iwm, sg);
            RS[(size_t)f * LS + n] = make_ulonglong2(pk2(sv.x, sv.x), pk2(sv.y, sv.y));
            RY2[(size_t)f * LS + n] = pk2(sv.y * sv.y, sv.y * sv.y);
            float2 *d = DS + ((size_t)f * LS + n) * 4;
            d[0] = cmul(iwm, cscale(sg, ln10));
            d[1] = cmul(iwm, dsg_dm);
            d[2] = cmul(iwm, cmul(dsg_dx, dx_dlt));
            d[3] = cmul(iwm, cmul(dsg_dx, dx_dc));
        }
        __syncthreads();

        // ---- the depth cutoff's thresholds (depth_cutoff.h), one frequency per
        // thread; each item then runs only the layers its abscissa needs (the
        // forward kernel runs at least those: the largest count of the item's
        // 32-item group), so a layer it drops contributes nothing to this
        // item's gradient, a change under exp(-att0) of the item's share
        const bool cut = att0 > 0.f && L > 1;
        if (cut)
            for (int f = tid; f < F; f += blockDim.x)
                depth_thresholds(
                    [&](int n) {
                        float sx, sy, t;
                        up2(RS[(size_t)f * LS + n].x, sx, t);
                        up2(RS[(size_t)f * LS + n].y, sy, t);
                        return make_float2(sx, sy);
                    },
                    thick, L, att0, TH + (size_t)f * LS);
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

        // ---- reverse sweep per pair of items, per-thread accumulators; the
        // log10 h entries hold sum w Im(u_j tb_j) until the reduction applies
        // -2 h_j ln10 (d Gamma_0 / d h_j = -2 u_j tb_j, tb_j as below)
        float acc[MAXL * kNP];
        for (int v = 0; v < L * kNP; ++v) acc[v] = 0.f;
        C2x2 Gam[MAXL];
        int f = tid / K2, k = tid - (tid / K2) * K2;
        for (int item = tid; item < FK2; item += blockDim.x) {
            const ulonglong2 lp = lamp[k];  // (lam^2 pair, lam pair)
            const float2 hw = hwp[k];
            const float a = af[f];
            const u64 wgt = pk2(a * hw.x, a * hw.y);
            const ulonglong2 *Sf = RS + (size_t)f * LS;
            const u64 *Yf = RY2 + (size_t)f * LS;
            const float2 *Df = DS + (size_t)f * LS * 4;
            const C2x2 air = c2(lp.y, kZero2);  // u of the air: lambda
            int Li = L;  // the layers this item runs
            if (cut) {
                float l2, lb2;
                up2(lp.x, l2, lb2);
                Li = depth_layers(l2, TH + (size_t)f * LS, L);
            }
            u64 imod;
            // bottom-up: Gamma_j for every interface j
            {
                C2x2 ub = c2root(lp.x, Sf[Li - 1], Yf[Li - 1], imod);
                for (int j = Li - 1; j >= 0; --j) {
                    const ulonglong2 sb = Sf[j];
                    C2x2 ua, dsab;  // u above the interface; s above minus s below
                    if (j > 0) {
                        const ulonglong2 sa = Sf[j - 1];
                        ua = c2root(lp.x, sa, Yf[j - 1], imod);
                        dsab = c2(sub2(sa.x, sb.x), sub2(sa.y, sb.y));
                    } else {
                        ua = air;
                        dsab = c2(sub2(kZero2, sb.x), sub2(kZero2, sb.y));
                    }
                    const C2x2 rho = c2div(dsab, c2sq(c2add(ua, ub)));
                    if (j == Li - 1) {
                        Gam[j] = rho;
                    } else {
                        const C2x2 b = c2mul(Gam[j + 1], c2expm(HE[j], ub));
                        Gam[j] = c2div(c2add(rho, b), c2add1(c2mul(rho, b)));
                    }
                    ub = ua;
                }
            }
            // top-down: adjoints.  gbar = d Gamma_0 / d Gamma_j; sbar_p, ubar_p
            // collect d Gamma_0 / d s_{j-1}, d / d u_{j-1} of the layer above
            C2x2 gbar = c2(kOne2, kZero2), up = air, sbar_p = c2(kZero2, kZero2), ubar_p = sbar_p;
            u64 imod_up = kZero2;
            ulonglong2 sp = make_ulonglong2(kZero2, kZero2);
            C2x2 uj = c2root(lp.x, Sf[0], Yf[0], imod);
            for (int j = 0; j < Li; ++j) {
                const ulonglong2 sj = Sf[j];
                const C2x2 q = c2add(up, uj);
                const u64 iqn = c2inorm(q);
                const C2x2 iqc = c2scale(q, iqn);  // conj(1 / q)
                const C2x2 iq2c = c2sq(iqc);       // conj(1 / q^2)
                const C2x2 rho = c2mulc(c2(sub2(sp.x, sj.x), sub2(sp.y, sj.y)), iq2c);
                C2x2 rbar, ubar_j = c2(kZero2, kZero2), gnext = ubar_j;
                if (j < Li - 1) {
                    const ulonglong2 he = HE[j];
                    const C2x2 E = c2expm(he, uj);
                    const C2x2 b = c2mul(Gam[j + 1], E);
                    // d Gamma_j / d rho = (1 - b^2) / den^2, d Gamma_j / d b = (1 - rho^2) / den^2
                    const C2x2 g2 = c2div(gbar, c2sq(c2add1(c2mul(rho, b))));
                    rbar = c2mul(g2, c2one_minus_sq(b));
                    const C2x2 tbar = c2mul(g2, c2one_minus_sq(rho));
                    // tb = tbar b = (d Gamma_0 / d E_j) E_j: d / d u_j through E_j is -2 h tb
                    const C2x2 tb = c2mul(tbar, b);
                    gnext = c2mul(tbar, E);
                    float h0, h1;
                    up2(mul2(wgt, fma2(uj.re, tb.im, mul2(uj.im, tb.re))), h0, h1);
                    acc[j * kNP + 1] += h0 + h1;
                    ubar_j = c2scale(tb, he.y);
                } else {
                    rbar = gbar;
                }
                // d rho / d u_{j-1} = d rho / d u_j = -2 rho / q; d rho / d s_{j-1} = 1 / q^2 = -d rho / d s_j
                // dq2 = rbar rho / q, so the rho term of d / d u is -2 dq2
                const C2x2 dq2 = c2mul(rbar, c2mulc(rho, iqc));
                const C2x2 rbi = c2mulc(rbar, iq2c);
                if (j > 0) {
                    // layer j-1 complete: s enters through u as well, du/ds = 1 / (2 u) = conj(u) / (2 |z|)
                    ubar_p = c2(fma2(dq2.re, kMinus2, ubar_p.re), fma2(dq2.im, kMinus2, ubar_p.im));
                    sbar_p = c2add(c2add(sbar_p, rbi), c2scale(c2mulc(ubar_p, up), imod_up));
                    float x0, x1, y0, y1;
                    up2(mul2(wgt, sbar_p.re), x0, x1);
                    up2(mul2(wgt, sbar_p.im), y0, y1);
                    const float swx = x0 + x1, swy = y0 + y1;
                    const float4 *d = reinterpret_cast<const float4 *>(Df + (size_t)(j - 1) * 4);
                    const float4 d01 = d[0], d23 = d[1];
                    float *ac = acc + (j - 1) * kNP;
                    ac[0] += fmaf(swx, d01.y, swy * d01.x);
                    ac[2] += fmaf(swx, d01.w, swy * d01.z);
                    ac[3] += fmaf(swx, d23.y, swy * d23.x);
                    ac[4] += fmaf(swx, d23.w, swy * d23.z);
                }
                sbar_p = c2neg(rbi);
                ubar_p = c2(fma2(dq2.re, kMinus2, ubar_j.re), fma2(dq2.im, kMinus2, ubar_j.im));
                up = uj;
                imod_up = imod;
                sp = sj;
                gbar = gnext;
                if (j + 1 < Li) uj = c2root(lp.x, Sf[j + 1], Yf[j + 1], imod);
            }
            {
                sbar_p = c2add(sbar_p, c2scale(c2mulc(ubar_p, up), imod_up));
                float x0, x1, y0, y1;
                up2(mul2(wgt, sbar_p.re), x0, x1);
                up2(mul2(wgt, sbar_p.im), y0, y1);
                const float swx = x0 + x1, swy = y0 + y1;
                const float4 *d = reinterpret_cast<const float4 *>(Df + (size_t)(Li - 1) * 4);
                const float4 d01 = d[0], d23 = d[1];
                float *ac = acc + (Li - 1) * kNP;
                ac[0] += fmaf(swx, d01.y, swy * d01.x);
                ac[2] += fmaf(swx, d01.w, swy * d01.z);
                ac[3] += fmaf(swx, d23.y, swy * d23.x);
                ac[4] += fmaf(swx, d23.w, swy * d23.z);
            }
            k += blockDim.x;
            while (k >= K2) {
                k -= K2;
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
            if (v < L * kNP) {
                for (int w = 0; w < kGW; ++w) s += part[w * LS * kNP + v];
                if (v % kNP == 1) s *= -2.f * thick[v / kNP] * ln10;
            }
            grad[(size_t)p * mv.lmax * kNP + v] = s;
        }
    }
}

}  // namespace
}  // namespace aem

using namespace aem;

namespace aem {

// scratch layout: the adjoint kernel's claim counter at 0, the forward
// kernel's at 64, the gates [P][G] from 256
constexpr size_t kGateOff = 256;
size_t grad_work_bytes(int n_models, int G) { return kGateOff + sizeof(float) * (size_t)n_models * G; }

int loglik_grad_f32_soundings(const aem_system *sys, const aem_models_f32 *models, const double *y_obs,
                              int models_per_sounding, const double *eps_an, double eps_mn, double *ll, float *grad,
                              cudaStream_t stream, void *work_ext, const int8_t *valid) {
    const SystemTables &h = sys->host;
    const int LS = models->lmax;
    const size_t smem = grad_smem_bytes(h.F, h.G, h.K, LS);
    auto kern = LS <= 10 ? loglik_grad_kernel<10> : loglik_grad_kernel<AEM_MAX_LAYERS>;
    // always: the static shared memory counts against the 48 KB default too
    AEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    AEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGT, smem));
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)sys->num_sms * per_sm;
    if (grid > models->n_models) grid = models->n_models;
    GradModels gm{models->n_models, models->lmax, models->nlayers, models->logsig, models->logh,
                  models->m, models->logtau, models->c};
    void *work = work_ext;
    if (!work_ext) AEM_CUDA_TRY(cudaMallocAsync(&work, grad_work_bytes(models->n_models, h.G), stream));
    int *counter = static_cast<int *>(work);
    int *fwd_counter = reinterpret_cast<int *>(static_cast<char *>(work) + 64);
    float *gates = reinterpret_cast<float *>(static_cast<char *>(work) + kGateOff);
    int rc = loglik_gates_f32_soundings(sys, models, y_obs, models_per_sounding, eps_an, eps_mn, ll, gates, stream,
                                        fwd_counter, valid);
    cudaError_t e = cudaSuccess;
    if (rc == AEM_OK) {
        e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
        if (e == cudaSuccess) {
            kern<<<(unsigned)grid, kGT, smem, stream>>>(gm, h.F, h.G, h.K, LS, h.cc_form, sys->d_omega_f, sys->d_lam_f,
                                                        sys->d_hw_f, sys->d_T_f, y_obs, models_per_sounding, eps_an,
                                                        eps_mn, gates, grad, counter, sys->depth_att, valid);
            e = cudaGetLastError();
        }
    }
    if (!work_ext) cudaFreeAsync(work, stream);
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
