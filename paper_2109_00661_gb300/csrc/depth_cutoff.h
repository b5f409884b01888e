// The depth cutoff of the FP32 forward model and its adjoint (forward.cu,
// adjoint.cu; aem_system_set_depth_cutoff in include/aem_rjsmc.h).
//
// The TE recursion (Section 2, Ward & Hohmann's reflection form) runs from the
// basement up, but everything below layer j reaches R_0 through the round-trip
// attenuation exp(-2 sum_{i<=j} Re(u_i) h_i) of the layers above, u_i =
// sqrt(lambda^2 + s_i), s_i = i omega mu0 sigma_i.  Where that is under
// exp(-att), att = att0 + ln(max_n |s_n| / |s_0|), the deeper layers change R_0
// by less than exp(-att) times the largest reflection coefficient below, and
// the recursion may treat layer j as the half-space.  A lower bound of the
// attenuation suffices: Re u_i >= Re sqrt(s_i), and, as Re u grows with
// lambda^2, Re u_i >= sqrt(lambda^2 - ms) with ms = max_n(-Re s_n).
#pragma once

#include "f32x2.h"

namespace aem {

// th[j], j < L - 1: the lambda^2 above which the bound through layers 0..j
// exceeds att (-1: every lambda); non-increasing in j.  s(n) gives (Re s_n,
// Im s_n), h[n] the thicknesses.  The hardware approximations suffice: the
// thresholds only need to be right to well under the exp(-att0) margin.
template <class S>
__device__ __forceinline__ void depth_thresholds(S s, const float *h, int L, float att0, float *th) {
    using namespace f32x2;
    float s2max = 0.f, ms = 0.f;
    for (int n = 0; n < L; ++n) {
        const float2 a = s(n);
        s2max = fmaxf(s2max, fmaf(a.x, a.x, a.y * a.y));
        ms = fmaxf(ms, -a.x);
    }
    const float2 a0 = s(0);
    const float att = att0 + 0.5f * __logf(s2max * rcp_approx(fmaf(a0.x, a0.x, a0.y * a0.y)));
    float C = 0.f, H = 0.f;
    for (int j = 0; j + 1 < L; ++j) {
        const float2 a = s(j);
        const float m = sqrt_approx(fmaf(a.x, a.x, a.y * a.y));
        // Re sqrt(s_j) without cancellation
        const float rs = a.x >= 0.f ? sqrt_approx(0.5f * (m + a.x)) : 0.5f * fabsf(a.y) * rsqrt_approx(0.5f * (m - a.x));
        C = fmaf(2.f * h[j], rs, C);
        H += h[j];
        const float q = 0.5f * att * rcp_approx(H);
        th[j] = C > att ? -1.f : fmaf(q, q, ms);
    }
}

// The layer count one abscissa needs: 1 + the number of thresholds lambda^2
// does not exceed (a prefix, as th is non-increasing).
__device__ __forceinline__ int depth_layers(float lam2, const float *th, int L) {
    int c = 1;
    for (int j = 0; j + 1 < L; ++j) c += lam2 <= th[j] ? 1 : 0;
    return c;
}

}  // namespace aem
