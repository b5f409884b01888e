// RJSMC stage on the GPU (Davies et al., arXiv 2109.00661, Algorithm 1):
//   reweight  - per-model log-sum-exp sums in FP64, gamma_t by bisection on
//               TESS = sum_k ESS_k (Section 3.2.1, App. C), Z_k update (App. D);
//   resample  - within-model systematic resampling on an integer CDF;
//   mutate    - RJMCMC sweeps: conductive / chargeable birth and death with
//               prior-drawn properties (App. E), depth moves, component-wise
//               Gaussian random walks, then the batched forward model and the
//               tempered Metropolis-Hastings test;
//   odds      - model counts, pi(k|y) = N_k / N and the BFIPD statistic.
// Optionally each stage ends with within-model Langevin (MALA) sweeps on the
// particles' continuous parameters, driven by the adjoint gradient of the
// log-likelihood (adjoint.cu) mapped back through the direct sum.
// Soundings are independent: per-sounding kernels run one CTA per sounding,
// per-particle kernels one thread per particle.  Random numbers come from
// Philox4x32-10 keyed by (seed, sounding) and counted by (particle, purpose,
// stage, sweep), so every draw is reproducible and independent of scheduling.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "aem_internal.h"

namespace aem {
namespace {

constexpr int KS = AEM_SMC_SLOTS;  // interface slots per profile
constexpr int kMoves = 6;
constexpr int kGroupThreads = 1024;
constexpr int kClusterThreads = 512;  // per CTA of the cluster-split reweight step
constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kPurposeMove = 64, kPurposeValue = 65, kPurposeAccept = 66, kPurposeResample = 67;
// Langevin: acceptance uniform, and normal j of the proposal from words
// 2 (j % 2), 2 (j % 2) + 1 of the block with purpose kPurposeLangevin0 + j / 2.
constexpr int kPurposeLangevinAccept = 68, kPurposeLangevin0 = 72;
// Adaptive within-model proposal: trial draws of the scale bisection.
constexpr int kPurposePcaTrial = 69;
// Particle-space gradient slots: phi_b, phi_c[KS], z_c[KS], z_m[KS], m[KS],
// tau coordinate, c.
constexpr int GD = AEM_SMC_GRAD_DIM;
constexpr int G_PHIB = 0, G_PHIC = 1, G_ZC = 1 + AEM_SMC_SLOTS, G_ZM = 1 + 2 * AEM_SMC_SLOTS,
              G_MV = 1 + 3 * AEM_SMC_SLOTS, G_TAU = 1 + 4 * AEM_SMC_SLOTS, G_C = 2 + 4 * AEM_SMC_SLOTS;
static_assert(G_C + 1 == AEM_SMC_GRAD_DIM, "gradient slot layout");
// Prior draw layout: draw d is word d % 4 of the block with purpose d / 4.
constexpr int kPriorSlots = 16;
constexpr int D_KAPPA = 0, D_LAM = 1, D_PHIB = 2, D_TAU = 3, D_C = 4, D_ZC = 5, D_PHIC = D_ZC + kPriorSlots,
              D_ZM = D_PHIC + kPriorSlots, D_MV = D_ZM + kPriorSlots;
constexpr int kCdfBits = 40;

// ------------------------------------------------------------------ Philox
struct Key {
    uint32_t k0, k1;
};

__host__ __device__ inline Key stream_key(unsigned long long seed, int sounding) {
    return {(uint32_t)(seed & 0xffffffffull), (uint32_t)((seed >> 32) ^ (unsigned long long)(uint32_t)sounding)};
}

// Philox4x32 with 10 rounds (Salmon, Moraes, Dror & Shaw, SC 2011).
__host__ __device__ inline void philox(uint32_t c[4], Key key) {
    uint32_t k0 = key.k0, k1 = key.k1;
    for (int r = 0; r < 10; ++r) {  // fixed trip count: unrolled by the compiler
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ inline void block_draws(uint32_t out[4], Key key, uint32_t particle, uint32_t purpose, uint32_t stage,
                                   uint32_t sweep) {
    out[0] = particle;
    out[1] = purpose;
    out[2] = stage;
    out[3] = sweep;
    philox(out, key);
}

// Uniform on (0, 1): ((x >> 8) + 1/2) 2^-24, formed exactly in double.
__device__ inline double u01(uint32_t x) { return ((double)(x >> 8) + 0.5) * 5.9604644775390625e-08; }
__device__ inline double u01_53(uint32_t x0, uint32_t x1) {
    return ((double)(x0 >> 6) * 134217728.0 + (double)(x1 >> 5) + 0.5) * 1.1102230246251565e-16;
}
// Box-Muller, first output: sqrt(-2 ln u1) cos(2 pi u2), in double.
__device__ inline double gauss(uint32_t x0, uint32_t x1) {
    double u1 = u01(x0), u2 = u01(x1);
    return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// ---------------------------------------------------------- particle state
struct PState {
    int *kappa, *lam;
    float *phib, *tau, *c, *zc, *phic, *zm, *mv;
    double *ll;
};

struct Params {
    int N, S, kappa_max, lambda_max, M, LMS, tau_log_prior, adaptive, DM;
    double zca_prob;
    double zmax, phi_lo, phi_hi, logtau_lo, logtau_hi, step_phi, step_m, step_tau, step_c, step_z;
    unsigned long long seed;
};

__device__ inline void copy_particle(PState d, int i, PState s, int j) {
    d.kappa[i] = s.kappa[j];
    d.lam[i] = s.lam[j];
    d.phib[i] = s.phib[j];
    d.tau[i] = s.tau[j];
    d.c[i] = s.c[j];
#pragma unroll
    for (int q = 0; q < KS; ++q) {
        d.zc[i * KS + q] = s.zc[j * KS + q];
        d.phic[i * KS + q] = s.phic[j * KS + q];
        d.zm[i * KS + q] = s.zm[j * KS + q];
        d.mv[i * KS + q] = s.mv[j * KS + q];
    }
    d.ll[i] = s.ll[j];
}

// Stable insertion sort of (z, v) pairs by z.
__device__ inline void sort_pairs(double *z, double *v, int n) {
    for (int a = 1; a < n; ++a) {
        double kz = z[a], kv = v[a];
        int b = a - 1;
        while (b >= 0 && z[b] > kz) {
            z[b + 1] = z[b];
            v[b + 1] = v[b];
            --b;
        }
        z[b + 1] = kz;
        v[b + 1] = kv;
    }
}

// --------------------------------------------------------------- prior draw
__global__ void prior_kernel(PState st, Params pr) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pr.S * pr.N) return;
    int s = i / pr.N, j = i - s * pr.N;
    Key key = stream_key(pr.seed, s);
    auto draw = [&](int d) -> double {
        uint32_t w[4];
        block_draws(w, key, (uint32_t)j, (uint32_t)(d >> 2), 0u, 0u);
        return u01(w[d & 3]);
    };
    int kappa = (int)(draw(D_KAPPA) * (pr.kappa_max + 1));
    kappa = kappa > pr.kappa_max ? pr.kappa_max : kappa;
    int lam = (int)(draw(D_LAM) * (pr.lambda_max + 1));
    lam = lam > pr.lambda_max ? pr.lambda_max : lam;
    double phib = __dadd_rn(pr.phi_lo, __dmul_rn(pr.phi_hi - pr.phi_lo, draw(D_PHIB)));
    double tau;
    if (pr.tau_log_prior)
        tau = pow(10.0, __dadd_rn(pr.logtau_lo, __dmul_rn(pr.logtau_hi - pr.logtau_lo, draw(D_TAU))));
    else
        tau = draw(D_TAU);
    double c = draw(D_C);
    double zc[KS], phic[KS], zm[KS], mv[KS];
    for (int q = 0; q < kappa; ++q) {
        zc[q] = __dmul_rn(pr.zmax, draw(D_ZC + q));
        phic[q] = __dadd_rn(pr.phi_lo, __dmul_rn(pr.phi_hi - pr.phi_lo, draw(D_PHIC + q)));
    }
    for (int q = 0; q < lam; ++q) {
        zm[q] = __dmul_rn(pr.zmax, draw(D_ZM + q));
        mv[q] = draw(D_MV + q);
    }
    sort_pairs(zc, phic, kappa);
    sort_pairs(zm, mv, lam);
    st.kappa[i] = kappa;
    st.lam[i] = lam;
    st.phib[i] = (float)phib;
    st.tau[i] = (float)tau;
    st.c[i] = (float)c;
    for (int q = 0; q < KS; ++q) {
        st.zc[i * KS + q] = q < kappa ? (float)zc[q] : 0.f;
        st.phic[i * KS + q] = q < kappa ? (float)phic[q] : 0.f;
        st.zm[i * KS + q] = q < lam ? (float)zm[q] : 0.f;
        st.mv[i * KS + q] = q < lam ? (float)mv[q] : 0.f;
    }
    st.ll[i] = 0.0;
}

// ------------------------------------------------------------- merge (a1)
// Direct sum of the two profiles (Section 2.1, Fig. 2): the merged
// interfaces are the sorted union; each merged layer takes log10 sigma from
// the conductive profile and m from the chargeable profile at its top.
// T = float for the FP32 forward model, double for the plain FP64 one (the
// particle's own parameters are floats either way; thicknesses and log10 tau
// are formed in double and rounded to T).
template <class T>
__global__ void merge_kernel(PState st, int P, int LMS, int8_t *nl, T *logsig, T *logh, T *m, T *logtau, T *cc) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const int kappa = st.kappa[i], lam = st.lam[i];
    float z[2 * KS];
    int a = 0, b = 0, n = 0;
    while (a < kappa || b < lam) {
        float za = a < kappa ? st.zc[i * KS + a] : 3.0e38f;
        float zb = b < lam ? st.zm[i * KS + b] : 3.0e38f;
        if (za <= zb) {
            z[n++] = za;
            ++a;
        } else {
            z[n++] = zb;
            ++b;
        }
    }
    const int L = n + 1;
    const T lt = (T)log10((double)st.tau[i]);
    const T cv = st.c[i];
    int ic = 0, jm = 0;
    for (int q = 0; q < L; ++q) {
        float top = q == 0 ? 0.f : z[q - 1];
        if (q > 0) {
            while (ic < kappa && st.zc[i * KS + ic] <= top) ++ic;
            while (jm < lam && st.zm[i * KS + jm] <= top) ++jm;
        }
        size_t o = (size_t)i * LMS + q;
        logsig[o] = ic == 0 ? st.phib[i] : st.phic[i * KS + ic - 1];
        m[o] = jm == 0 ? T(0) : (T)st.mv[i * KS + jm - 1];
        double th = q < L - 1 ? (double)z[q] - (double)top : 1.0;
        logh[o] = (T)log10(th > 1e-30 ? th : 1e-30);
        logtau[o] = lt;
        cc[o] = cv;
    }
    for (int q = L; q < LMS; ++q) {
        size_t o = (size_t)i * LMS + q;
        logsig[o] = T(0);
        m[o] = T(0);
        logh[o] = T(0);
        logtau[o] = lt;
        cc[o] = cv;
    }
    nl[i] = (int8_t)L;
}

// ------------------------------------------------ grouping by model (stable)
// One CTA per sounding: counts N_k, offsets and the particle indices of each
// model in increasing index order (warp per model, ballot scans).
__global__ void __launch_bounds__(kGroupThreads) group_kernel(const int *kappa, const int *lam, int N, int lp1,
                                                              int M, int *perm, int *off, int *counts) {
    extern __shared__ unsigned char mid[];
    __shared__ int s_cnt[AEM_SMC_MAX_MODELS];
    __shared__ int s_off[AEM_SMC_MAX_MODELS + 1];
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int base = s * N;
    for (int j = tid; j < N; j += blockDim.x) mid[j] = (unsigned char)(kappa[base + j] * lp1 + lam[base + j]);
    __syncthreads();
    for (int k = warp; k < M; k += nw) {
        int cnt = 0;
        for (int b0 = 0; b0 < N; b0 += 32) {
            int j = b0 + lane;
            cnt += __popc(__ballot_sync(kFullMask, j < N && mid[j] == k));
        }
        if (lane == 0) s_cnt[k] = cnt;
    }
    __syncthreads();
    if (tid == 0) {
        s_off[0] = 0;
        for (int k = 0; k < M; ++k) s_off[k + 1] = s_off[k] + s_cnt[k];
    }
    __syncthreads();
    for (int k = warp; k < M; k += nw) {
        int pos = s_off[k];
        for (int b0 = 0; b0 < N; b0 += 32) {
            int j = b0 + lane;
            bool p = j < N && mid[j] == k;
            unsigned bal = __ballot_sync(kFullMask, p);
            if (p) perm[base + pos + __popc(bal & ((1u << lane) - 1u))] = base + j;
            pos += __popc(bal);
        }
    }
    for (int k = tid; k < M; k += blockDim.x) counts[s * M + k] = s_cnt[k];
    for (int k = tid; k <= M; k += blockDim.x) off[s * (M + 1) + k] = s_off[k];
}

template <class T>
__device__ inline T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
    return v;
}

__device__ inline double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFullMask, v, o));
    return v;
}

// -------------------------------------------------------------- reweight (a7)
// One CTA per sounding.  With W uniform within each model after the last
// resample, a_i = dgamma * ll_i, S1_k = sum e^{a_i - a_max}, S2_k = sum e^{2(a_i - a_max)},
// ESS_k = S1^2 / S2 and TESS = sum_k ESS_k.  gamma_t by bisection on TESS = alpha N.
// dense (dynamic shared memory of reweight_dense_bytes(N)): the sounding's
// log-likelihoods are staged once in model-grouped order, and each evaluation
// forms every particle's e^{a_i - a_max} once, one particle per thread, before
// the per-model sums read them (the FP64 exponentials are the step's cost on
// this part, and per-model lanes would leave most of them idle on small
// models); the sums, and so every result, are the same as without it.
constexpr int kDenseMaxParticles = 12000;
size_t reweight_dense_bytes(int N) {
    return N <= kDenseMaxParticles ? (size_t)N * (2 * sizeof(double) + 1) : 0;
}
__global__ void __launch_bounds__(kGroupThreads)
    reweight_kernel(const double *ll, const int *perm, const int *off, const int *counts, int N, int M, double alpha,
                    int iters, double *gamma, double *logz, double *Wg, double *dgamma_out, int *done_out,
                    int *status = nullptr, int dense = 0) {
    extern __shared__ __align__(16) unsigned char rw_smem[];
    double *sv = reinterpret_cast<double *>(rw_smem);               // [N] ll at each grouped position
    double *se = sv + N;                                             // [N] e^{a - a_max} of the evaluation
    unsigned char *spm = reinterpret_cast<unsigned char *>(se + N);  // [N] model at each grouped position
    __shared__ double s_max[AEM_SMC_MAX_MODELS], s_s1[AEM_SMC_MAX_MODELS], s_ess[AEM_SMC_MAX_MODELS];
    __shared__ double s_tess;
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int *o = off + s * (M + 1);
    const int *cnt = counts + s * M;
    const double g0 = gamma[s];
    if (g0 >= 1.0) {
        if (tid == 0) {
            dgamma_out[s] = 0.0;
            done_out[s] = 1;
        }
        return;
    }
    for (int k = warp; k < M; k += nw) {
        double mx = -INFINITY;
        for (int r = lane; r < cnt[k]; r += 32) mx = fmax(mx, ll[perm[s * N + o[k] + r]]);
        mx = warp_max(mx);
        if (lane == 0) s_max[k] = mx;
    }
    __syncthreads();
    // no particle of the sounding with a finite log-likelihood: there is no
    // weight to form; record AEM_ERR_NONFINITE, keep gamma and log Z, and
    // leave uniform weights within each model so the resample stays defined
    if (tid == 0) {
        bool any = false;
        for (int k = 0; k < M; ++k) any = any || s_max[k] > -INFINITY;
        s_tess = any ? 1.0 : 0.0;
    }
    __syncthreads();
    if (s_tess == 0.0) {
        for (int k = warp; k < M; k += nw)
            for (int r = lane; r < cnt[k]; r += 32) Wg[s * N + o[k] + r] = 1.0 / (double)cnt[k];
        if (tid == 0) {
            dgamma_out[s] = 0.0;
            done_out[s] = 0;
            if (status) atomicExch(status, (int)AEM_ERR_NONFINITE);
        }
        return;
    }
    if (dense) {
        for (int k = warp; k < M; k += nw)
            for (int r = lane; r < cnt[k]; r += 32) {
                sv[o[k] + r] = ll[perm[s * N + o[k] + r]];
                spm[o[k] + r] = (unsigned char)k;
            }
        __syncthreads();
    }
    auto evaluate = [&](double dg) {
        if (dense) {
            for (int q = tid; q < o[M]; q += blockDim.x) {
                const double v = sv[q];
                se[q] = (v == -INFINITY) ? 0.0 : exp(dg * (v - s_max[spm[q]]));
            }
            __syncthreads();
        }
        for (int k = warp; k < M; k += nw) {
            double s1 = 0.0, s2 = 0.0;
            const double mk = s_max[k];
            for (int r = lane; r < cnt[k]; r += 32) {
                double e;
                if (dense) {
                    e = se[o[k] + r];
                } else {
                    const double v = ll[perm[s * N + o[k] + r]];
                    e = (v == -INFINITY) ? 0.0 : exp(dg * (v - mk));
                }
                s1 += e;
                s2 += e * e;
            }
            s1 = warp_sum_t(s1);
            s2 = warp_sum_t(s2);
            if (lane == 0) {
                s_s1[k] = s1;
                s_ess[k] = (cnt[k] > 0 && s2 > 0.0) ? s1 * s1 / s2 : 0.0;
            }
        }
        __syncthreads();
        if (warp == 0) {
            double t = 0.0;
            for (int k = lane; k < M; k += 32) t += s_ess[k];
            t = warp_sum_t(t);
            if (lane == 0) s_tess = t;
        }
        __syncthreads();
        return s_tess;
    };
    const double target = alpha * (double)o[M];  // N, less any particle the grouping left out
    double hi = 1.0 - g0, dg;
    int done;
    if (evaluate(hi) >= target) {
        dg = hi;
        done = 1;
    } else {
        double lo = 0.0;
        for (int it = 0; it < iters; ++it) {
            double mid = 0.5 * (lo + hi);
            if (evaluate(mid) >= target)
                lo = mid;
            else
                hi = mid;
        }
        // lo = 0: no probed step kept TESS >= alpha N (more than (1 - alpha) N
        // particles with ll = -inf drop out at any positive step); take the
        // smallest probed step and record AEM_ERR_NO_BRACKET
        if (lo == 0.0 && status && tid == 0) atomicExch(status, (int)AEM_ERR_NO_BRACKET);
        dg = lo > 0.0 ? lo : hi;
        done = 0;
        evaluate(dg);
    }
    for (int k = warp; k < M; k += nw) {
        const int n = cnt[k];
        if (n == 0) continue;
        const double mk = s_max[k], s1 = s_s1[k];
        for (int r = lane; r < n; r += 32) {
            // the last evaluation was at dg: its e^{a - a_max} are in se
            double e;
            if (dense) {
                e = se[o[k] + r];
            } else {
                const double v = ll[perm[s * N + o[k] + r]];
                e = (v == -INFINITY) ? 0.0 : exp(dg * (v - mk));
            }
            Wg[s * N + o[k] + r] = e / s1;
        }
        if (lane == 0) logz[s * M + k] += dg * mk + log(s1) - log((double)n);
    }
    if (tid == 0) {
        gamma[s] = done ? 1.0 : g0 + dg;
        dgamma_out[s] = dg;
        done_out[s] = done;
    }
}

// The same reweight step split over a thread-block cluster of C CTAs per
// sounding, for samplers with few soundings and many particles (one CTA per
// sounding would leave most SMs idle while its FP64 sums run 60 bisection
// passes).  CTA r of the cluster takes the r-th of C equal slices of the
// sounding's model-grouped particle positions; every evaluation forms, per
// model, the partial sums S1, S2 (and once the maximum) over its slice, then
// after one cluster barrier every CTA adds the C partials of each model in
// rank order through distributed shared memory, so all CTAs evaluate TESS
// identically and take the same bisection decisions.  The partials are
// double-buffered: evaluation e writes buffer e mod 2, and the barrier of
// evaluation e + 1 is passed only after every CTA has read evaluation e's.
__global__ void __launch_bounds__(kClusterThreads)
    reweight_cluster_kernel(const double *ll, const int *perm, const int *off, const int *counts, int N, int M,
                            double alpha, int iters, double *gamma, double *logz, double *Wg, double *dgamma_out,
                            int *done_out, int *status) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    __shared__ double p_s1[2][AEM_SMC_MAX_MODELS], p_s2[2][AEM_SMC_MAX_MODELS], p_max[AEM_SMC_MAX_MODELS];
    __shared__ double s_max[AEM_SMC_MAX_MODELS], s_s1[AEM_SMC_MAX_MODELS], s_ess[AEM_SMC_MAX_MODELS];
    __shared__ double s_tess;
    const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int s = blockIdx.x / C, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int *o = off + s * (M + 1);
    const int *cnt = counts + s * M;
    const double g0 = gamma[s];
    if (g0 >= 1.0) {  // the same for every CTA of the cluster: none reaches a barrier
        if (tid == 0 && rank == 0) {
            dgamma_out[s] = 0.0;
            done_out[s] = 1;
        }
        return;
    }
    const int total = o[M];
    const int lo_pos = (int)((long long)total * rank / C), hi_pos = (int)((long long)total * (rank + 1) / C);
    // positions of model k inside this CTA's slice
    auto span = [&](int k, int &a, int &b) {
        a = o[k] > lo_pos ? o[k] : lo_pos;
        b = o[k + 1] < hi_pos ? o[k + 1] : hi_pos;
    };
    for (int k = warp; k < M; k += nw) {
        int a, b;
        span(k, a, b);
        double mx = -INFINITY;
        for (int q = a + lane; q < b; q += 32) mx = fmax(mx, ll[perm[s * N + q]]);
        mx = warp_max(mx);
        if (lane == 0) p_max[k] = mx;
    }
    cl.sync();
    for (int k = tid; k < M; k += blockDim.x) {
        double mx = -INFINITY;
        for (int q = 0; q < C; ++q) mx = fmax(mx, *cl.map_shared_rank(&p_max[k], q));
        s_max[k] = mx;
    }
    __syncthreads();
    if (tid == 0) {
        bool any = false;
        for (int k = 0; k < M; ++k) any = any || s_max[k] > -INFINITY;
        s_tess = any ? 1.0 : 0.0;
    }
    __syncthreads();
    if (s_tess == 0.0) {  // no finite log-likelihood in the sounding (see reweight_kernel)
        for (int k = warp; k < M; k += nw) {
            int a, b;
            span(k, a, b);
            for (int q = a + lane; q < b; q += 32) Wg[s * N + q] = 1.0 / (double)cnt[k];
        }
        if (tid == 0 && rank == 0) {
            dgamma_out[s] = 0.0;
            done_out[s] = 0;
            if (status) atomicExch(status, (int)AEM_ERR_NONFINITE);
        }
        cl.sync();  // no CTA leaves while another may still read its p_max
        return;
    }
    int buf = 0;
    auto evaluate = [&](double dg) {
        for (int k = warp; k < M; k += nw) {
            int a, b;
            span(k, a, b);
            double s1 = 0.0, s2 = 0.0;
            const double mk = s_max[k];
            for (int q = a + lane; q < b; q += 32) {
                const double v = ll[perm[s * N + q]];
                const double e = (v == -INFINITY) ? 0.0 : exp(dg * (v - mk));
                s1 += e;
                s2 += e * e;
            }
            s1 = warp_sum_t(s1);
            s2 = warp_sum_t(s2);
            if (lane == 0) {
                p_s1[buf][k] = s1;
                p_s2[buf][k] = s2;
            }
        }
        cl.sync();
        for (int k = tid; k < M; k += blockDim.x) {
            double s1 = 0.0, s2 = 0.0;
            for (int q = 0; q < C; ++q) {
                s1 += *cl.map_shared_rank(&p_s1[buf][k], q);
                s2 += *cl.map_shared_rank(&p_s2[buf][k], q);
            }
            s_s1[k] = s1;
            s_ess[k] = (cnt[k] > 0 && s2 > 0.0) ? s1 * s1 / s2 : 0.0;
        }
        __syncthreads();
        if (warp == 0) {
            double t = 0.0;
            for (int k = lane; k < M; k += 32) t += s_ess[k];
            t = warp_sum_t(t);
            if (lane == 0) s_tess = t;
        }
        __syncthreads();
        buf ^= 1;
        return s_tess;
    };
    const double target = alpha * (double)total;
    double hi = 1.0 - g0, dg;
    int done;
    if (evaluate(hi) >= target) {
        dg = hi;
        done = 1;
    } else {
        double lo = 0.0;
        for (int it = 0; it < iters; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (evaluate(mid) >= target)
                lo = mid;
            else
                hi = mid;
        }
        if (lo == 0.0 && status && tid == 0 && rank == 0) atomicExch(status, (int)AEM_ERR_NO_BRACKET);
        dg = lo > 0.0 ? lo : hi;
        done = 0;
        evaluate(dg);
    }
    for (int k = warp; k < M; k += nw) {
        int a, b;
        span(k, a, b);
        const double mk = s_max[k], s1 = s_s1[k];
        for (int q = a + lane; q < b; q += 32) {
            const double v = ll[perm[s * N + q]];
            Wg[s * N + q] = (v == -INFINITY) ? 0.0 : exp(dg * (v - mk)) / s1;
        }
    }
    if (rank == 0) {
        for (int k = tid; k < M; k += blockDim.x)
            if (cnt[k] > 0) logz[s * M + k] += dg * s_max[k] + log(s_s1[k]) - log((double)cnt[k]);
        if (tid == 0) {
            gamma[s] = done ? 1.0 : g0 + dg;
            dgamma_out[s] = dg;
            done_out[s] = done;
        }
    }
    cl.sync();  // every CTA's partials stay readable until all have finished
}

// Non-finite log-likelihoods (NaN, or +inf, which no Gaussian likelihood can
// reach) become -inf, so the particle carries zero weight and every proposal
// that produced one is rejected; each is counted per sounding.
__global__ void sanitize_ll_kernel(double *ll, int P, int N, int *nonfinite, const int *active = nullptr) {
    if (active && *active == 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const double v = ll[i];
    if (isnan(v) || v == INFINITY) {
        ll[i] = -INFINITY;
        atomicAdd(&nonfinite[i / N], 1);
    }
}

// ---------------------------------------------------------- model odds (a10)
// One thread per sounding, FP64: pi(k|y) = N_k / N and the BFIPD statistic of
// Section 2.3.3 with the sampler's uniform p(k) (uniform on kappa and on
// lambda), B = |M_kappa| sum_IP (pi / p) / (|M_lambda| sum_nonIP (pi / p)),
// |M_kappa| = kappa_max + 1 and |M_lambda| = (kappa_max + 1) lambda_max:
// +inf when no particle is non-chargeable, -inf when none is chargeable.
__global__ void odds_kernel(const int *counts, int S, int M, int lp1, int N, double *post, double *lbf) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const double pk = 1.0 / (double)M;
    double s_ip = 0.0, s_non = 0.0;
    for (int k = 0; k < M; ++k) {
        const double v = (double)counts[s * M + k] / (double)N;
        post[s * M + k] = v;
        if (k % lp1 == 0)
            s_non += v / pk;
        else
            s_ip += v / pk;
    }
    const double m_kappa = (double)(M / lp1), m_lambda = (double)(M / lp1) * (double)(lp1 - 1);
    if (s_non == 0.0)
        lbf[s] = INFINITY;
    else if (s_ip == 0.0)
        lbf[s] = -INFINITY;
    else
        lbf[s] = log(m_kappa * s_ip) - log(m_lambda * s_non);
}

// ------------------------------------------------------------- resample (a8)
// One CTA per sounding, warp per model.  q_r = round(W_r 2^40), C = prefix
// sums with the last entry forced to 2^40; output slot j takes the smallest r
// with C_r > floor((j 2^40 + u40_k) / N_k).
__global__ void __launch_bounds__(kGroupThreads)
    resample_kernel(const double *Wg, const int *perm, const int *off, const int *counts, int N, int M,
                    const unsigned long long *u40_in, unsigned long long seed, int stage, const int *stage_dev,
                    unsigned long long *C,
                    int *anc) {
    const int s = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int *o = off + s * (M + 1);
    const int *cnt = counts + s * M;
    const unsigned long long one = 1ull << kCdfBits;
    for (int k = warp; k < M; k += nw) {
        const int n = cnt[k];
        if (n == 0) continue;
        const int b = s * N + o[k];
        unsigned long long u40;
        if (u40_in) {
            u40 = u40_in[s * M + k];
        } else {
            uint32_t w[4];
            block_draws(w, stream_key(seed, s), (uint32_t)k, (uint32_t)kPurposeResample,
                        (uint32_t)(stage_dev ? *stage_dev : stage), 0u);
            u40 = (((unsigned long long)w[0] << 8) | (unsigned long long)(w[1] >> 24)) & (one - 1ull);
        }
        unsigned long long carry = 0;
        for (int r0 = 0; r0 < n; r0 += 32) {
            int r = r0 + lane;
            unsigned long long q = r < n ? (unsigned long long)__double2ll_rn(Wg[b + r] * (double)one) : 0ull;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                unsigned long long t = __shfl_up_sync(kFullMask, q, d);
                if (lane >= d) q += t;
            }
            if (r < n) C[b + r] = carry + q;
            carry += __shfl_sync(kFullMask, q, 31);
        }
        __syncwarp();
        if (lane == 0) C[b + n - 1] = one;
        __syncwarp();
        for (int j = lane; j < n; j += 32) {
            unsigned long long thr = ((unsigned long long)j * one + u40) / (unsigned long long)n;
            int lo = 0, hi = n - 1;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (C[b + mid] > thr)
                    hi = mid;
                else
                    lo = mid + 1;
            }
            anc[perm[b + j]] = perm[b + lo];
        }
    }
}

__global__ void gather_kernel(PState dst, PState src, const int *anc, int P) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P) copy_particle(dst, i, src, anc[i]);
}

// ---------------------------------------------------------- RJ proposal (a9)
// Adaptive principal-direction step (defined with the Langevin helpers below).
struct PcaView {
    const double *U, *lam, *a;
    const int *ok;
    const double *Z;  // ZCA roots U Lambda^(1/2) U^T [DM][DM] per (sounding, model)
};
__device__ bool pca_step(PState cur, PState prop, int i, int s, int kappa, int lam, const Params &pr, PcaView pv,
                         double a, double u_comp, double xi);
// Appendix F's ZCA-coloured birth / death (defined below): returns false when
// the move does not apply (no fit of the target model, or a full / empty
// profile), otherwise writes the proposal and sets ok and the log factor.
__device__ bool zca_move(PState cur, PState prop, int i, int s, bool birth, bool cond, const Params &pr, PcaView pv,
                         double u1, double xi, bool &ok, double &lf);
__device__ inline bool in_bounds_open(double v, double lo, double hi) { return lo < v && v < hi; }

__global__ void propose_kernel(PState cur, PState prop, int8_t *move_out, int8_t *valid_out, Params pr, int stage_arg,
                               int sweep, PcaView pv, const int *stage_dev, double *lf_out,
                               const int *active = nullptr) {
    if (active && *active == 0) return;  // a sweep beyond the device-side sweep count
    const int stage = stage_dev ? *stage_dev : stage_arg;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pr.S * pr.N) return;
    const int s = i / pr.N, j = i - s * pr.N;
    const Key key = stream_key(pr.seed, s);
    uint32_t d0[4], d1[4];
    block_draws(d0, key, (uint32_t)j, (uint32_t)kPurposeMove, (uint32_t)stage, (uint32_t)sweep);
    block_draws(d1, key, (uint32_t)j, (uint32_t)kPurposeValue, (uint32_t)stage, (uint32_t)sweep);
    const double u0 = u01(d0[0]), u1 = u01(d0[1]), u2 = u01(d0[2]);
    int move = (int)(u0 * 6.0);
    move = move > 5 ? 5 : move;
    copy_particle(prop, i, cur, i);
    int kappa = cur.kappa[i], lam = cur.lam[i];
    bool ok = true;
    double lf = 0.0;
    // a state-independent choice between the ZCA-coloured pair and the
    // prior-drawn one keeps the mixture reversible
    const bool zca = pr.adaptive && pr.zca_prob > 0.0 && move <= 3 && u01(d1[3]) < pr.zca_prob &&
                     zca_move(cur, prop, i, s, move == 0 || move == 2, move <= 1, pr, pv, u1, gauss(d1[1], d1[2]),
                              ok, lf);
    if (zca) {
        // proposal written by zca_move
    } else if (move == 0 || move == 2) {  // birth: depth U(0, zmax), property from the prior
        const bool cond = move == 0;
        const int n = cond ? kappa : lam;
        if (n >= (cond ? pr.kappa_max : pr.lambda_max)) {
            ok = false;
        } else {
            float *zz = cond ? prop.zc : prop.zm;
            float *vv = cond ? prop.phic : prop.mv;
            const double z = __dmul_rn(pr.zmax, u1);
            const double v = cond ? __dadd_rn(pr.phi_lo, __dmul_rn(pr.phi_hi - pr.phi_lo, u2)) : u2;
            int at = 0;
            while (at < n && (double)zz[i * KS + at] < z) ++at;
            for (int q = n; q > at; --q) {
                zz[i * KS + q] = zz[i * KS + q - 1];
                vv[i * KS + q] = vv[i * KS + q - 1];
            }
            zz[i * KS + at] = (float)z;
            vv[i * KS + at] = (float)v;
            if (cond)
                prop.kappa[i] = kappa + 1;
            else
                prop.lam[i] = lam + 1;
        }
    } else if (move == 1 || move == 3) {  // death of a uniformly chosen interface
        const bool cond = move == 1;
        const int n = cond ? kappa : lam;
        if (n == 0) {
            ok = false;
        } else {
            int at = (int)(u1 * n);
            at = at > n - 1 ? n - 1 : at;
            float *zz = cond ? prop.zc : prop.zm;
            float *vv = cond ? prop.phic : prop.mv;
            for (int q = at; q < n - 1; ++q) {
                zz[i * KS + q] = zz[i * KS + q + 1];
                vv[i * KS + q] = vv[i * KS + q + 1];
            }
            zz[i * KS + n - 1] = 0.f;
            vv[i * KS + n - 1] = 0.f;
            if (cond)
                prop.kappa[i] = kappa - 1;
            else
                prop.lam[i] = lam - 1;
        }
    } else if (move == 4) {  // depth move, order kept within the profile
        const int nint = kappa + lam;
        if (nint == 0) {
            ok = false;
        } else {
            int at = (int)(u1 * nint);
            at = at > nint - 1 ? nint - 1 : at;
            const double step = pr.step_z * gauss(d1[1], d1[2]);
            float *zz = at < kappa ? prop.zc : prop.zm;
            const int n = at < kappa ? kappa : lam;
            const int q = at < kappa ? at : at - kappa;
            const double z = (double)zz[i * KS + q] + step;
            const double lo = q > 0 ? (double)zz[i * KS + q - 1] : 0.0;
            const double hi = q + 1 < n ? (double)zz[i * KS + q + 1] : pr.zmax;
            if (!(lo < z && z < hi))
                ok = false;
            else
                zz[i * KS + q] = (float)z;
        }
    } else if (pr.adaptive && pv.ok[s * pr.M + kappa * (pr.lambda_max + 1) + lam]) {
        // the paper's adaptive move: a random walk along a principal direction
        // of the model's fitted Gaussian (Section 3.2)
        const int k = s * pr.M + kappa * (pr.lambda_max + 1) + lam;
        ok = pca_step(cur, prop, i, s, kappa, lam, pr, pv, pv.a[k], u1, gauss(d1[1], d1[2]));
    } else {  // component-wise Gaussian random walk
        const int ncomp = 1 + kappa + lam + 2;
        int at = (int)(u1 * ncomp);
        at = at > ncomp - 1 ? ncomp - 1 : at;
        const double g = gauss(d1[1], d1[2]);
        if (at == 0) {
            double v = (double)cur.phib[i] + pr.step_phi * g;
            ok = in_bounds_open(v, pr.phi_lo, pr.phi_hi);
            prop.phib[i] = (float)v;
        } else if (at <= kappa) {
            double v = (double)cur.phic[i * KS + at - 1] + pr.step_phi * g;
            ok = in_bounds_open(v, pr.phi_lo, pr.phi_hi);
            prop.phic[i * KS + at - 1] = (float)v;
        } else if (at <= kappa + lam) {
            double v = (double)cur.mv[i * KS + at - 1 - kappa] + pr.step_m * g;
            ok = in_bounds_open(v, 0.0, 1.0);
            prop.mv[i * KS + at - 1 - kappa] = (float)v;
        } else if (at == kappa + lam + 1) {
            double v;
            if (pr.tau_log_prior) {
                double lt = log10((double)cur.tau[i]) + pr.step_tau * g;
                ok = in_bounds_open(lt, pr.logtau_lo, pr.logtau_hi);
                v = pow(10.0, lt);
            } else {
                v = (double)cur.tau[i] + pr.step_tau * g;
                ok = in_bounds_open(v, 0.0, 1.0);
            }
            prop.tau[i] = (float)v;
        } else {
            double v = (double)cur.c[i] + pr.step_c * g;
            ok = in_bounds_open(v, 0.0, 1.0);
            prop.c[i] = (float)v;
        }
    }
    if (!ok) copy_particle(prop, i, cur, i);
    move_out[i] = (int8_t)move;
    valid_out[i] = ok ? 1 : 0;
    if (lf_out) lf_out[i] = lf;
}

// Tempered Metropolis-Hastings test: accept when ln u < gamma_t (l' - l).
// With prior-drawn birth properties and uniform move selection the prior and
// proposal ratios cancel (App. E), and the random walks are symmetric inside
// the uniform prior support.
__global__ void accept_kernel(PState cur, PState prop, const int8_t *move, const int8_t *valid, const double *gamma,
                              Params pr, int stage_arg, int sweep, int *acc, int *nprop, const int *stage_dev,
                              const double *lf, const int *active = nullptr) {
    if (active && *active == 0) return;
    const int stage = stage_dev ? *stage_dev : stage_arg;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pr.S * pr.N) return;
    const int s = i / pr.N, j = i - s * pr.N;
    const int mv = move[i];
    atomicAdd(&nprop[s * kMoves + mv], 1);
    if (!valid[i]) return;
    uint32_t w[4];
    block_draws(w, stream_key(pr.seed, s), (uint32_t)j, (uint32_t)kPurposeAccept, (uint32_t)stage, (uint32_t)sweep);
    const double u = u01_53(w[0], w[1]);
    const double dl = prop.ll[i] - cur.ll[i];
    if (log(u) < gamma[s] * dl + (lf ? lf[i] : 0.0)) {
        copy_particle(cur, i, prop, i);
        atomicAdd(&acc[s * kMoves + mv], 1);
    }
}

// ------------------------------------------------- Langevin (MALA) moves
// Chain rule from the merged-layer gradient [P][LMS][5] of (log10 sigma,
// log10 h, m, log10 tau, c) to the particle's parameters, following the
// direct sum of merge_kernel (same interface order, same tie rule): a layer's
// log10 sigma belongs to phi_b or the conductive value above it, its m to the
// chargeable value above it; an interface at merged position q thickens layer
// q and thins layer q + 1; tau and c are shared by every layer.
__global__ void pgrad_kernel(PState st, const float *mgrad, int P, int LMS, int tau_log_prior, float *pg) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const int kappa = st.kappa[i], lam = st.lam[i];
    float z[2 * KS];
    int src[2 * KS];  // >= 0: conductive index; < 0: -(chargeable index) - 1
    int a = 0, b = 0, n = 0;
    while (a < kappa || b < lam) {
        float za = a < kappa ? st.zc[i * KS + a] : 3.0e38f;
        float zb = b < lam ? st.zm[i * KS + b] : 3.0e38f;
        if (za <= zb) {
            src[n] = a;
            z[n++] = za;
            ++a;
        } else {
            src[n] = -b - 1;
            z[n++] = zb;
            ++b;
        }
    }
    const int L = n + 1;
    float g[GD];
#pragma unroll
    for (int q = 0; q < GD; ++q) g[q] = 0.f;
    double dl_dh[2 * KS + 1];
    double slt = 0.0, sc = 0.0;
    const double ln10 = 2.302585092994046;
    int ic = 0, jm = 0;
    for (int q = 0; q < L; ++q) {
        const float top = q == 0 ? 0.f : z[q - 1];
        if (q > 0) {
            while (ic < kappa && st.zc[i * KS + ic] <= top) ++ic;
            while (jm < lam && st.zm[i * KS + jm] <= top) ++jm;
        }
        const float *gm = mgrad + ((size_t)i * LMS + q) * 5;
        if (ic == 0)
            g[G_PHIB] += gm[0];
        else
            g[G_PHIC + ic - 1] += gm[0];
        if (jm > 0) g[G_MV + jm - 1] += gm[2];
        if (q < L - 1) {
            double th = (double)z[q] - (double)top;
            th = th > 1e-30 ? th : 1e-30;
            dl_dh[q] = (double)gm[1] / (th * ln10);
        }
        slt += gm[3];
        sc += gm[4];
    }
    for (int q = 0; q < n; ++q) {
        const double d = dl_dh[q] - (q + 1 < n ? dl_dh[q + 1] : 0.0);
        if (src[q] >= 0)
            g[G_ZC + src[q]] += (float)d;
        else
            g[G_ZM - src[q] - 1] += (float)d;
    }
    g[G_TAU] = tau_log_prior ? (float)slt : (float)(slt / ((double)st.tau[i] * ln10));
    g[G_C] = (float)sc;
#pragma unroll
    for (int q = 0; q < GD; ++q) pg[(size_t)i * GD + q] = g[q];
}

// Component j of the particle's continuous vector theta (phi_b, phi_c[kappa],
// z_c[kappa], z_m[lambda], m[lambda], tau coordinate, c): its storage, its
// gradient slot and its preconditioner scale (the random walk's step).
struct ThetaRef {
    float *x;
    int slot;
    double scale;
    bool is_tau;
};

__device__ inline ThetaRef theta_ref(PState ps, int i, int j, int kappa, int lam, const Params &pr) {
    if (j == 0) return {&ps.phib[i], G_PHIB, pr.step_phi, false};
    j -= 1;
    if (j < kappa) return {&ps.phic[i * KS + j], G_PHIC + j, pr.step_phi, false};
    j -= kappa;
    if (j < kappa) return {&ps.zc[i * KS + j], G_ZC + j, pr.step_z, false};
    j -= kappa;
    if (j < lam) return {&ps.zm[i * KS + j], G_ZM + j, pr.step_z, false};
    j -= lam;
    if (j < lam) return {&ps.mv[i * KS + j], G_MV + j, pr.step_m, false};
    j -= lam;
    if (j == 0) return {&ps.tau[i], G_TAU, pr.step_tau, true};
    return {&ps.c[i], G_C, pr.step_c, false};
}

__device__ inline double theta_value(const ThetaRef &r, const Params &pr) {
    const double v = (double)*r.x;
    return (r.is_tau && pr.tau_log_prior) ? log10(v) : v;
}

__device__ inline bool ordered_open(const float *z, int n, double zmax) {
    for (int q = 0; q < n; ++q) {
        const double lo = q > 0 ? (double)z[q - 1] : 0.0;
        if (!((double)z[q] > lo)) return false;
    }
    return n == 0 || (double)z[n - 1] < zmax;
}

// Preconditioned Langevin proposal at gamma_t:
//   theta' = theta + (h^2 / 2) D gamma_t grad l(theta) + h D^(1/2) xi,
//   D = diag(scale_j^2), xi ~ N(0, I);
// valid when theta' is inside the uniform prior support with ordered
// interfaces; lq = log q(theta' | theta) = -|xi|^2 / 2 (+ const).
__global__ void langevin_propose_kernel(PState cur, PState prop, const float *gcur, const double *gamma,
                                        const double *lang_h, Params pr, int stage_arg, int sweep, int8_t *valid_out,
                                        double *lq, const int *stage_dev) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pr.S * pr.N) return;
    const int stage = stage_dev ? *stage_dev : stage_arg;
    const int s = i / pr.N, jp = i - s * pr.N;
    const Key key = stream_key(pr.seed, s);
    copy_particle(prop, i, cur, i);
    const int kappa = cur.kappa[i], lam = cur.lam[i];
    const int d = 3 + 2 * kappa + 2 * lam;
    const double gm = gamma[s], h = lang_h[s];
    double lqf = 0.0;
    uint32_t w[4];
    for (int j = 0; j < d; ++j) {
        if ((j & 1) == 0)
            block_draws(w, key, (uint32_t)jp, (uint32_t)(kPurposeLangevin0 + j / 2), (uint32_t)stage,
                        (uint32_t)sweep);
        const double xi = gauss(w[2 * (j & 1)], w[2 * (j & 1) + 1]);
        const ThetaRef rc = theta_ref(cur, i, j, kappa, lam, pr);
        const ThetaRef rp = theta_ref(prop, i, j, kappa, lam, pr);
        const double sc = rc.scale;
        const double th = theta_value(rc, pr) + 0.5 * h * h * sc * sc * gm * (double)gcur[(size_t)i * GD + rc.slot] +
                          h * sc * xi;
        *rp.x = (float)((rp.is_tau && pr.tau_log_prior) ? pow(10.0, th) : th);
        lqf -= 0.5 * xi * xi;
    }
    bool ok = in_bounds_open(prop.phib[i], pr.phi_lo, pr.phi_hi) && in_bounds_open(prop.c[i], 0.0, 1.0);
    for (int q = 0; q < kappa; ++q) ok = ok && in_bounds_open(prop.phic[i * KS + q], pr.phi_lo, pr.phi_hi);
    for (int q = 0; q < lam; ++q) ok = ok && in_bounds_open(prop.mv[i * KS + q], 0.0, 1.0);
    ok = ok && ordered_open(prop.zc + (size_t)i * KS, kappa, pr.zmax) &&
         ordered_open(prop.zm + (size_t)i * KS, lam, pr.zmax);
    if (pr.tau_log_prior)
        ok = ok && prop.tau[i] > 0.f && in_bounds_open(log10((double)prop.tau[i]), pr.logtau_lo, pr.logtau_hi);
    else
        ok = ok && in_bounds_open(prop.tau[i], 0.0, 1.0);
    if (!ok) copy_particle(prop, i, cur, i);
    valid_out[i] = ok ? 1 : 0;
    lq[i] = lqf;
}

// Metropolis-Hastings test of the Langevin proposal at gamma_t:
//   ln u < gamma_t (l' - l) + log q(theta | theta') - log q(theta' | theta);
// on acceptance the particle and its gradient row take the proposal's.
__global__ void langevin_accept_kernel(PState cur, PState prop, float *gcur, const float *gprop,
                                       const int8_t *valid, const double *lq, const double *gamma,
                                       const double *lang_h, Params pr, int stage_arg, int sweep, int *lacc,
                                       int *lprop, const int *stage_dev) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pr.S * pr.N) return;
    const int stage = stage_dev ? *stage_dev : stage_arg;
    const int s = i / pr.N, jp = i - s * pr.N;
    atomicAdd(&lprop[s], 1);
    if (!valid[i]) return;
    const int kappa = cur.kappa[i], lam = cur.lam[i];
    const int d = 3 + 2 * kappa + 2 * lam;
    const double gm = gamma[s], h = lang_h[s];
    double lqr = 0.0;
    for (int j = 0; j < d; ++j) {
        const ThetaRef rc = theta_ref(cur, i, j, kappa, lam, pr);
        const ThetaRef rp = theta_ref(prop, i, j, kappa, lam, pr);
        const double sc = rc.scale;
        const double mean = theta_value(rp, pr) + 0.5 * h * h * sc * sc * gm * (double)gprop[(size_t)i * GD + rp.slot];
        const double zz = (theta_value(rc, pr) - mean) / (h * sc);
        lqr -= 0.5 * zz * zz;
    }
    uint32_t w[4];
    block_draws(w, stream_key(pr.seed, s), (uint32_t)jp, (uint32_t)kPurposeLangevinAccept, (uint32_t)stage,
                (uint32_t)sweep);
    const double u = u01_53(w[0], w[1]);
    if (log(u) < gm * (prop.ll[i] - cur.ll[i]) + lqr - lq[i]) {
        copy_particle(cur, i, prop, i);
        for (int q = 0; q < GD; ++q) gcur[(size_t)i * GD + q] = gprop[(size_t)i * GD + q];
        atomicAdd(&lacc[s], 1);
    }
}

// ------------------------------------------- adaptive within-model proposal
// Section 3.2: per (sounding, model) a Gaussian fitted to the model's
// particles, its eigen-decomposition, and a random walk along a uniformly
// chosen principal direction U_r with standard deviation a sqrt(Lambda_r).
__device__ bool pca_step(PState cur, PState prop, int i, int s, int kappa, int lam, const Params &pr, PcaView pv,
                         double a, double u_comp, double xi) {
    const int k = s * pr.M + kappa * (pr.lambda_max + 1) + lam;
    const int d = 3 + 2 * kappa + 2 * lam, DM = pr.DM;
    int r = (int)(u_comp * d);
    r = r > d - 1 ? d - 1 : r;
    const double *U = pv.U + (size_t)k * DM * DM;
    const double step = a * sqrt(pv.lam[(size_t)k * DM + r]) * xi;
    for (int j = 0; j < d; ++j) {
        const ThetaRef rc = theta_ref(cur, i, j, kappa, lam, pr);
        const ThetaRef rp = theta_ref(prop, i, j, kappa, lam, pr);
        const double v = theta_value(rc, pr) + step * U[(size_t)j * DM + r];
        *rp.x = (float)((rp.is_tau && pr.tau_log_prior) ? pow(10.0, v) : v);
    }
    bool ok = in_bounds_open(prop.phib[i], pr.phi_lo, pr.phi_hi) && in_bounds_open(prop.c[i], 0.0, 1.0);
    for (int q = 0; q < kappa; ++q) ok = ok && in_bounds_open(prop.phic[i * KS + q], pr.phi_lo, pr.phi_hi);
    for (int q = 0; q < lam; ++q) ok = ok && in_bounds_open(prop.mv[i * KS + q], 0.0, 1.0);
    ok = ok && ordered_open(prop.zc + (size_t)i * KS, kappa, pr.zmax) &&
         ordered_open(prop.zm + (size_t)i * KS, lam, pr.zmax);
    if (pr.tau_log_prior)
        ok = ok && prop.tau[i] > 0.f && in_bounds_open(log10((double)prop.tau[i]), pr.logtau_lo, pr.logtau_hi);
    else
        ok = ok && in_bounds_open(prop.tau[i], 0.0, 1.0);
    return ok;
}

// ZCA-coloured birth / death (Appendix F).  Birth k -> k+1 at depth
// u_d = zmax u1: the new value starts as a copy of the value of the layer it
// splits (0 for a chargeable layer above every chargeable interface), then
// every component but the new depth moves by u Z[i, j], u ~ N(0, 1), with
// Z = U Lambda^(1/2) U^T the ZCA root of model k+1's fit and i the new value's
// component; the factor multiplying (L'/L)^gamma is |J| / (width phi(u)),
// J = Z[i, i] - Z[i, h] (h the copied value's component, absent for the m = 0
// background).  Death: the interface floor(u1 n) of model k, u solved from
// the two values, the reciprocal factor.
__device__ inline void theta_store(const ThetaRef &r, const Params &pr, double v) {
    *r.x = (float)((r.is_tau && pr.tau_log_prior) ? pow(10.0, v) : v);
}

__device__ bool zca_move(PState cur, PState prop, int i, int s, bool birth, bool cond, const Params &pr, PcaView pv,
                         double u1, double xi, bool &ok, double &lf) {
    const int kappa = cur.kappa[i], lam = cur.lam[i];
    const int lp1 = pr.lambda_max + 1, DM = pr.DM;
    const double width = cond ? pr.phi_hi - pr.phi_lo : 1.0;
    const double log_phi0 = -0.91893853320467274;  // log(1 / sqrt(2 pi))
    if (birth) {
        const int n = cond ? kappa : lam;
        if (n >= (cond ? pr.kappa_max : pr.lambda_max)) return false;
        const int kk = s * pr.M + (cond ? (kappa + 1) * lp1 + lam : kappa * lp1 + lam + 1);
        if (!pv.ok[kk]) return false;
        float *zz = cond ? prop.zc : prop.zm;
        float *vv = cond ? prop.phic : prop.mv;
        const double z = __dmul_rn(pr.zmax, u1);
        int at = 0;
        while (at < n && (double)zz[i * KS + at] < z) ++at;
        const float src = cond ? (at == 0 ? cur.phib[i] : cur.phic[i * KS + at - 1]) : (at == 0 ? 0.f : cur.mv[i * KS + at - 1]);
        for (int q = n; q > at; --q) {
            zz[i * KS + q] = zz[i * KS + q - 1];
            vv[i * KS + q] = vv[i * KS + q - 1];
        }
        zz[i * KS + at] = (float)z;
        vv[i * KS + at] = src;
        const int k2 = cond ? kappa + 1 : kappa, l2 = cond ? lam : lam + 1;
        if (cond)
            prop.kappa[i] = k2;
        else
            prop.lam[i] = l2;
        const int d = 3 + 2 * k2 + 2 * l2;
        const int o_val = cond ? 1 : 1 + 2 * k2 + l2, o_dep = cond ? 1 + k2 : 1 + 2 * k2;
        const int j_new = o_val + at, j_z = o_dep + at, h = cond ? (at == 0 ? 0 : o_val + at - 1) : (at == 0 ? -1 : o_val + at - 1);
        const double *Zk = pv.Z + (size_t)kk * DM * DM + (size_t)j_new * DM;  // row j_new of the ZCA root
        double th[3 + 4 * AEM_SMC_SLOTS];
        // the new value's base is the copied value (exact in float), then the shift
        for (int jj = 0; jj < d; ++jj) th[jj] = theta_value(theta_ref(prop, i, jj, k2, l2, pr), pr);
        for (int jj = 0; jj < d; ++jj)
            if (jj != j_z) th[jj] += Zk[jj] * xi;
        for (int jj = 0; jj < d; ++jj) theta_store(theta_ref(prop, i, jj, k2, l2, pr), pr, th[jj]);
        const double jac = Zk[j_new] - (h >= 0 ? Zk[h] : 0.0);
        lf = log(fabs(jac)) - log(width) - (log_phi0 - 0.5 * xi * xi);
    } else {
        const int n = cond ? kappa : lam;
        if (n == 0) return false;
        const int kk = s * pr.M + kappa * lp1 + lam;
        if (!pv.ok[kk]) return false;
        int at = (int)(u1 * n);
        at = at > n - 1 ? n - 1 : at;
        const int d = 3 + 2 * kappa + 2 * lam;
        const int o_val = cond ? 1 : 1 + 2 * kappa + lam, o_dep = cond ? 1 + kappa : 1 + 2 * kappa;
        const int j_new = o_val + at, j_z = o_dep + at, h = cond ? (at == 0 ? 0 : o_val + at - 1) : (at == 0 ? -1 : o_val + at - 1);
        const double *Zk = pv.Z + (size_t)kk * DM * DM + (size_t)j_new * DM;
        double th[3 + 4 * AEM_SMC_SLOTS];
        for (int jj = 0; jj < d; ++jj) th[jj] = theta_value(theta_ref(cur, i, jj, kappa, lam, pr), pr);
        const double jac = Zk[j_new] - (h >= 0 ? Zk[h] : 0.0);
        const double u = (th[j_new] - (h >= 0 ? th[h] : 0.0)) / jac;
        for (int jj = 0; jj < d; ++jj)
            if (jj != j_z && jj != j_new) th[jj] -= Zk[jj] * u;
        // drop the two components, then the interface from the profile
        int w = 0;
        for (int jj = 0; jj < d; ++jj)
            if (jj != j_z && jj != j_new) th[w++] = th[jj];
        float *zz = cond ? prop.zc : prop.zm;
        float *vv = cond ? prop.phic : prop.mv;
        for (int q = at; q < n - 1; ++q) {
            zz[i * KS + q] = zz[i * KS + q + 1];
            vv[i * KS + q] = vv[i * KS + q + 1];
        }
        zz[i * KS + n - 1] = 0.f;
        vv[i * KS + n - 1] = 0.f;
        const int k2 = cond ? kappa - 1 : kappa, l2 = cond ? lam : lam - 1;
        if (cond)
            prop.kappa[i] = k2;
        else
            prop.lam[i] = l2;
        for (int jj = 0; jj < w; ++jj) theta_store(theta_ref(prop, i, jj, k2, l2, pr), pr, th[jj]);
        lf = log(width) + (log_phi0 - 0.5 * u * u) - log(fabs(jac));
    }
    const int k2 = prop.kappa[i], l2 = prop.lam[i];
    ok = in_bounds_open(prop.phib[i], pr.phi_lo, pr.phi_hi) && in_bounds_open(prop.c[i], 0.0, 1.0);
    for (int q = 0; q < k2; ++q) ok = ok && in_bounds_open(prop.phic[i * KS + q], pr.phi_lo, pr.phi_hi);
    for (int q = 0; q < l2; ++q) ok = ok && in_bounds_open(prop.mv[i * KS + q], 0.0, 1.0);
    ok = ok && ordered_open(prop.zc + (size_t)i * KS, k2, pr.zmax) && ordered_open(prop.zm + (size_t)i * KS, l2, pr.zmax);
    if (pr.tau_log_prior)
        ok = ok && prop.tau[i] > 0.f && in_bounds_open(log10((double)prop.tau[i]), pr.logtau_lo, pr.logtau_hi);
    else
        ok = ok && in_bounds_open(prop.tau[i], 0.0, 1.0);
    ok = ok && isfinite(lf);
    return true;
}

constexpr int kFitThreads = 128;
constexpr int kJacobiSweeps = 30;
constexpr int kMaxPairs = (AEM_SMC_GRAD_DIM + 1) / 2;  // rotations per round of the parallel ordering

// Fixed-order CTA reduction over kFitThreads threads (sum or maximum).
__device__ inline double block_reduce_128(double v, double *red, bool take_max) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            red[threadIdx.x] = take_max ? fmax(red[threadIdx.x], red[threadIdx.x + w]) : red[threadIdx.x] + red[threadIdx.x + w];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// Cyclic Jacobi rotations on the symmetric d x d matrix A (row stride DM) in
// shared memory, accumulating the rotations in V, by the whole CTA: each
// round of a sweep rotates n / 2 disjoint (p, q) pairs at once (the
// round-robin ordering of the indices, n = d rounded up to even; an index d
// pairs with nothing), as A <- A J, A <- J^T A, then the rotated 2 x 2 blocks
// take their exact values (A_pp - t A_pq, A_qq + t A_pq, 0) and the lower
// triangle is copied from the upper one.  Each rotation zeroes A_pq with
// t = tan(phi) the smaller root of t^2 + 2 t th - 1 = 0, th = (A_qq - A_pp) /
// (2 A_pq).  On return A's diagonal holds the eigenvalues and V's columns the
// eigenvectors.  At most kJacobiSweeps sweeps; stops when the off-diagonal
// mass falls below 1e-30 of the diagonal's.
__device__ void jacobi_eigen_block(double *A, double *V, int d, int DM, double *red) {
    __shared__ double rc[kMaxPairs], rs[kMaxPairs], rt[kMaxPairs], ra[kMaxPairs], rpp[kMaxPairs], rqq[kMaxPairs];
    __shared__ int rp[kMaxPairs], rq[kMaxPairs];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int n = d + (d & 1), half = n / 2;
    const double scale2 = block_reduce_128(tid < d ? A[tid * DM + tid] * A[tid * DM + tid] : 0.0, red, false);
    for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
        double o = 0.0;
        for (int e = tid; e < d * d; e += nt) {
            const int j = e / d, l = e - j * d;
            if (l > j) o += A[j * DM + l] * A[j * DM + l];
        }
        if (block_reduce_128(o, red, false) <= 1e-30 * scale2) break;
        for (int round = 0; round < n - 1; ++round) {
            if (tid < half) {
                const int a = tid == 0 ? n - 1 : (round + tid) % (n - 1);
                const int b = tid == 0 ? round : (round - tid + (n - 1)) % (n - 1);
                const int p = a < b ? a : b, q = a < b ? b : a;
                double c = 1.0, sn = 0.0, t = 0.0, apq = 0.0;
                if (q < d) {
                    apq = A[p * DM + q];
                    if (apq != 0.0) {
                        const double th = (A[q * DM + q] - A[p * DM + p]) / (2.0 * apq);
                        t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        sn = t * c;
                    }
                    rpp[tid] = A[p * DM + p];
                    rqq[tid] = A[q * DM + q];
                }
                rp[tid] = p;
                rq[tid] = apq != 0.0 ? q : d;  // d: nothing to rotate
                rc[tid] = c;
                rs[tid] = sn;
                rt[tid] = t;
                ra[tid] = apq;
            }
            __syncthreads();
            for (int e = tid; e < d * half; e += nt) {  // columns p, q of A and V
                const int i = e / d, r = e - i * d, p = rp[i], q = rq[i];
                if (q >= d) continue;
                const double c = rc[i], sn = rs[i];
                const double arp = A[r * DM + p], arq = A[r * DM + q];
                A[r * DM + p] = c * arp - sn * arq;
                A[r * DM + q] = sn * arp + c * arq;
                const double vrp = V[r * DM + p], vrq = V[r * DM + q];
                V[r * DM + p] = c * vrp - sn * vrq;
                V[r * DM + q] = sn * vrp + c * vrq;
            }
            __syncthreads();
            for (int e = tid; e < d * half; e += nt) {  // rows p, q of A
                const int i = e / d, r = e - i * d, p = rp[i], q = rq[i];
                if (q >= d) continue;
                const double c = rc[i], sn = rs[i];
                const double apr = A[p * DM + r], aqr = A[q * DM + r];
                A[p * DM + r] = c * apr - sn * aqr;
                A[q * DM + r] = sn * apr + c * aqr;
            }
            __syncthreads();
            if (tid < half && rq[tid] < d) {
                const int p = rp[tid], q = rq[tid];
                A[p * DM + p] = rpp[tid] - rt[tid] * ra[tid];
                A[q * DM + q] = rqq[tid] + rt[tid] * ra[tid];
                A[p * DM + q] = 0.0;
            }
            __syncthreads();
            for (int e = tid; e < d * d; e += nt) {
                const int j = e / d, l = e - j * d;
                if (l < j) A[j * DM + l] = A[l * DM + j];
            }
            __syncthreads();
        }
    }
}

// The weighted Gaussian fit of one model in one CTA, shared by the plain and
// the recycled fit.  cand(c) gives candidate c's particle index and weight
// (weight 0: not used) for c < C.  Candidates are taken kFitThreads at a
// time into shared memory (theta rows X, weights W); the mean and then the
// covariance of the deviations accumulate per entry in candidate order (the
// serial order of the definition), each entry on its own thread.  Adds
// (ridge * step_j)^2 on the diagonal, then A = U Lambda U^T by
// jacobi_eigen_block; writes mu, U, Lambda (clipped at 0) and ok = 1.
template <class Cand>
__device__ void fit_model_block(const PState &ps, Cand cand, int C, double sw, int kappa, int lam, const Params &pr,
                                double ridge, double *sm, double *red, int b, double *mu_out, double *U_out,
                                double *lam_out, int *ok_out, double *Z_out) {
    const int DM = pr.DM, tid = threadIdx.x, d = 3 + 2 * kappa + 2 * lam;
    double *A = sm, *V = A + DM * DM, *mu = V + DM * DM, *X = mu + DM, *W = X + (size_t)kFitThreads * DM;
    constexpr int kMaxEntries = (AEM_SMC_GRAD_DIM * (AEM_SMC_GRAD_DIM + 1) / 2 + kFitThreads - 1) / kFitThreads;
    const int ne = d * (d + 1) / 2;
    int ej[kMaxEntries], el[kMaxEntries];  // this thread's entries of the upper triangle, row-major
#pragma unroll
    for (int u = 0; u < kMaxEntries; ++u) {
        int j = 0, rem = tid + u * kFitThreads;
        while (j < d && rem >= d - j) {
            rem -= d - j;
            ++j;
        }
        ej[u] = j;
        el[u] = j + rem;
    }
    // pass 1: the weighted mean; pass 2: the weighted covariance of the deviations
    for (int pass = 0; pass < 2; ++pass) {
        double acc[kMaxEntries];
#pragma unroll
        for (int u = 0; u < kMaxEntries; ++u) acc[u] = 0.0;
        for (int base = 0; base < C; base += kFitThreads) {
            const int c = base + tid;
            int i = -1;
            double w = 0.0;
            if (c < C) cand(c, i, w);
            W[tid] = w;
            for (int j = 0; j < d; ++j) {
                double x = 0.0;
                if (w != 0.0) {
                    x = theta_value(theta_ref(ps, i, j, kappa, lam, pr), pr);
                    if (pass == 1) x -= mu[j];
                }
                X[tid * DM + j] = x;
            }
            __syncthreads();
            const int nc = C - base < kFitThreads ? C - base : kFitThreads;
            if (pass == 0) {
                if (tid < d)
                    for (int q = 0; q < nc; ++q) acc[0] += W[q] * X[q * DM + tid];
            } else {
#pragma unroll
                for (int u = 0; u < kMaxEntries; ++u) {
                    const int e = tid + u * kFitThreads;
                    if (e < ne) {
                        const int j = ej[u], l = el[u];
                        for (int q = 0; q < nc; ++q) acc[u] += W[q] * X[q * DM + j] * X[q * DM + l];
                    }
                }
            }
            __syncthreads();
        }
        if (pass == 0) {
            if (tid < d) mu[tid] = acc[0] / sw;
        } else {
#pragma unroll
            for (int u = 0; u < kMaxEntries; ++u) {
                const int e = tid + u * kFitThreads;
                if (e < ne) {
                    const int j = ej[u], l = el[u];
                    double cv = acc[u] / sw;
                    if (j == l) {
                        const double sj = ridge * theta_ref(ps, 0, j, kappa, lam, pr).scale;
                        cv += sj * sj;
                    }
                    A[j * DM + l] = cv;
                    A[l * DM + j] = cv;
                }
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < d * d; e += kFitThreads) {
        const int j = e / d, l = e - (e / d) * d;
        V[j * DM + l] = j == l ? 1.0 : 0.0;
    }
    __syncthreads();
    jacobi_eigen_block(A, V, d, DM, red);
    for (int e = tid; e < d * d; e += kFitThreads) {
        const int j = e / d, l = e - (e / d) * d;
        U_out[(size_t)b * DM * DM + (size_t)j * DM + l] = V[j * DM + l];
    }
    for (int j = tid; j < d; j += kFitThreads) {
        mu_out[(size_t)b * DM + j] = mu[j];
        const double lj = A[j * DM + j];
        lam_out[(size_t)b * DM + j] = lj > 0.0 ? lj : 0.0;
    }
    // the ZCA root Z = U Lambda^(1/2) U^T (Lambda clipped at 0), summed over r in order
    for (int e = tid; e < d * d; e += kFitThreads) {
        const int j = e / d, l = e - (e / d) * d;
        double z = 0.0;
        for (int r = 0; r < d; ++r) {
            const double lr = A[r * DM + r];
            z += V[j * DM + r] * sqrt(lr > 0.0 ? lr : 0.0) * V[l * DM + r];
        }
        Z_out[(size_t)b * DM * DM + (size_t)j * DM + l] = z;
    }
    if (tid == 0) ok_out[b] = 1;
}

// Shared memory of the fit kernels, in doubles: A, V [DM][DM], mu [DM], the
// candidate tile X [kFitThreads][DM] and its weights [kFitThreads].
size_t fit_smem_bytes(int DM) {
    return sizeof(double) * (2 * (size_t)DM * DM + DM + (size_t)kFitThreads * DM + kFitThreads);
}

// One CTA per (sounding, model): mean and (biased) covariance of theta over
// the model's particles in FP64 with fixed-order sums, plus
// (ridge * step_j)^2 on the diagonal, then Sigma = U Lambda U^T by parallel
// Jacobi rotations in shared memory.  Models with fewer than two particles get
// ok = 0 and their scale reset to 1.
__global__ void __launch_bounds__(kFitThreads) pca_fit_kernel(PState st, const int *perm, const int *off,
                                                              const int *counts, Params pr, double ridge,
                                                              double *mu_out, double *U_out, double *lam_out,
                                                              int *ok_out, double *a_out, double *Z_out) {
    extern __shared__ double sm_fit[];
    __shared__ double red[kFitThreads];
    const int b = blockIdx.x, s = b / pr.M, k = b - (b / pr.M) * pr.M;
    const int kappa = k / (pr.lambda_max + 1), lam = k - kappa * (pr.lambda_max + 1);
    const int n = counts[b];
    const int *idx = perm + (size_t)s * pr.N + off[s * (pr.M + 1) + k];
    if (n < 2) {
        if (threadIdx.x == 0) {
            ok_out[b] = 0;
            a_out[b] = 1.0;
        }
        return;
    }
    auto cand = [&](int c, int &i, double &w) {
        i = idx[c];
        w = 1.0;
    };
    fit_model_block(st, cand, n, (double)n, kappa, lam, pr, ridge, sm_fit, red, b, mu_out, U_out, lam_out, ok_out,
                    Z_out);
}

// ----------------------------------------------------- particle recycling
// Section 3.2 ("Overcoming particle impoverishment"): the fit of each model's
// proposal uses the particles of the last H stages, each weighted by the
// deterministic-mixture weight
//   log nu = gamma_t l - log( (1/(t+1)) sum_{l=0}^{t} exp(gamma_l l - log Z_{l,k}) )
// (the prior cancels; the printed 1/t over t + 1 terms read as 1/(t+1)).
constexpr int kMaxRecycleStages = 1024;  // stages whose gamma and log Z are kept

// With stage_dev the stage t comes from the device counter and n_used =
// min(t + 1, H) (the grid then covers H x P).
__global__ void recycle_weight_kernel(PState hist, int P, int n_used, int N, int M, int lp1, int t,
                                      const double *gamma_hist, const double *logz_hist, double *lognu, int H,
                                      const int *stage_dev) {
    if (stage_dev) {
        t = *stage_dev;
        n_used = t + 1 < H ? t + 1 : H;
    }
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n_used * P) return;
    const int i = (int)(idx % (size_t)P), s = i / N;
    const int k = hist.kappa[idx] * lp1 + hist.lam[idx];
    const double l = hist.ll[idx];
    const double *g = gamma_hist + (size_t)s * kMaxRecycleStages;
    const double *lz = logz_hist + (size_t)s * kMaxRecycleStages * M + k;
    double m = -INFINITY;
    for (int q = 0; q <= t; ++q) m = fmax(m, g[q] * l - lz[(size_t)q * M]);
    double acc = 0.0;
    for (int q = 0; q <= t; ++q) acc += exp(g[q] * l - lz[(size_t)q * M] - m);
    lognu[idx] = g[t] * l - (m + log(acc) - log((double)(t + 1)));
}

// One CTA (128 threads) per (sounding, model) with at least two current
// particles: normalised recycling weights over the model's stored particles
// (written to wbuf), the weighted mean and covariance of theta in FP64 with
// fixed-order sums, the ridge, then the same Jacobi decomposition as the
// plain fit.
__global__ void __launch_bounds__(kFitThreads) pca_fit_recycle_kernel(PState hist, const double *lognu, double *wbuf,
                                                                      int n_used, int P, const int *counts, Params pr,
                                                                      double ridge, double *mu_out, double *U_out,
                                                                      double *lam_out, int *ok_out, double *a_out,
                                                                      int H, const int *stage_dev, double *Z_out) {
    if (stage_dev) n_used = *stage_dev + 1 < H ? *stage_dev + 1 : H;
    extern __shared__ double sm_fit[];
    __shared__ double red[kFitThreads];
    const int b = blockIdx.x, s = b / pr.M, k = b - (b / pr.M) * pr.M;
    const int lp1 = pr.lambda_max + 1, kappa = k / lp1, lam = k - kappa * lp1;
    const int tid = threadIdx.x;
    if (counts[b] < 2) {
        if (tid == 0) {
            ok_out[b] = 0;
            a_out[b] = 1.0;
        }
        return;
    }
    const int C = n_used * pr.N;  // candidates: every stored particle of this sounding
    auto cand = [&](int c) -> size_t { return (size_t)(c / pr.N) * P + (size_t)s * pr.N + (c % pr.N); };
    auto member = [&](size_t idx) { return hist.kappa[idx] == kappa && hist.lam[idx] == lam; };
    double m = -INFINITY;
    for (int c = tid; c < C; c += blockDim.x) {
        const size_t idx = cand(c);
        if (member(idx)) m = fmax(m, lognu[idx]);
    }
    m = block_reduce_128(m, red, true);
    double sw = 0.0;
    for (int c = tid; c < C; c += blockDim.x) {
        const size_t idx = cand(c);
        if (member(idx)) {
            const double w = exp(lognu[idx] - m);
            wbuf[idx] = w;
            sw += w;
        }
    }
    sw = block_reduce_128(sw, red, false);  // also orders the wbuf writes before the reads below
    auto wcand = [&](int c, int &i, double &w) {
        const size_t idx = cand(c);
        i = (int)idx;
        w = member(idx) ? wbuf[idx] : 0.0;
    };
    fit_model_block(hist, wcand, C, sw, kappa, lam, pr, ridge, sm_fit, red, b, mu_out, U_out, lam_out, ok_out,
                    Z_out);
}

// Stores the current particles as history slot `slot` and this stage's gamma
// and log Z (per sounding) at row t.
__global__ void record_slot_kernel(PState hist, PState cur, int P, int slot, int H, const int *stage_dev) {
    if (stage_dev) slot = *stage_dev % H;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P) copy_particle(hist, slot * P + i, cur, i);
}

__global__ void record_stage_kernel(const double *gamma, const double *logz, int S, int M, int t, double *gamma_hist,
                                    double *logz_hist, const int *stage_dev) {
    if (stage_dev) t = *stage_dev;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S || t >= kMaxRecycleStages) return;
    gamma_hist[(size_t)s * kMaxRecycleStages + t] = gamma[s];
    for (int k = 0; k < M; ++k)
        logz_hist[((size_t)s * kMaxRecycleStages + t) * M + k] = logz[(size_t)s * M + k];
}

// Trial proposals of the scale bisection: every particle of a fitted model
// steps along its trial direction at scale exp((lo + hi) / 2) of its model;
// the trial draws (purpose kPurposePcaTrial, sweep 0) are the same at every
// bisection step.
__global__ void pca_trial_kernel(PState cur, PState prop, int8_t *valid_out, Params pr, PcaView pv,
                                 const double *lo, const double *hi, int stage_arg, const int *stage_dev) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pr.S * pr.N) return;
    const int stage = stage_dev ? *stage_dev : stage_arg;
    const int s = i / pr.N, j = i - s * pr.N;
    const int kappa = cur.kappa[i], lam = cur.lam[i];
    const int k = s * pr.M + kappa * (pr.lambda_max + 1) + lam;
    copy_particle(prop, i, cur, i);
    if (!pv.ok[k]) {
        valid_out[i] = 0;
        return;
    }
    uint32_t w[4];
    block_draws(w, stream_key(pr.seed, s), (uint32_t)j, (uint32_t)kPurposePcaTrial, (uint32_t)stage, 0u);
    const double a = exp(0.5 * (lo[k] + hi[k]));
    const bool ok = pca_step(cur, prop, i, s, kappa, lam, pr, pv, a, u01(w[0]), gauss(w[1], w[2]));
    if (!ok) copy_particle(prop, i, cur, i);
    valid_out[i] = ok ? 1 : 0;
}

// One CTA per (sounding, model): mean over the model's particles of
// min(1, (L'/L)^gamma) (0 for trials outside the support), in FP64 with a
// fixed-order reduction; moves the bracket towards the target acceptance.
__global__ void __launch_bounds__(128) pca_stat_kernel(const double *ll_cur, const double *ll_prop,
                                                       const int8_t *valid, const int *perm, const int *off,
                                                       const int *counts, const int *ok, const double *gamma,
                                                       Params pr, double target, double *lo, double *hi) {
    __shared__ double red[128];
    const int b = blockIdx.x, s = b / pr.M, k = b - (b / pr.M) * pr.M;
    if (!ok[b]) return;
    const int n = counts[b];
    const int *idx = perm + (size_t)s * pr.N + off[s * (pr.M + 1) + k];
    double acc = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int i = idx[q];
        if (valid[i]) {
            const double dl = gamma[s] * (ll_prop[i] - ll_cur[i]);
            acc += dl >= 0.0 ? 1.0 : exp(dl);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mid = 0.5 * (lo[b] + hi[b]);
        if (red[0] / n > target)
            lo[b] = mid;
        else
            hi[b] = mid;
    }
}

__global__ void pca_bracket_kernel(const int *ok, const double *a, int n, double span, double *lo, double *hi) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const double la = log(a[b]);
    lo[b] = la - span;
    hi[b] = la + span;
}

__global__ void pca_finish_kernel(const int *ok, const double *lo, const double *hi, int n, double *a) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n && ok[b]) a[b] = exp(0.5 * (lo[b] + hi[b]));
}

// Between stages: h <- h exp(2 (rate - 0.574)) per sounding, clamped to
// [1e-6, 10] (0.574: the optimal MALA acceptance of Roberts & Rosenthal 1998).
__global__ void langevin_adapt_kernel(const int *lacc, const int *lprop, int S, double *lang_h) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const double rate = lprop[s] > 0 ? (double)lacc[s] / lprop[s] : 0.574;
    const double h = lang_h[s] * exp(2.0 * (rate - 0.574));
    lang_h[s] = h < 1e-6 ? 1e-6 : (h > 10.0 ? 10.0 : h);
}

// Posterior predictive summaries (Section 4.1): one CTA per (sounding, gate)
// over the sounding's equally weighted particles, FP64 with fixed-order
// reductions: mean, variance of the predictive mixture (noise variance plus
// the spread of the predictions), and the data standardised to it.
__global__ void __launch_bounds__(256) ppd_kernel(const float *gates, int N, int G, const double *y_obs,
                                                  const double *eps_an, double eps_mn, double *mean, double *var,
                                                  double *z) {
    const int s = blockIdx.x / G, g = blockIdx.x - (blockIdx.x / G) * G;
    __shared__ double red[256];
    const float *col = gates + (size_t)s * N * G + g;
    double a = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) a += (double)col[(size_t)i * G];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double mu = red[0] / N;
    __syncthreads();
    const double ea = eps_an[g];
    double b = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double yh = (double)col[(size_t)i * G];
        const double d = yh - mu;
        b += ea * ea + (eps_mn * yh) * (eps_mn * yh) + d * d;
    }
    red[threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double v = red[0] / N;
        mean[(size_t)s * G + g] = mu;
        var[(size_t)s * G + g] = v;
        z[(size_t)s * G + g] = (y_obs[(size_t)s * G + g] - mu) / sqrt(v);
    }
}

// Graph-captured stages: the stage counter advances on the device; the loop
// condition (another stage needed) is set on the device from the new gammas.
__global__ void stage_inc_kernel(int *d_stage) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_stage += 1;
}

__global__ void stage_cond_kernel(const double *gamma, int S, const int *d_stage, int stop_stage, const int *status,
                                  cudaGraphConditionalHandle h) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    bool all = true;
    for (int s = 0; s < S; ++s) all = all && gamma[s] >= 1.0;
    // a failed reweight step (status word set) ends the loop after this stage
    cudaGraphSetConditional(h, (!all && *d_stage < stop_stage && *status == 0) ? 1u : 0u);
}

// App. B's sweep count on the device, from the acceptance counts of the
// previous stage's sweeps (the first sounding's, as the host path takes them):
// R = ceil(log c / log(1 - p_min)) clamped to 1..r_max, r_max without counts.
__global__ void sweep_count_kernel(const int *acc, const int *nprop, const int *have_prev, double c_mut, int r_max,
                                   int *sweeps) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    if (!*have_prev) {
        *sweeps = r_max;
        return;
    }
    double pmin = 1.0;
    for (int m = 0; m < kMoves; ++m) {
        const double r = nprop[m] > 0 ? (double)acc[m] / nprop[m] : 1.0;
        pmin = r < pmin ? r : pmin;
    }
    int R;
    if (pmin <= 0.0)
        R = r_max;
    else if (pmin >= 1.0)
        R = 1;
    else
        R = (int)ceil(log(c_mut) / log(1.0 - pmin));
    *sweeps = R < 1 ? 1 : (R > r_max ? r_max : R);
}

__global__ void sweep_gate_kernel(const int *sweeps, int sweep, int *gate) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *gate = sweep < *sweeps ? 1 : 0;
}

__global__ void set_flag_kernel(int *flag, int v) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *flag = v;
}

__global__ void copy_state_kernel(PState dst, PState src, int P) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P) copy_particle(dst, i, src, i);
}

__global__ void philox_kernel(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
    philox(c, Key{k0, k1});
    for (int q = 0; q < 4; ++q) out[4 * i + q] = c[q];
}

// Model ids from a plain int array (the standalone reweight / resample entry
// points take the model of each particle directly).
// Model ids of the standalone a7 / a8 entries.  An id outside [0, n_models)
// takes no part: it is given a group key no model has (255 > AEM_SMC_MAX_MODELS),
// and its ancestor (resample) or weight (reweight) output is set to -1 / 0.
__global__ void split_model_kernel(const int *model, int n, int n_models, int *kappa, int *lam, int *anc_out,
                                   double *w_out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int id = model[i];
    const bool ok = id >= 0 && id < n_models;
    kappa[i] = ok ? id : 255;
    lam[i] = 0;
    if (!ok && anc_out) anc_out[i] = -1;
    if (!ok && w_out) w_out[i] = 0.0;
}

// perm lists the grouped particles only (off[M] of them, fewer than n when
// some ids were out of range)
__global__ void scatter_kernel(const double *Wg, const int *perm, const int *off, int M, double *W) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < off[M]) W[perm[i]] = Wg[i];
}

__global__ void gather_weights_kernel(const double *W, const int *perm, const int *off, int M, double *Wg) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < off[M]) Wg[i] = W[perm[i]];
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace aem

// ========================================================================
// Host side
// ========================================================================
using namespace aem;

struct smc_state {
    const aem_system *sys = nullptr;
    smc_desc d{};
    Params pr{};
    int S = 0, N = 0, P = 0, M = 0, LMS = 0;
    cudaStream_t stream = nullptr;
    PState cur{}, alt{}, prop{};
    std::vector<void *> allocs;
    int8_t *move = nullptr, *valid = nullptr;
    double *lf = nullptr;  // per-proposal log factor of the ZCA-coloured birth / death (0 otherwise)
    int *anc = nullptr, *perm = nullptr, *off = nullptr, *counts = nullptr, *acc = nullptr, *nprop = nullptr,
        *done = nullptr;
    double *Wg = nullptr, *gamma = nullptr, *logz = nullptr, *dgamma = nullptr;
    unsigned long long *C = nullptr;
    int8_t *m_nl = nullptr;
    float *m_logsig = nullptr, *m_logh = nullptr, *m_m = nullptr, *m_logtau = nullptr, *m_c = nullptr;
    double *y = nullptr, *eps_an = nullptr;
    double eps_mn = 0.0;
    // Langevin: merged-layer gradient, particle-space gradients of the current
    // and proposed particles, log q(theta' | theta), per-sounding counts.
    float *mgrad = nullptr, *gcur = nullptr, *gprop = nullptr;
    unsigned char *grad_work = nullptr;  // the adjoint's claim counters and gates (grad_work_bytes)
    float *ppd_gates = nullptr;  // [P][G], allocated on the first smc_ppd call
    // adaptive within-model proposal, per (sounding, model): mean [DM], U
    // [DM][DM] (column r = direction r), Lambda [DM], ok, scale a, bracket
    double *pca_mu = nullptr, *pca_U = nullptr, *pca_lam = nullptr, *pca_a = nullptr, *pca_lo = nullptr,
           *pca_hi = nullptr, *pca_Z = nullptr;
    int *pca_ok = nullptr;
    // particle recycling: the last H post-resample populations ([H * P] in
    // every particle array, slot = stage mod H), their log nu and weights, and
    // every stage's gamma [S][1024] and log Z [S][1024][M]
    PState hist{};
    double *hist_lognu = nullptr, *hist_w = nullptr, *gamma_hist = nullptr, *logz_hist = nullptr;
    double *ppd_out = nullptr;   // [3][S][G]
    double *lq = nullptr, *lang_h = nullptr;
    int *lacc = nullptr, *lprop = nullptr;
    bool gcur_valid = false;
    int stage = 0;
    // device-side stage counter (graph-captured runs) and the forward kernel's
    // model-claim counter, owned by the sampler so its launches allocate nothing
    int *d_stage = nullptr, *fwd_counter = nullptr;
    // graph form with App. B's sweep count: R_t, this sweep's gate, whether a
    // previous stage's acceptance counts exist
    int *d_sweeps = nullptr, *d_gate = nullptr, *d_have_prev = nullptr;
    // failure reporting: the sampler's status word (AEM_ERR_NONFINITE /
    // AEM_ERR_NO_BRACKET recorded by the reweight step, read and cleared by
    // smc_status) and the per-sounding count of non-finite log-likelihoods
    // mapped to -inf since smc_init
    int *d_status = nullptr, *nonfinite = nullptr;
    // model odds formed on the device in FP64: post [S][M], log BFIPD [S]
    double *d_post = nullptr, *d_lbf = nullptr;
    // merged models in FP64 for the plain double-precision forward model
    // (desc.precision = AEM_SMC_FP64)
    double *m64_logsig = nullptr, *m64_logh = nullptr, *m64_m = nullptr, *m64_logtau = nullptr, *m64_c = nullptr;
    std::vector<int> acc_prev, nprop_prev;
    bool have_prev = false;
};

namespace {

template <class T>
int dalloc(smc_state *st, T **p, size_t n) {
    void *q = nullptr;
    AEM_CUDA_TRY(cudaMalloc(&q, n * sizeof(T) + 16));
    st->allocs.push_back(q);
    *p = (T *)q;
    return AEM_OK;
}

int alloc_pstate(smc_state *st, PState *ps, size_t count = 0) {
    const size_t P = count ? count : (size_t)st->P;
    int rc;
    if ((rc = dalloc(st, &ps->kappa, P)) || (rc = dalloc(st, &ps->lam, P)) || (rc = dalloc(st, &ps->phib, P)) ||
        (rc = dalloc(st, &ps->tau, P)) || (rc = dalloc(st, &ps->c, P)) || (rc = dalloc(st, &ps->zc, P * KS)) ||
        (rc = dalloc(st, &ps->phic, P * KS)) || (rc = dalloc(st, &ps->zm, P * KS)) ||
        (rc = dalloc(st, &ps->mv, P * KS)) || (rc = dalloc(st, &ps->ll, P)))
        return rc;
    return AEM_OK;
}

int sanitize(smc_state *st, double *ll, const int *active = nullptr) {
    sanitize_ll_kernel<<<blocks_for(st->P, 256), 256, 0, st->stream>>>(ll, st->P, st->N, st->nonfinite, active);
    AEM_CUDA_TRY(cudaGetLastError());
    return AEM_OK;
}

// Merge and forward model + log-likelihood of a particle set, in FP32 or, with
// desc.precision = AEM_SMC_FP64, in the plain FP64 form; non-finite results
// become -inf.  valid (proposals): particles flagged 0 made no move (their
// proposal is a copy of the current particle, which the accept step leaves
// as it is), so the forward model skips them.
int run_loglik(smc_state *st, PState ps, const int *active = nullptr, const int8_t *valid = nullptr) {
    int rc;
    if (st->d.precision == AEM_SMC_FP64) {
        merge_kernel<double><<<blocks_for(st->P, 256), 256, 0, st->stream>>>(
            ps, st->P, st->LMS, st->m_nl, st->m64_logsig, st->m64_logh, st->m64_m, st->m64_logtau, st->m64_c);
        AEM_CUDA_TRY(cudaGetLastError());
        aem_models_f64 mm{st->P, st->LMS, st->m_nl, st->m64_logsig, st->m64_logh, st->m64_m, st->m64_logtau, st->m64_c};
        rc = loglik_f64_soundings(st->sys, &mm, st->y, st->N, st->eps_an, st->eps_mn, ps.ll, st->stream, active,
                                  valid);
    } else {
        merge_kernel<float><<<blocks_for(st->P, 256), 256, 0, st->stream>>>(
            ps, st->P, st->LMS, st->m_nl, st->m_logsig, st->m_logh, st->m_m, st->m_logtau, st->m_c);
        AEM_CUDA_TRY(cudaGetLastError());
        aem_models_f32 mm{st->P, st->LMS, st->m_nl, st->m_logsig, st->m_logh, st->m_m, st->m_logtau, st->m_c};
        rc = loglik_f32_soundings(st->sys, &mm, st->y, st->N, st->eps_an, st->eps_mn, ps.ll, st->stream,
                                  st->fwd_counter, active, valid);
    }
    if (rc) return rc;
    return sanitize(st, ps.ll, active);
}

// Log-likelihood and particle-space gradient of a particle set: merge, the
// adjoint kernel on the merged models, then the chain rule back to the
// particle's parameters.
// valid (proposals): particles flagged 0 are skipped, as in run_loglik.
int run_grad(smc_state *st, PState ps, float *pg, const int8_t *valid = nullptr) {
    merge_kernel<float><<<blocks_for(st->P, 256), 256, 0, st->stream>>>(ps, st->P, st->LMS, st->m_nl, st->m_logsig,
                                                                st->m_logh, st->m_m, st->m_logtau, st->m_c);
    AEM_CUDA_TRY(cudaGetLastError());
    aem_models_f32 mm{st->P, st->LMS, st->m_nl, st->m_logsig, st->m_logh, st->m_m, st->m_logtau, st->m_c};
    int rc = loglik_grad_f32_soundings(st->sys, &mm, st->y, st->N, st->eps_an, st->eps_mn, ps.ll, st->mgrad,
                                       st->stream, st->grad_work, valid);
    if (rc) return rc;
    if ((rc = sanitize(st, ps.ll))) return rc;
    pgrad_kernel<<<blocks_for(st->P, 128), 128, 0, st->stream>>>(ps, st->mgrad, st->P, st->LMS,
                                                                 st->d.tau_log_prior, pg);
    AEM_CUDA_TRY(cudaGetLastError());
    return AEM_OK;
}

int check_desc(const smc_desc *d) {
    if (!d) return fail(AEM_ERR_INVALID_ARG, "smc_create: desc is NULL");
    if (d->n_particles < 2 || d->n_particles > AEM_SMC_MAX_PARTICLES)
        return fail(AEM_ERR_INVALID_ARG, "smc_create: n_particles outside 2..AEM_SMC_MAX_PARTICLES");
    if (d->n_soundings < 1) return fail(AEM_ERR_INVALID_ARG, "smc_create: n_soundings < 1");
    if (d->kappa_max < 0 || d->lambda_max < 0 || d->kappa_max >= AEM_SMC_SLOTS || d->lambda_max >= AEM_SMC_SLOTS ||
        d->kappa_max + d->lambda_max + 1 > AEM_MAX_LAYERS)
        return fail(AEM_ERR_INVALID_ARG, "smc_create: kappa_max / lambda_max out of range");
    if ((d->kappa_max + 1) * (d->lambda_max + 1) > AEM_SMC_MAX_MODELS)
        return fail(AEM_ERR_INVALID_ARG, "smc_create: too many models");
    if (!(d->zmax > 0) || !(d->alpha > 0 && d->alpha < 1) || !(d->c_mut > 0 && d->c_mut < 1) || d->r_max < 1 ||
        !(d->phi_hi > d->phi_lo) || d->bisect_iters < 1 || d->bisect_iters > 200)
        return fail(AEM_ERR_INVALID_ARG, "smc_create: invalid zmax / alpha / c_mut / r_max / prior bounds");
    if (d->tau_log_prior && !(d->logtau_hi > d->logtau_lo))
        return fail(AEM_ERR_INVALID_ARG, "smc_create: invalid log10 tau bounds");
    if (d->adaptive && (!(d->pca_target > 0 && d->pca_target < 1) || d->pca_bisect_iters < 1 ||
                        d->pca_bisect_iters > 60 || !(d->pca_ridge >= 0)))
        return fail(AEM_ERR_INVALID_ARG, "smc_create: invalid pca_target / pca_bisect_iters / pca_ridge");
    if (!(d->zca >= 0.0 && d->zca <= 1.0) || (d->zca > 0.0 && !d->adaptive))
        return fail(AEM_ERR_INVALID_ARG, "smc_create: zca outside [0, 1], or set without adaptive");
    if (d->recycle_stages < 0 || d->recycle_stages > 32 || (d->recycle_stages > 0 && !d->adaptive))
        return fail(AEM_ERR_INVALID_ARG, "smc_create: recycle_stages outside 0..32, or set without adaptive");
    if (d->n_langevin < 0 || d->n_langevin > 1000 || !(d->langevin_h > 0))
        return fail(AEM_ERR_INVALID_ARG, "smc_create: n_langevin outside 0..1000 or langevin_h <= 0");
    if (d->precision != AEM_SMC_FP32 && d->precision != AEM_SMC_FP64)
        return fail(AEM_ERR_INVALID_ARG, "smc_create: precision is neither AEM_SMC_FP32 nor AEM_SMC_FP64");
    if (d->precision == AEM_SMC_FP64 && d->n_langevin > 0)
        return fail(AEM_ERR_UNSUPPORTED, "smc_create: the Langevin moves use the FP32 adjoint; not with AEM_SMC_FP64");
    return AEM_OK;
}

}  // namespace

extern "C" int smc_desc_defaults(smc_desc *d) {
    if (!d) return fail(AEM_ERR_INVALID_ARG, "smc_desc_defaults: NULL");
    *d = smc_desc{};
    d->n_particles = 256;
    d->n_soundings = 1;
    d->kappa_max = 3;
    d->lambda_max = 4;
    d->zmax = 500.0;
    d->alpha = 0.5;
    d->c_mut = 0.01;
    d->r_max = 10;
    d->step_phi = 0.2;
    d->step_m = 0.05;
    d->step_tau = 0.05;
    d->step_c = 0.05;
    d->step_z = 10.0;
    d->phi_lo = -4.0;
    d->phi_hi = 2.0;
    d->tau_log_prior = 0;
    d->logtau_lo = -6.0;
    d->logtau_hi = -1.0;
    d->seed = 0;
    d->bisect_iters = 60;
    d->n_langevin = 0;
    d->langevin_h = 0.1;
    d->langevin_adapt = 1;
    d->adaptive = 0;
    d->pca_target = 0.44;
    d->pca_bisect_iters = 6;
    d->pca_ridge = 0.01;
    d->recycle_stages = 0;
    d->zca = 0.0;
    d->precision = AEM_SMC_FP32;
    return AEM_OK;
}

extern "C" int smc_create(const aem_system *sys, const smc_desc *desc, const double *y_obs, const double *eps_an,
                          double eps_mn, void *stream, smc_state **out) {
    if (!out) return fail(AEM_ERR_INVALID_ARG, "smc_create: out is NULL");
    *out = nullptr;
    if (!sys || !y_obs || !eps_an) return fail(AEM_ERR_INVALID_ARG, "smc_create: NULL system or data");
    int rc = check_desc(desc);
    if (rc) return rc;
    smc_state *st = new smc_state();
    st->sys = sys;
    st->d = *desc;
    st->S = desc->n_soundings;
    st->N = desc->n_particles;
    st->P = st->S * st->N;
    st->M = (desc->kappa_max + 1) * (desc->lambda_max + 1);
    st->LMS = desc->kappa_max + desc->lambda_max + 1;
    st->stream = (cudaStream_t)stream;
    st->eps_mn = eps_mn;
    Params &p = st->pr;
    p.N = st->N;
    p.S = st->S;
    p.kappa_max = desc->kappa_max;
    p.lambda_max = desc->lambda_max;
    p.M = st->M;
    p.LMS = st->LMS;
    p.tau_log_prior = desc->tau_log_prior;
    p.zmax = desc->zmax;
    p.phi_lo = desc->phi_lo;
    p.phi_hi = desc->phi_hi;
    p.logtau_lo = desc->logtau_lo;
    p.logtau_hi = desc->logtau_hi;
    p.step_phi = desc->step_phi;
    p.step_m = desc->step_m;
    p.step_tau = desc->step_tau;
    p.step_c = desc->step_c;
    p.step_z = desc->step_z;
    p.seed = desc->seed;
    p.adaptive = desc->adaptive;
    p.zca_prob = desc->zca;
    p.DM = 3 + 2 * desc->kappa_max + 2 * desc->lambda_max;
    const int G = sys->host.G;
    const size_t P = st->P;
    if ((rc = alloc_pstate(st, &st->cur)) || (rc = alloc_pstate(st, &st->alt)) || (rc = alloc_pstate(st, &st->prop)) ||
        (rc = dalloc(st, &st->move, P)) || (rc = dalloc(st, &st->valid, P)) || (rc = dalloc(st, &st->anc, P)) ||
        (rc = dalloc(st, &st->perm, P)) || (rc = dalloc(st, &st->off, (size_t)st->S * (st->M + 1))) ||
        (rc = dalloc(st, &st->counts, (size_t)st->S * st->M)) || (rc = dalloc(st, &st->acc, (size_t)st->S * kMoves)) ||
        (rc = dalloc(st, &st->nprop, (size_t)st->S * kMoves)) || (rc = dalloc(st, &st->done, (size_t)st->S)) ||
        (rc = dalloc(st, &st->Wg, P)) || (rc = dalloc(st, &st->gamma, (size_t)st->S)) ||
        (rc = dalloc(st, &st->logz, (size_t)st->S * st->M)) || (rc = dalloc(st, &st->dgamma, (size_t)st->S)) ||
        (rc = dalloc(st, &st->C, P)) || (rc = dalloc(st, &st->m_nl, P)) ||
        (rc = dalloc(st, &st->m_logsig, P * st->LMS)) || (rc = dalloc(st, &st->m_logh, P * st->LMS)) ||
        (rc = dalloc(st, &st->m_m, P * st->LMS)) || (rc = dalloc(st, &st->m_logtau, P * st->LMS)) ||
        (rc = dalloc(st, &st->m_c, P * st->LMS)) || (rc = dalloc(st, &st->y, (size_t)st->S * G)) ||
        (rc = dalloc(st, &st->eps_an, (size_t)G)) || (rc = dalloc(st, &st->mgrad, P * st->LMS * 5)) ||
        (rc = dalloc(st, &st->grad_work, grad_work_bytes((int)P, G))) ||
        (rc = dalloc(st, &st->gcur, P * GD)) || (rc = dalloc(st, &st->gprop, P * GD)) ||
        (rc = dalloc(st, &st->lq, P)) || (rc = dalloc(st, &st->lacc, (size_t)st->S)) ||
        (rc = dalloc(st, &st->lprop, (size_t)st->S)) || (rc = dalloc(st, &st->lang_h, (size_t)st->S)) ||
        (rc = dalloc(st, &st->pca_mu, (size_t)st->S * st->M * p.DM)) ||
        (rc = dalloc(st, &st->pca_U, (size_t)st->S * st->M * p.DM * p.DM)) ||
        (rc = dalloc(st, &st->pca_Z, (size_t)st->S * st->M * p.DM * p.DM)) ||
        (rc = dalloc(st, &st->pca_lam, (size_t)st->S * st->M * p.DM)) ||
        (rc = dalloc(st, &st->pca_a, (size_t)st->S * st->M)) || (rc = dalloc(st, &st->pca_lo, (size_t)st->S * st->M)) ||
        (rc = dalloc(st, &st->pca_hi, (size_t)st->S * st->M)) || (rc = dalloc(st, &st->pca_ok, (size_t)st->S * st->M)) ||
        (rc = dalloc(st, &st->d_stage, 1)) || (rc = dalloc(st, &st->fwd_counter, 1)) ||
        (rc = dalloc(st, &st->d_sweeps, 1)) || (rc = dalloc(st, &st->d_gate, 1)) ||
        (rc = dalloc(st, &st->d_have_prev, 1)) || (rc = dalloc(st, &st->d_status, 1)) ||
        (rc = dalloc(st, &st->nonfinite, (size_t)st->S)) || (rc = dalloc(st, &st->d_post, (size_t)st->S * st->M)) ||
        (rc = dalloc(st, &st->d_lbf, (size_t)st->S)) ||
        (desc->precision == AEM_SMC_FP64 &&
         ((rc = dalloc(st, &st->m64_logsig, P * st->LMS)) || (rc = dalloc(st, &st->m64_logh, P * st->LMS)) ||
          (rc = dalloc(st, &st->m64_m, P * st->LMS)) || (rc = dalloc(st, &st->m64_logtau, P * st->LMS)) ||
          (rc = dalloc(st, &st->m64_c, P * st->LMS)))) ||
        (rc = dalloc(st, &st->lf, P))) {
        smc_destroy(st);
        return rc;
    }
    cudaError_t e = cudaMemcpy(st->y, y_obs, sizeof(double) * st->S * G, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(st->eps_an, eps_an, sizeof(double) * G, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        std::vector<double> h0(st->S, desc->langevin_h);
        e = cudaMemcpy(st->lang_h, h0.data(), sizeof(double) * st->S, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
        std::vector<double> a0((size_t)st->S * st->M, 1.0);
        e = cudaMemcpy(st->pca_a, a0.data(), sizeof(double) * a0.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(st->pca_ok, 0, sizeof(int) * st->S * st->M);
    if (e == cudaSuccess) e = cudaMemset(st->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(st->nonfinite, 0, sizeof(int) * st->S);
    if (e == cudaSuccess && desc->recycle_stages > 0) {
        const size_t HP = (size_t)desc->recycle_stages * st->P;
        if (HP * KS >= ((size_t)1 << 31)) {
            smc_destroy(st);
            return fail(AEM_ERR_INVALID_ARG, "smc_create: recycle_stages x particles too large for the history");
        }
        if ((rc = alloc_pstate(st, &st->hist, HP)) || (rc = dalloc(st, &st->hist_lognu, HP)) ||
            (rc = dalloc(st, &st->hist_w, HP)) ||
            (rc = dalloc(st, &st->gamma_hist, (size_t)st->S * kMaxRecycleStages)) ||
            (rc = dalloc(st, &st->logz_hist, (size_t)st->S * kMaxRecycleStages * st->M))) {
            smc_destroy(st);
            return rc;
        }
    }
    if (e != cudaSuccess) {
        smc_destroy(st);
        return cuda_fail(e, "smc_create: upload data");
    }
    // the reweight step's staging of the sounding's log-likelihoods: set now,
    // not during a stream capture of the stage loop
    const size_t rw_smem = reweight_dense_bytes(st->N);
    if (rw_smem > 48 * 1024) {
        e = cudaFuncSetAttribute(reweight_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rw_smem);
        if (e != cudaSuccess) {
            smc_destroy(st);
            return cuda_fail(e, "smc_create: reweight shared memory");
        }
    }
    *out = st;
    return AEM_OK;
}

extern "C" int smc_destroy(smc_state *st) {
    if (!st) return AEM_OK;
    for (void *q : st->allocs) cudaFree(q);
    delete st;
    return AEM_OK;
}

static int record_history(smc_state *st, const int *stage_dev = nullptr);

extern "C" int smc_init(smc_state *st) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_init: NULL state");
    prior_kernel<<<blocks_for(st->P, 128), 128, 0, st->stream>>>(st->cur, st->pr);
    AEM_CUDA_TRY(cudaGetLastError());
    AEM_CUDA_TRY(cudaMemsetAsync(st->gamma, 0, sizeof(double) * st->S, st->stream));
    AEM_CUDA_TRY(cudaMemsetAsync(st->logz, 0, sizeof(double) * st->S * st->M, st->stream));
    AEM_CUDA_TRY(cudaMemsetAsync(st->acc, 0, sizeof(int) * st->S * kMoves, st->stream));
    AEM_CUDA_TRY(cudaMemsetAsync(st->nprop, 0, sizeof(int) * st->S * kMoves, st->stream));
    AEM_CUDA_TRY(cudaMemsetAsync(st->lacc, 0, sizeof(int) * st->S, st->stream));
    AEM_CUDA_TRY(cudaMemsetAsync(st->lprop, 0, sizeof(int) * st->S, st->stream));
    AEM_CUDA_TRY(cudaMemsetAsync(st->d_status, 0, sizeof(int), st->stream));
    AEM_CUDA_TRY(cudaMemsetAsync(st->nonfinite, 0, sizeof(int) * st->S, st->stream));
    {
        std::vector<double> h0(st->S, st->d.langevin_h);
        std::vector<double> a0((size_t)st->S * st->M, 1.0);
        AEM_CUDA_TRY(cudaMemcpyAsync(st->lang_h, h0.data(), sizeof(double) * st->S, cudaMemcpyHostToDevice,
                                     st->stream));
        AEM_CUDA_TRY(cudaMemcpyAsync(st->pca_a, a0.data(), sizeof(double) * a0.size(), cudaMemcpyHostToDevice,
                                     st->stream));
        AEM_CUDA_TRY(cudaMemsetAsync(st->pca_ok, 0, sizeof(int) * st->S * st->M, st->stream));
        AEM_CUDA_TRY(cudaStreamSynchronize(st->stream));
    }
    st->stage = 0;
    st->have_prev = false;
    st->gcur_valid = false;
    int rc = run_loglik(st, st->cur);
    if (rc) return rc;
    return record_history(st);
}

// Synchronises the stream, then reads and clears the sampler's status word:
// AEM_OK, or the AEM_ERR_NONFINITE / AEM_ERR_NO_BRACKET a reweight step recorded.
static int take_status(smc_state *st) {
    int v = 0;
    AEM_CUDA_TRY(cudaMemcpyAsync(&v, st->d_status, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
    AEM_CUDA_TRY(cudaStreamSynchronize(st->stream));
    if (v == 0) return AEM_OK;
    AEM_CUDA_TRY(cudaMemsetAsync(st->d_status, 0, sizeof(int), st->stream));
    return fail(v, v == AEM_ERR_NO_BRACKET
                       ? "reweight: no tempering step kept TESS >= alpha N (bisection could not bracket)"
                       : "reweight: a sounding has no particle with a finite log-likelihood");
}

// The reweight step of every sounding: one CTA per sounding, or, when the
// soundings are few (the cluster of C CTAs per sounding still fits the SMs,
// C <= 8) and large (N >= 1024), the cluster-split form.
static int launch_reweight(smc_state *st, cudaStream_t stream) {
    int C = 1;
    if (st->N >= 1024)
        while (C < 8 && (long long)st->S * C * 2 <= st->sys->num_sms) C *= 2;
    if (C == 1) {
        const size_t smem = reweight_dense_bytes(st->N);
        reweight_kernel<<<st->S, kGroupThreads, smem, stream>>>(st->cur.ll, st->perm, st->off, st->counts, st->N,
                                                                st->M, st->d.alpha, st->d.bisect_iters, st->gamma,
                                                                st->logz, st->Wg, st->dgamma, st->done, st->d_status,
                                                                smem > 0);
        AEM_CUDA_TRY(cudaGetLastError());
        return AEM_OK;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(st->S * C), 1, 1);
    cfg.blockDim = dim3(kClusterThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    AEM_CUDA_TRY(cudaLaunchKernelEx(&cfg, reweight_cluster_kernel, (const double *)st->cur.ll, (const int *)st->perm,
                                    (const int *)st->off, (const int *)st->counts, st->N, st->M, st->d.alpha,
                                    st->d.bisect_iters, st->gamma, st->logz, st->Wg, st->dgamma, st->done,
                                    st->d_status));
    return AEM_OK;
}

static int launch_group(smc_state *st) {
    group_kernel<<<st->S, kGroupThreads, st->N, st->stream>>>(st->cur.kappa, st->cur.lam, st->N,
                                                              st->d.lambda_max + 1, st->M, st->perm, st->off,
                                                              st->counts);
    AEM_CUDA_TRY(cudaGetLastError());
    return AEM_OK;
}

extern "C" int smc_reweight(smc_state *st, double *gamma_out) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_reweight: NULL state");
    int rc = launch_group(st);
    if (rc) return rc;
    st->stage += 1;
    if ((rc = launch_reweight(st, st->stream))) return rc;
    if (gamma_out) {
        AEM_CUDA_TRY(cudaMemcpyAsync(gamma_out, st->gamma, sizeof(double) * st->S, cudaMemcpyDeviceToHost, st->stream));
        return take_status(st);  // synchronises
    }
    return AEM_OK;
}

extern "C" int smc_resample(smc_state *st) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_resample: NULL state");
    resample_kernel<<<st->S, kGroupThreads, 0, st->stream>>>(st->Wg, st->perm, st->off, st->counts, st->N, st->M,
                                                             nullptr, st->d.seed, st->stage, nullptr, st->C,
                                                             st->anc);
    AEM_CUDA_TRY(cudaGetLastError());
    gather_kernel<<<blocks_for(st->P, 256), 256, 0, st->stream>>>(st->alt, st->cur, st->anc, st->P);
    AEM_CUDA_TRY(cudaGetLastError());
    PState t = st->cur;
    st->cur = st->alt;
    st->alt = t;
    st->gcur_valid = false;
    return record_history(st);
}

static PcaView pca_view(smc_state *st) { return PcaView{st->pca_U, st->pca_lam, st->pca_a, st->pca_ok, st->pca_Z}; }

extern "C" int smc_propose(smc_state *st, int stage, int sweep) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_propose: NULL state");
    propose_kernel<<<blocks_for(st->P, 128), 128, 0, st->stream>>>(st->cur, st->prop, st->move, st->valid, st->pr,
                                                                    stage, sweep, pca_view(st), nullptr, st->lf);
    AEM_CUDA_TRY(cudaGetLastError());
    return AEM_OK;
}

// Section 3.2's adaptive within-model proposal for the current stage: fit
// each (sounding, model)'s Gaussian, then bisect its scale on trial
// proposals (desc.pca_bisect_iters forward passes) towards desc.pca_target.
// Particle recycling: the current (post-resample) particles become history
// slot stage mod H; this stage's gamma and log Z are kept for the weights.
// stage_dev (graph form): the stage comes from the device counter, whose
// bound the caller has checked.
static int record_history(smc_state *st, const int *stage_dev) {
    if (st->d.recycle_stages <= 0) return AEM_OK;
    const int t = st->stage, H = st->d.recycle_stages;
    if (!stage_dev && t >= kMaxRecycleStages)
        return fail(AEM_ERR_INVALID_ARG, "particle recycling keeps at most 1024 stages");
    record_slot_kernel<<<blocks_for(st->P, 256), 256, 0, st->stream>>>(st->hist, st->cur, st->P, t % H, H,
                                                                       stage_dev);
    AEM_CUDA_TRY(cudaGetLastError());
    record_stage_kernel<<<blocks_for(st->S, 128), 128, 0, st->stream>>>(st->gamma, st->logz, st->S, st->M, t,
                                                                        st->gamma_hist, st->logz_hist, stage_dev);
    AEM_CUDA_TRY(cudaGetLastError());
    return AEM_OK;
}

static int adapt_stage(smc_state *st, const int *stage_dev = nullptr) {
    int rc = launch_group(st);
    if (rc) return rc;
    const int nb = st->S * st->M, DM = st->pr.DM;
    const size_t smem = fit_smem_bytes(DM);
    if (smem > 48 * 1024)
        AEM_CUDA_TRY(cudaFuncSetAttribute(pca_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (st->d.recycle_stages > 0) {
        const int t = st->stage, H = st->d.recycle_stages;
        // with the device counter the grid covers every slot and the kernels
        // take t and the slots in use from the counter
        const int n_used = stage_dev ? H : (t + 1 < H ? t + 1 : H);
        if (smem > 48 * 1024)
            AEM_CUDA_TRY(cudaFuncSetAttribute(pca_fit_recycle_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        recycle_weight_kernel<<<blocks_for((long long)n_used * st->P, 128), 128, 0, st->stream>>>(
            st->hist, st->P, n_used, st->N, st->M, st->d.lambda_max + 1, t, st->gamma_hist, st->logz_hist,
            st->hist_lognu, H, stage_dev);
        AEM_CUDA_TRY(cudaGetLastError());
        pca_fit_recycle_kernel<<<nb, kFitThreads, smem, st->stream>>>(
            st->hist, st->hist_lognu, st->hist_w, n_used, st->P, st->counts, st->pr, st->d.pca_ridge, st->pca_mu,
            st->pca_U, st->pca_lam, st->pca_ok, st->pca_a, H, stage_dev, st->pca_Z);
    } else {
        pca_fit_kernel<<<nb, kFitThreads, smem, st->stream>>>(st->cur, st->perm, st->off, st->counts, st->pr,
                                                               st->d.pca_ridge, st->pca_mu, st->pca_U, st->pca_lam,
                                                               st->pca_ok, st->pca_a, st->pca_Z);
    }
    AEM_CUDA_TRY(cudaGetLastError());
    pca_bracket_kernel<<<blocks_for(nb, 128), 128, 0, st->stream>>>(st->pca_ok, st->pca_a, nb, 3.0, st->pca_lo,
                                                                     st->pca_hi);
    AEM_CUDA_TRY(cudaGetLastError());
    for (int it = 0; it < st->d.pca_bisect_iters; ++it) {
        pca_trial_kernel<<<blocks_for(st->P, 128), 128, 0, st->stream>>>(st->cur, st->prop, st->valid, st->pr,
                                                                          pca_view(st), st->pca_lo, st->pca_hi,
                                                                          st->stage, stage_dev);
        AEM_CUDA_TRY(cudaGetLastError());
        if ((rc = run_loglik(st, st->prop, nullptr, st->valid))) return rc;
        pca_stat_kernel<<<nb, 128, 0, st->stream>>>(st->cur.ll, st->prop.ll, st->valid, st->perm, st->off,
                                                    st->counts, st->pca_ok, st->gamma, st->pr, st->d.pca_target,
                                                    st->pca_lo, st->pca_hi);
        AEM_CUDA_TRY(cudaGetLastError());
    }
    pca_finish_kernel<<<blocks_for(nb, 128), 128, 0, st->stream>>>(st->pca_ok, st->pca_lo, st->pca_hi, nb,
                                                                    st->pca_a);
    AEM_CUDA_TRY(cudaGetLastError());
    return AEM_OK;
}

static int langevin_sweeps(smc_state *st, int n, const int *stage_dev = nullptr) {
    AEM_CUDA_TRY(cudaMemsetAsync(st->lacc, 0, sizeof(int) * st->S, st->stream));
    AEM_CUDA_TRY(cudaMemsetAsync(st->lprop, 0, sizeof(int) * st->S, st->stream));
    if (n <= 0) return AEM_OK;
    int rc;
    // the current particles' likelihood and gradient come from the adjoint
    // kernel, so both sides of every Langevin test use the same evaluation
    if ((rc = run_grad(st, st->cur, st->gcur))) return rc;
    st->gcur_valid = true;
    for (int l = 0; l < n; ++l) {
        langevin_propose_kernel<<<blocks_for(st->P, 128), 128, 0, st->stream>>>(
            st->cur, st->prop, st->gcur, st->gamma, st->lang_h, st->pr, st->stage, l, st->valid, st->lq, stage_dev);
        AEM_CUDA_TRY(cudaGetLastError());
        if ((rc = run_grad(st, st->prop, st->gprop, st->valid))) return rc;
        langevin_accept_kernel<<<blocks_for(st->P, 128), 128, 0, st->stream>>>(
            st->cur, st->prop, st->gcur, st->gprop, st->valid, st->lq, st->gamma, st->lang_h, st->pr, st->stage, l,
            st->lacc, st->lprop, stage_dev);
        AEM_CUDA_TRY(cudaGetLastError());
    }
    return AEM_OK;
}

static int sweeps_for_stage(smc_state *st, int n_sweeps, int *R) {
    if (n_sweeps > 0) {
        *R = n_sweeps;
        return AEM_OK;
    }
    if (!st->have_prev) {
        *R = st->d.r_max;
        return AEM_OK;
    }
    // App. B: R = ceil(log c / log(1 - p_min)) from the previous stage's
    // acceptance rates (the first sounding's; soundings share R).
    double pmin = 1.0;
    for (int m = 0; m < kMoves; ++m) {
        int np = st->nprop_prev[m];
        double r = np > 0 ? (double)st->acc_prev[m] / np : 1.0;
        pmin = r < pmin ? r : pmin;
    }
    int r;
    if (pmin <= 0.0)
        r = st->d.r_max;
    else if (pmin >= 1.0)
        r = 1;
    else
        r = (int)std::ceil(std::log(st->d.c_mut) / std::log(1.0 - pmin));
    *R = r < 1 ? 1 : (r > st->d.r_max ? st->d.r_max : r);
    return AEM_OK;
}

extern "C" int smc_mutate(smc_state *st, int n_sweeps) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_mutate: NULL state");
    int R = 0, rc;
    if ((rc = sweeps_for_stage(st, n_sweeps, &R))) return rc;
    AEM_CUDA_TRY(cudaMemsetAsync(st->acc, 0, sizeof(int) * st->S * kMoves, st->stream));
    AEM_CUDA_TRY(cudaMemsetAsync(st->nprop, 0, sizeof(int) * st->S * kMoves, st->stream));
    if (st->d.adaptive && (rc = adapt_stage(st))) return rc;
    for (int sw = 0; sw < R; ++sw) {
        if ((rc = smc_propose(st, st->stage, sw))) return rc;
        if ((rc = run_loglik(st, st->prop, nullptr, st->valid))) return rc;
        accept_kernel<<<blocks_for(st->P, 256), 256, 0, st->stream>>>(st->cur, st->prop, st->move, st->valid,
                                                                      st->gamma, st->pr, st->stage, sw, st->acc,
                                                                      st->nprop, nullptr, st->lf);
        AEM_CUDA_TRY(cudaGetLastError());
    }
    if (R > 0) st->gcur_valid = false;
    if ((rc = langevin_sweeps(st, st->d.n_langevin))) return rc;
    if (st->d.n_langevin > 0 && st->d.langevin_adapt) {
        langevin_adapt_kernel<<<blocks_for(st->S, 128), 128, 0, st->stream>>>(st->lacc, st->lprop, st->S,
                                                                              st->lang_h);
        AEM_CUDA_TRY(cudaGetLastError());
    }
    st->acc_prev.assign(st->S * kMoves, 0);
    st->nprop_prev.assign(st->S * kMoves, 0);
    AEM_CUDA_TRY(cudaMemcpyAsync(st->acc_prev.data(), st->acc, sizeof(int) * st->S * kMoves, cudaMemcpyDeviceToHost,
                                 st->stream));
    AEM_CUDA_TRY(cudaMemcpyAsync(st->nprop_prev.data(), st->nprop, sizeof(int) * st->S * kMoves,
                                 cudaMemcpyDeviceToHost, st->stream));
    AEM_CUDA_TRY(cudaStreamSynchronize(st->stream));
    st->have_prev = true;
    return AEM_OK;
}

extern "C" int smc_run(smc_state *st, int max_stages, int n_sweeps, int *stages_out) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_run: NULL state");
    std::vector<double> g(st->S);
    int rc, t = 0;
    for (; t < max_stages; ++t) {
        if ((rc = smc_reweight(st, g.data()))) return rc;
        if ((rc = smc_resample(st))) return rc;
        if ((rc = smc_mutate(st, n_sweeps))) return rc;
        bool all = true;
        for (double v : g) all = all && v >= 1.0;
        if (all) {
            ++t;
            break;
        }
    }
    if (stages_out) *stages_out = t;
    return AEM_OK;
}

// One stage of Algorithm 1 (reweight, resample, R sweeps of the moves, with
// the recycling record after the resample, the adaptive fit and scale
// bisection before the sweeps and the Langevin sweeps after them when the
// descriptor turns those on) enqueued on st->stream without host
// synchronisation or allocation, reading the stage number from st->d_stage;
// ends with the loop condition.
static int enqueue_graph_stage(smc_state *st, int R, int stop_stage, cudaGraphConditionalHandle h) {
    // R <= 0: App. B's sweep count, decided on the device each stage; the
    // graph holds r_max gated sweeps
    const bool adaptive_r = R <= 0;
    cudaStream_t s = st->stream;
    stage_inc_kernel<<<1, 32, 0, s>>>(st->d_stage);
    AEM_CUDA_TRY(cudaGetLastError());
    int rc = launch_group(st);
    if (rc) return rc;
    if ((rc = launch_reweight(st, s))) return rc;
    resample_kernel<<<st->S, kGroupThreads, 0, s>>>(st->Wg, st->perm, st->off, st->counts, st->N, st->M, nullptr,
                                                    st->d.seed, 0, st->d_stage, st->C, st->anc);
    AEM_CUDA_TRY(cudaGetLastError());
    gather_kernel<<<blocks_for(st->P, 256), 256, 0, s>>>(st->alt, st->cur, st->anc, st->P);
    AEM_CUDA_TRY(cudaGetLastError());
    copy_state_kernel<<<blocks_for(st->P, 256), 256, 0, s>>>(st->cur, st->alt, st->P);
    AEM_CUDA_TRY(cudaGetLastError());
    if ((rc = record_history(st, st->d_stage))) return rc;
    if (adaptive_r) {  // from the previous stage's counts, before they are cleared
        sweep_count_kernel<<<1, 32, 0, s>>>(st->acc, st->nprop, st->d_have_prev, st->d.c_mut, st->d.r_max,
                                            st->d_sweeps);
        AEM_CUDA_TRY(cudaGetLastError());
    }
    AEM_CUDA_TRY(cudaMemsetAsync(st->acc, 0, sizeof(int) * st->S * kMoves, s));
    AEM_CUDA_TRY(cudaMemsetAsync(st->nprop, 0, sizeof(int) * st->S * kMoves, s));
    if (st->d.adaptive && (rc = adapt_stage(st, st->d_stage))) return rc;
    const int n_sw = adaptive_r ? st->d.r_max : R;
    const int *gate = adaptive_r ? st->d_gate : nullptr;
    for (int sw = 0; sw < n_sw; ++sw) {
        if (adaptive_r) {
            sweep_gate_kernel<<<1, 32, 0, s>>>(st->d_sweeps, sw, st->d_gate);
            AEM_CUDA_TRY(cudaGetLastError());
        }
        propose_kernel<<<blocks_for(st->P, 128), 128, 0, s>>>(st->cur, st->prop, st->move, st->valid, st->pr, 0, sw,
                                                               pca_view(st), st->d_stage, st->lf, gate);
        AEM_CUDA_TRY(cudaGetLastError());
        if ((rc = run_loglik(st, st->prop, gate, st->valid))) return rc;
        accept_kernel<<<blocks_for(st->P, 256), 256, 0, s>>>(st->cur, st->prop, st->move, st->valid, st->gamma,
                                                             st->pr, 0, sw, st->acc, st->nprop, st->d_stage, st->lf,
                                                             gate);
        AEM_CUDA_TRY(cudaGetLastError());
    }
    if ((rc = langevin_sweeps(st, st->d.n_langevin, st->d_stage))) return rc;
    if (st->d.n_langevin > 0 && st->d.langevin_adapt) {
        langevin_adapt_kernel<<<blocks_for(st->S, 128), 128, 0, s>>>(st->lacc, st->lprop, st->S, st->lang_h);
        AEM_CUDA_TRY(cudaGetLastError());
    }
    set_flag_kernel<<<1, 32, 0, s>>>(st->d_have_prev, 1);
    AEM_CUDA_TRY(cudaGetLastError());
    stage_cond_kernel<<<1, 32, 0, s>>>(st->gamma, st->S, st->d_stage, stop_stage, st->d_status, h);
    AEM_CUDA_TRY(cudaGetLastError());
    return AEM_OK;
}

extern "C" int smc_run_graph(smc_state *st, int max_stages, int n_sweeps, int *stages_out) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_run_graph: NULL state");
    if (max_stages < 1) return fail(AEM_ERR_INVALID_ARG, "smc_run_graph: max_stages must be >= 1");
    const int s0 = st->stage;
    if (st->d.recycle_stages > 0 && (long long)s0 + max_stages >= kMaxRecycleStages)
        return fail(AEM_ERR_INVALID_ARG, "smc_run_graph: particle recycling keeps at most 1024 stages");
    AEM_CUDA_TRY(cudaStreamSynchronize(st->stream));
    AEM_CUDA_TRY(cudaMemcpy(st->d_stage, &s0, sizeof(int), cudaMemcpyHostToDevice));
    // the previous stage's acceptance counts as the host path holds them (the
    // device copies may predate a restore)
    const int hp = st->have_prev ? 1 : 0;
    AEM_CUDA_TRY(cudaMemcpy(st->d_have_prev, &hp, sizeof(int), cudaMemcpyHostToDevice));
    if (st->have_prev) {
        AEM_CUDA_TRY(cudaMemcpy(st->acc, st->acc_prev.data(), sizeof(int) * st->S * kMoves, cudaMemcpyHostToDevice));
        AEM_CUDA_TRY(cudaMemcpy(st->nprop, st->nprop_prev.data(), sizeof(int) * st->S * kMoves,
                                cudaMemcpyHostToDevice));
    }
    cudaStream_t user = st->stream, cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = AEM_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaGraphCreate(&graph, 0);
    cudaGraphConditionalHandle handle{};
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np{};
    cudaGraphNode_t loop = nullptr;
    if (e == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = handle;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&loop, graph, nullptr, nullptr, 0, &np);
    }
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            st->stream = cap;
            rc = enqueue_graph_stage(st, n_sweeps, s0 + max_stages, handle);
            st->stream = user;
            cudaGraph_t captured = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(cap, &captured);
            if (rc == AEM_OK) e = e2;
        }
    }
    if (rc == AEM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (rc == AEM_OK && e == cudaSuccess) e = cudaGraphLaunch(exec, user);
    if (rc == AEM_OK && e == cudaSuccess) e = cudaStreamSynchronize(user);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "smc_run_graph");
    int s1 = s0;
    AEM_CUDA_TRY(cudaMemcpy(&s1, st->d_stage, sizeof(int), cudaMemcpyDeviceToHost));
    st->stage = s1;
    st->gcur_valid = false;
    st->acc_prev.assign(st->S * kMoves, 0);
    st->nprop_prev.assign(st->S * kMoves, 0);
    AEM_CUDA_TRY(cudaMemcpy(st->acc_prev.data(), st->acc, sizeof(int) * st->S * kMoves, cudaMemcpyDeviceToHost));
    AEM_CUDA_TRY(cudaMemcpy(st->nprop_prev.data(), st->nprop, sizeof(int) * st->S * kMoves, cudaMemcpyDeviceToHost));
    st->have_prev = true;
    if (stages_out) *stages_out = s1 - s0;
    return take_status(st);
}

extern "C" int smc_model_odds(const smc_state *cst, double *post_k, double *log_bfipd, double *log_z_k) {
    smc_state *st = const_cast<smc_state *>(cst);
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_model_odds: NULL state");
    int rc = launch_group(st);
    if (rc) return rc;
    odds_kernel<<<blocks_for(st->S, 128), 128, 0, st->stream>>>(st->counts, st->S, st->M, st->d.lambda_max + 1, st->N,
                                                                st->d_post, st->d_lbf);
    AEM_CUDA_TRY(cudaGetLastError());
    if (post_k)
        AEM_CUDA_TRY(cudaMemcpyAsync(post_k, st->d_post, sizeof(double) * st->S * st->M, cudaMemcpyDeviceToHost,
                                     st->stream));
    if (log_bfipd)
        AEM_CUDA_TRY(cudaMemcpyAsync(log_bfipd, st->d_lbf, sizeof(double) * st->S, cudaMemcpyDeviceToHost, st->stream));
    if (log_z_k)
        AEM_CUDA_TRY(cudaMemcpyAsync(log_z_k, st->logz, sizeof(double) * st->S * st->M, cudaMemcpyDeviceToHost,
                                     st->stream));
    AEM_CUDA_TRY(cudaStreamSynchronize(st->stream));
    return AEM_OK;
}

extern "C" int smc_status(smc_state *st, int *status, int *nonfinite) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_status: NULL state");
    if (nonfinite)
        AEM_CUDA_TRY(cudaMemcpyAsync(nonfinite, st->nonfinite, sizeof(int) * st->S, cudaMemcpyDeviceToHost,
                                     st->stream));
    int v = 0;
    AEM_CUDA_TRY(cudaMemcpyAsync(&v, st->d_status, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
    AEM_CUDA_TRY(cudaStreamSynchronize(st->stream));
    if (v) AEM_CUDA_TRY(cudaMemsetAsync(st->d_status, 0, sizeof(int), st->stream));
    if (status) *status = v;
    return AEM_OK;
}

extern "C" int smc_stats(const smc_state *st, double *gamma, int *stage, int *accepted, int *proposed) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_stats: NULL state");
    if (gamma) AEM_CUDA_TRY(cudaMemcpy(gamma, st->gamma, sizeof(double) * st->S, cudaMemcpyDeviceToHost));
    if (stage) *stage = st->stage;
    if (accepted) AEM_CUDA_TRY(cudaMemcpy(accepted, st->acc, sizeof(int) * st->S * kMoves, cudaMemcpyDeviceToHost));
    if (proposed) AEM_CUDA_TRY(cudaMemcpy(proposed, st->nprop, sizeof(int) * st->S * kMoves, cudaMemcpyDeviceToHost));
    return AEM_OK;
}

static PState pick(smc_state *st, int which) { return which == 1 ? st->prop : st->cur; }

extern "C" int smc_get_particles(const smc_state *cst, int which, smc_particles_host *h) {
    smc_state *st = const_cast<smc_state *>(cst);
    if (!st || !h) return fail(AEM_ERR_INVALID_ARG, "smc_get_particles: NULL argument");
    AEM_CUDA_TRY(cudaStreamSynchronize(st->stream));
    PState p = pick(st, which);
    const size_t P = st->P;
    AEM_CUDA_TRY(cudaMemcpy(h->kappa, p.kappa, sizeof(int) * P, cudaMemcpyDeviceToHost));
    AEM_CUDA_TRY(cudaMemcpy(h->lam, p.lam, sizeof(int) * P, cudaMemcpyDeviceToHost));
    AEM_CUDA_TRY(cudaMemcpy(h->phib, p.phib, sizeof(float) * P, cudaMemcpyDeviceToHost));
    AEM_CUDA_TRY(cudaMemcpy(h->tau, p.tau, sizeof(float) * P, cudaMemcpyDeviceToHost));
    AEM_CUDA_TRY(cudaMemcpy(h->c, p.c, sizeof(float) * P, cudaMemcpyDeviceToHost));
    AEM_CUDA_TRY(cudaMemcpy(h->zc, p.zc, sizeof(float) * P * KS, cudaMemcpyDeviceToHost));
    AEM_CUDA_TRY(cudaMemcpy(h->phic, p.phic, sizeof(float) * P * KS, cudaMemcpyDeviceToHost));
    AEM_CUDA_TRY(cudaMemcpy(h->zm, p.zm, sizeof(float) * P * KS, cudaMemcpyDeviceToHost));
    AEM_CUDA_TRY(cudaMemcpy(h->mv, p.mv, sizeof(float) * P * KS, cudaMemcpyDeviceToHost));
    AEM_CUDA_TRY(cudaMemcpy(h->ll, p.ll, sizeof(double) * P, cudaMemcpyDeviceToHost));
    if (h->move && which == 1) AEM_CUDA_TRY(cudaMemcpy(h->move, st->move, P, cudaMemcpyDeviceToHost));
    if (h->valid && which == 1) AEM_CUDA_TRY(cudaMemcpy(h->valid, st->valid, P, cudaMemcpyDeviceToHost));
    return AEM_OK;
}

extern "C" int smc_set_particles(smc_state *st, const smc_particles_host *h, const double *gamma, const double *log_z,
                                 int stage) {
    if (!st || !h) return fail(AEM_ERR_INVALID_ARG, "smc_set_particles: NULL argument");
    const size_t P = st->P;
    PState p = st->cur;
    AEM_CUDA_TRY(cudaStreamSynchronize(st->stream));
    AEM_CUDA_TRY(cudaMemcpy(p.kappa, h->kappa, sizeof(int) * P, cudaMemcpyHostToDevice));
    AEM_CUDA_TRY(cudaMemcpy(p.lam, h->lam, sizeof(int) * P, cudaMemcpyHostToDevice));
    AEM_CUDA_TRY(cudaMemcpy(p.phib, h->phib, sizeof(float) * P, cudaMemcpyHostToDevice));
    AEM_CUDA_TRY(cudaMemcpy(p.tau, h->tau, sizeof(float) * P, cudaMemcpyHostToDevice));
    AEM_CUDA_TRY(cudaMemcpy(p.c, h->c, sizeof(float) * P, cudaMemcpyHostToDevice));
    AEM_CUDA_TRY(cudaMemcpy(p.zc, h->zc, sizeof(float) * P * KS, cudaMemcpyHostToDevice));
    AEM_CUDA_TRY(cudaMemcpy(p.phic, h->phic, sizeof(float) * P * KS, cudaMemcpyHostToDevice));
    AEM_CUDA_TRY(cudaMemcpy(p.zm, h->zm, sizeof(float) * P * KS, cudaMemcpyHostToDevice));
    AEM_CUDA_TRY(cudaMemcpy(p.mv, h->mv, sizeof(float) * P * KS, cudaMemcpyHostToDevice));
    AEM_CUDA_TRY(cudaMemcpy(p.ll, h->ll, sizeof(double) * P, cudaMemcpyHostToDevice));
    if (gamma) AEM_CUDA_TRY(cudaMemcpy(st->gamma, gamma, sizeof(double) * st->S, cudaMemcpyHostToDevice));
    if (log_z) AEM_CUDA_TRY(cudaMemcpy(st->logz, log_z, sizeof(double) * st->S * st->M, cudaMemcpyHostToDevice));
    if (stage >= 0) st->stage = stage;
    st->gcur_valid = false;
    return AEM_OK;
}

extern "C" int smc_loglik_current(smc_state *st) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_loglik_current: NULL state");
    st->gcur_valid = false;
    return run_loglik(st, st->cur);
}

extern "C" int smc_grad_current(smc_state *st, float *grad_host) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_grad_current: NULL state");
    int rc = run_grad(st, st->cur, st->gcur);
    if (rc) return rc;
    st->gcur_valid = true;
    if (grad_host) {
        AEM_CUDA_TRY(cudaMemcpyAsync(grad_host, st->gcur, sizeof(float) * (size_t)st->P * GD, cudaMemcpyDeviceToHost,
                                     st->stream));
        AEM_CUDA_TRY(cudaStreamSynchronize(st->stream));
    }
    return AEM_OK;
}

extern "C" int smc_langevin_propose(smc_state *st, int stage, int sweep) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_langevin_propose: NULL state");
    if (!st->gcur_valid)
        return fail(AEM_ERR_INVALID_ARG, "smc_langevin_propose: no gradient of the current particles (smc_grad_current)");
    langevin_propose_kernel<<<blocks_for(st->P, 128), 128, 0, st->stream>>>(
        st->cur, st->prop, st->gcur, st->gamma, st->lang_h, st->pr, stage, sweep, st->valid, st->lq, nullptr);
    AEM_CUDA_TRY(cudaGetLastError());
    return AEM_OK;
}

extern "C" int smc_langevin(smc_state *st, int n_sweeps) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_langevin: NULL state");
    if (n_sweeps < 0 || n_sweeps > 1000) return fail(AEM_ERR_INVALID_ARG, "smc_langevin: n_sweeps outside 0..1000");
    int rc = langevin_sweeps(st, n_sweeps);
    if (rc) return rc;
    AEM_CUDA_TRY(cudaStreamSynchronize(st->stream));
    return AEM_OK;
}

extern "C" int smc_ppd(smc_state *st, double *mean, double *var, double *z, float *gates_host) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_ppd: NULL state");
    const int G = st->sys->host.G;
    const size_t P = st->P, S = st->S;
    int rc;
    if (!st->ppd_gates) {
        if ((rc = dalloc(st, &st->ppd_gates, P * G)) || (rc = dalloc(st, &st->ppd_out, 3 * S * G))) return rc;
    }
    merge_kernel<float><<<blocks_for(st->P, 256), 256, 0, st->stream>>>(st->cur, st->P, st->LMS, st->m_nl, st->m_logsig,
                                                                st->m_logh, st->m_m, st->m_logtau, st->m_c);
    AEM_CUDA_TRY(cudaGetLastError());
    aem_models_f32 mm{st->P, st->LMS, st->m_nl, st->m_logsig, st->m_logh, st->m_m, st->m_logtau, st->m_c};
    if ((rc = aem_forward_f32(st->sys, &mm, st->ppd_gates, nullptr, st->stream))) return rc;
    double *o = st->ppd_out;
    ppd_kernel<<<(unsigned)(S * G), 256, 0, st->stream>>>(st->ppd_gates, st->N, G, st->y, st->eps_an, st->eps_mn, o,
                                                          o + S * G, o + 2 * S * G);
    AEM_CUDA_TRY(cudaGetLastError());
    if (mean) AEM_CUDA_TRY(cudaMemcpyAsync(mean, o, sizeof(double) * S * G, cudaMemcpyDeviceToHost, st->stream));
    if (var) AEM_CUDA_TRY(cudaMemcpyAsync(var, o + S * G, sizeof(double) * S * G, cudaMemcpyDeviceToHost, st->stream));
    if (z) AEM_CUDA_TRY(cudaMemcpyAsync(z, o + 2 * S * G, sizeof(double) * S * G, cudaMemcpyDeviceToHost, st->stream));
    if (gates_host)
        AEM_CUDA_TRY(cudaMemcpyAsync(gates_host, st->ppd_gates, sizeof(float) * P * G, cudaMemcpyDeviceToHost,
                                     st->stream));
    AEM_CUDA_TRY(cudaStreamSynchronize(st->stream));
    return AEM_OK;
}

extern "C" int smc_get_log_factors(const smc_state *cst, double *lf) {
    smc_state *st = const_cast<smc_state *>(cst);
    if (!st || !lf) return fail(AEM_ERR_INVALID_ARG, "smc_get_log_factors: NULL argument");
    AEM_CUDA_TRY(cudaStreamSynchronize(st->stream));
    AEM_CUDA_TRY(cudaMemcpy(lf, st->lf, sizeof(double) * st->P, cudaMemcpyDeviceToHost));
    return AEM_OK;
}

extern "C" int smc_adapt(smc_state *st) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_adapt: NULL state");
    return adapt_stage(st);
}

extern "C" int smc_get_adaptation(const smc_state *cst, double *mu, double *U, double *lam, double *scale, int *ok) {
    smc_state *st = const_cast<smc_state *>(cst);
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_get_adaptation: NULL state");
    const size_t nb = (size_t)st->S * st->M, DM = st->pr.DM;
    AEM_CUDA_TRY(cudaStreamSynchronize(st->stream));
    if (mu) AEM_CUDA_TRY(cudaMemcpy(mu, st->pca_mu, sizeof(double) * nb * DM, cudaMemcpyDeviceToHost));
    if (U) AEM_CUDA_TRY(cudaMemcpy(U, st->pca_U, sizeof(double) * nb * DM * DM, cudaMemcpyDeviceToHost));
    if (lam) AEM_CUDA_TRY(cudaMemcpy(lam, st->pca_lam, sizeof(double) * nb * DM, cudaMemcpyDeviceToHost));
    if (scale) AEM_CUDA_TRY(cudaMemcpy(scale, st->pca_a, sizeof(double) * nb, cudaMemcpyDeviceToHost));
    if (ok) AEM_CUDA_TRY(cudaMemcpy(ok, st->pca_ok, sizeof(int) * nb, cudaMemcpyDeviceToHost));
    return AEM_OK;
}

extern "C" int smc_langevin_stats(const smc_state *st, int *accepted, int *proposed, double *h) {
    if (!st) return fail(AEM_ERR_INVALID_ARG, "smc_langevin_stats: NULL state");
    if (h) AEM_CUDA_TRY(cudaMemcpy(h, st->lang_h, sizeof(double) * st->S, cudaMemcpyDeviceToHost));
    if (accepted) AEM_CUDA_TRY(cudaMemcpy(accepted, st->lacc, sizeof(int) * st->S, cudaMemcpyDeviceToHost));
    if (proposed) AEM_CUDA_TRY(cudaMemcpy(proposed, st->lprop, sizeof(int) * st->S, cudaMemcpyDeviceToHost));
    return AEM_OK;
}

// ------------------------------------------------------ checkpoint / restore
// Image layout (little-endian host order, version 2): a fixed header, then the
// current particles (kappa, lam int32 [P]; phib, tau, c float [P]; zc, phic,
// zm, mv float [P][SLOTS]; ll double [P]), gamma [S], log Z [S][M], Langevin
// step [S] (doubles), and the previous stage's acceptance counts [S][6] x 2
// (int32, valid when have_prev).  With the adaptive proposal follows the
// scale a_k of every (sounding, model) [S][M] (double: the next stage's
// bisection is centred on it; the fit itself is rebuilt at the start of the
// next stage's sweeps).  With particle recycling follow the H history slots
// (H x P particle records in the layout of the current particles) and the
// gamma [S][t+1] and log Z [S][t+1][M] of stages 0..t, t the stage counter.
namespace {
constexpr char kCkptMagic[8] = {'A', 'E', 'M', 'S', 'M', 'C', 'C', 'K'};
constexpr int32_t kCkptVersion = 2;
struct CkptHeader {
    char magic[8];
    int32_t version, S, N, M, kappa_max, lambda_max, stage, have_prev;
    int32_t adaptive, recycle_stages, reserved0, reserved1;
    uint64_t seed;
    uint64_t payload_bytes;
};

size_t particle_bytes(size_t n) {
    return n * (2 * sizeof(int32_t) + 3 * sizeof(float) + 4 * KS * sizeof(float) + sizeof(double));
}

size_t ckpt_payload(const smc_state *st, int stage) {
    const size_t S = st->S, M = st->M;
    size_t b = particle_bytes(st->P) + S * (2 + M) * sizeof(double) + 2 * S * kMoves * sizeof(int32_t);
    if (st->d.adaptive) b += S * M * sizeof(double);
    if (st->d.recycle_stages > 0)
        b += particle_bytes((size_t)st->d.recycle_stages * st->P) + S * (size_t)(stage + 1) * (1 + M) * sizeof(double);
    return b;
}

template <class T>
int d2h(unsigned char *&o, const T *src, size_t n, cudaStream_t s) {
    AEM_CUDA_TRY(cudaMemcpyAsync(o, src, n * sizeof(T), cudaMemcpyDeviceToHost, s));
    o += n * sizeof(T);
    return AEM_OK;
}

template <class T>
int h2d(T *dst, const unsigned char *&i, size_t n, cudaStream_t s) {
    AEM_CUDA_TRY(cudaMemcpyAsync(dst, i, n * sizeof(T), cudaMemcpyHostToDevice, s));
    i += n * sizeof(T);
    return AEM_OK;
}

int particles_d2h(unsigned char *&o, const PState &c, size_t n, cudaStream_t s) {
    int rc;
    if ((rc = d2h(o, c.kappa, n, s)) || (rc = d2h(o, c.lam, n, s)) || (rc = d2h(o, c.phib, n, s)) ||
        (rc = d2h(o, c.tau, n, s)) || (rc = d2h(o, c.c, n, s)) || (rc = d2h(o, c.zc, n * KS, s)) ||
        (rc = d2h(o, c.phic, n * KS, s)) || (rc = d2h(o, c.zm, n * KS, s)) || (rc = d2h(o, c.mv, n * KS, s)) ||
        (rc = d2h(o, c.ll, n, s)))
        return rc;
    return AEM_OK;
}

int particles_h2d(const PState &c, const unsigned char *&i, size_t n, cudaStream_t s) {
    int rc;
    if ((rc = h2d(c.kappa, i, n, s)) || (rc = h2d(c.lam, i, n, s)) || (rc = h2d(c.phib, i, n, s)) ||
        (rc = h2d(c.tau, i, n, s)) || (rc = h2d(c.c, i, n, s)) || (rc = h2d(c.zc, i, n * KS, s)) ||
        (rc = h2d(c.phic, i, n * KS, s)) || (rc = h2d(c.zm, i, n * KS, s)) || (rc = h2d(c.mv, i, n * KS, s)) ||
        (rc = h2d(c.ll, i, n, s)))
        return rc;
    return AEM_OK;
}

// rows of a [S][kMaxRecycleStages][w] device array, the first `cols` entries
// (of w doubles) of each sounding's row, packed on the host
int hist_rows_d2h(unsigned char *&o, const double *src, size_t S, size_t cols, size_t w, cudaStream_t s) {
    const size_t width = cols * w * sizeof(double);
    AEM_CUDA_TRY(cudaMemcpy2DAsync(o, width, src, (size_t)kMaxRecycleStages * w * sizeof(double), width, S,
                                   cudaMemcpyDeviceToHost, s));
    o += width * S;
    return AEM_OK;
}

int hist_rows_h2d(double *dst, const unsigned char *&i, size_t S, size_t cols, size_t w, cudaStream_t s) {
    const size_t width = cols * w * sizeof(double);
    AEM_CUDA_TRY(cudaMemcpy2DAsync(dst, (size_t)kMaxRecycleStages * w * sizeof(double), i, width, width, S,
                                   cudaMemcpyHostToDevice, s));
    i += width * S;
    return AEM_OK;
}
}  // namespace

extern "C" int smc_checkpoint(const smc_state *cst, void *buf, size_t *size) {
    smc_state *st = const_cast<smc_state *>(cst);
    if (!st || !size) return fail(AEM_ERR_INVALID_ARG, "smc_checkpoint: NULL state or size");
    const size_t need = sizeof(CkptHeader) + ckpt_payload(st, st->stage);
    if (!buf) {
        *size = need;
        return AEM_OK;
    }
    if (*size < need) return fail(AEM_ERR_INVALID_ARG, "smc_checkpoint: buffer smaller than the image");
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = kCkptVersion;
    h.S = st->S;
    h.N = st->N;
    h.M = st->M;
    h.kappa_max = st->d.kappa_max;
    h.lambda_max = st->d.lambda_max;
    h.stage = st->stage;
    h.have_prev = st->have_prev ? 1 : 0;
    h.adaptive = st->d.adaptive ? 1 : 0;
    h.recycle_stages = st->d.recycle_stages;
    h.seed = st->d.seed;
    h.payload_bytes = ckpt_payload(st, st->stage);
    unsigned char *o = (unsigned char *)buf;
    std::memcpy(o, &h, sizeof h);
    o += sizeof h;
    const size_t P = st->P, S = st->S, M = st->M;
    cudaStream_t sm = st->stream;
    int rc;
    if ((rc = particles_d2h(o, st->cur, P, sm)) || (rc = d2h(o, st->gamma, S, sm)) ||
        (rc = d2h(o, st->logz, S * M, sm)) || (rc = d2h(o, st->lang_h, S, sm)))
        return rc;
    unsigned char *counts = o;
    o += 2 * S * kMoves * sizeof(int32_t);
    if (st->d.adaptive && (rc = d2h(o, st->pca_a, S * M, sm))) return rc;
    if (st->d.recycle_stages > 0) {
        const size_t cols = (size_t)st->stage + 1;
        if ((rc = particles_d2h(o, st->hist, (size_t)st->d.recycle_stages * P, sm)) ||
            (rc = hist_rows_d2h(o, st->gamma_hist, S, cols, 1, sm)) ||
            (rc = hist_rows_d2h(o, st->logz_hist, S, cols, M, sm)))
            return rc;
    }
    AEM_CUDA_TRY(cudaStreamSynchronize(sm));
    const size_t nc = S * kMoves;
    for (size_t q = 0; q < nc; ++q) {
        const int32_t a = st->have_prev ? st->acc_prev[q] : 0, b = st->have_prev ? st->nprop_prev[q] : 0;
        std::memcpy(counts + q * sizeof(int32_t), &a, sizeof a);
        std::memcpy(counts + (nc + q) * sizeof(int32_t), &b, sizeof b);
    }
    *size = need;
    return AEM_OK;
}

extern "C" int smc_restore(smc_state *st, const void *buf, size_t size) {
    if (!st || !buf) return fail(AEM_ERR_INVALID_ARG, "smc_restore: NULL state or buffer");
    CkptHeader h{};
    if (size < sizeof h) return fail(AEM_ERR_INVALID_ARG, "smc_restore: buffer shorter than the header");
    std::memcpy(&h, buf, sizeof h);
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != kCkptVersion)
        return fail(AEM_ERR_INVALID_ARG, "smc_restore: not a version-2 sampler checkpoint");
    if (h.S != st->S || h.N != st->N || h.M != st->M || h.kappa_max != st->d.kappa_max ||
        h.lambda_max != st->d.lambda_max)
        return fail(AEM_ERR_INVALID_ARG, "smc_restore: checkpoint sizes differ from this sampler's");
    if (h.adaptive != (st->d.adaptive ? 1 : 0) || h.recycle_stages != st->d.recycle_stages)
        return fail(AEM_ERR_INVALID_ARG, "smc_restore: adaptive proposal or recycling window differs from this sampler's");
    if (h.stage < 0 || (h.recycle_stages > 0 && h.stage >= kMaxRecycleStages))
        return fail(AEM_ERR_INVALID_ARG, "smc_restore: stage counter out of range");
    if (h.payload_bytes != ckpt_payload(st, h.stage) || size < sizeof h + h.payload_bytes)
        return fail(AEM_ERR_INVALID_ARG, "smc_restore: truncated checkpoint");
    const unsigned char *i = (const unsigned char *)buf + sizeof h;
    const size_t P = st->P, S = st->S, M = st->M;
    cudaStream_t sm = st->stream;
    AEM_CUDA_TRY(cudaStreamSynchronize(sm));
    int rc;
    if ((rc = particles_h2d(st->cur, i, P, sm)) || (rc = h2d(st->gamma, i, S, sm)) ||
        (rc = h2d(st->logz, i, S * M, sm)) || (rc = h2d(st->lang_h, i, S, sm)))
        return rc;
    const unsigned char *counts = i;
    i += 2 * S * kMoves * sizeof(int32_t);
    if (st->d.adaptive && (rc = h2d(st->pca_a, i, S * M, sm))) return rc;
    if (st->d.recycle_stages > 0) {
        const size_t cols = (size_t)h.stage + 1;
        if ((rc = particles_h2d(st->hist, i, (size_t)st->d.recycle_stages * P, sm)) ||
            (rc = hist_rows_h2d(st->gamma_hist, i, S, cols, 1, sm)) ||
            (rc = hist_rows_h2d(st->logz_hist, i, S, cols, M, sm)))
            return rc;
    }
    AEM_CUDA_TRY(cudaStreamSynchronize(sm));
    const size_t nc = S * kMoves;
    st->acc_prev.assign(nc, 0);
    st->nprop_prev.assign(nc, 0);
    for (size_t q = 0; q < nc; ++q) {
        std::memcpy(&st->acc_prev[q], counts + q * sizeof(int32_t), sizeof(int32_t));
        std::memcpy(&st->nprop_prev[q], counts + (nc + q) * sizeof(int32_t), sizeof(int32_t));
    }
    st->have_prev = h.have_prev != 0;
    st->stage = h.stage;
    st->gcur_valid = false;
    return AEM_OK;
}

// ----------------------------------------------------- standalone entries
extern "C" size_t aem_smc_workspace_bytes(int n, int n_models) {
    if (n < 0 || n_models < 1) return 0;
    size_t b = 0;
    b += sizeof(int) * 2 * (size_t)n;                 // kappa, lam split of the model ids
    b += sizeof(int) * (size_t)n;                     // perm
    b += sizeof(int) * (size_t)(2 * n_models + 1);    // off, counts
    b += sizeof(double) * (size_t)n;                  // grouped weights
    b += sizeof(unsigned long long) * (size_t)n;      // integer CDF
    b += sizeof(double) + sizeof(int) + 64 * 8;       // gamma, done, alignment slack
    return b;
}

namespace {
struct Workspace {
    int *kappa, *lam, *perm, *off, *counts, *done;
    double *Wg, *gamma;
    unsigned long long *C;
};

Workspace carve(void *base, int n, int M) {
    auto align = [](size_t v) { return (v + 63) & ~(size_t)63; };
    char *p = (char *)base;
    size_t o = 0;
    Workspace w;
    w.Wg = (double *)(p + o);
    o = align(o + sizeof(double) * n);
    w.C = (unsigned long long *)(p + o);
    o = align(o + sizeof(unsigned long long) * n);
    w.gamma = (double *)(p + o);
    o = align(o + sizeof(double));
    w.kappa = (int *)(p + o);
    o = align(o + sizeof(int) * n);
    w.lam = (int *)(p + o);
    o = align(o + sizeof(int) * n);
    w.perm = (int *)(p + o);
    o = align(o + sizeof(int) * n);
    w.off = (int *)(p + o);
    o = align(o + sizeof(int) * (M + 1));
    w.counts = (int *)(p + o);
    o = align(o + sizeof(int) * M);
    w.done = (int *)(p + o);
    return w;
}

int check_standalone(int n, int n_models, const void *work, size_t bytes, const char *name) {
    if (n < 1 || n > AEM_SMC_MAX_PARTICLES || n_models < 1 || n_models > AEM_SMC_MAX_MODELS)
        return fail(AEM_ERR_INVALID_ARG, std::string(name) + ": n or n_models out of range");
    if (!work || bytes < aem_smc_workspace_bytes(n, n_models) || ((uintptr_t)work & 63))
        return fail(AEM_ERR_INVALID_ARG, std::string(name) + ": workspace missing, too small or not 64-byte aligned");
    return AEM_OK;
}
}  // namespace

extern "C" int aem_reweight(const double *ll, const int *model, int n, int n_models, double gamma_prev, double alpha,
                            int bisect_iters, double *dgamma, int *reached_one, double *logz_inc, double *W, void *work,
                            size_t work_bytes, void *stream) {
    int rc = check_standalone(n, n_models, work, work_bytes, "aem_reweight");
    if (rc) return rc;
    if (!ll || !model || !dgamma || !reached_one || !logz_inc || !W || !(alpha > 0 && alpha < 1) ||
        !(gamma_prev >= 0 && gamma_prev < 1) || bisect_iters < 1 || bisect_iters > 200)
        return fail(AEM_ERR_INVALID_ARG, "aem_reweight: NULL pointer or value out of range");
    cudaStream_t s = (cudaStream_t)stream;
    Workspace w = carve(work, n, n_models);
    split_model_kernel<<<blocks_for(n, 256), 256, 0, s>>>(model, n, n_models, w.kappa, w.lam, nullptr, W);
    group_kernel<<<1, kGroupThreads, n, s>>>(w.kappa, w.lam, n, 1, n_models, w.perm, w.off, w.counts);
    AEM_CUDA_TRY(cudaMemcpyAsync(w.gamma, &gamma_prev, sizeof(double), cudaMemcpyHostToDevice, s));
    AEM_CUDA_TRY(cudaMemsetAsync(logz_inc, 0, sizeof(double) * n_models, s));
    const size_t smem = reweight_dense_bytes(n);
    if (smem > 48 * 1024)
        AEM_CUDA_TRY(cudaFuncSetAttribute(reweight_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    reweight_kernel<<<1, kGroupThreads, smem, s>>>(ll, w.perm, w.off, w.counts, n, n_models, alpha, bisect_iters,
                                                   w.gamma, logz_inc, w.Wg, dgamma, reached_one, nullptr, smem > 0);
    scatter_kernel<<<blocks_for(n, 256), 256, 0, s>>>(w.Wg, w.perm, w.off, n_models, W);
    AEM_CUDA_TRY(cudaGetLastError());
    return AEM_OK;
}

extern "C" int aem_resample_systematic(const double *W, const int *model, int n, int n_models,
                                       const unsigned long long *u40, int *ancestor, void *work, size_t work_bytes,
                                       void *stream) {
    int rc = check_standalone(n, n_models, work, work_bytes, "aem_resample_systematic");
    if (rc) return rc;
    if (!W || !model || !u40 || !ancestor) return fail(AEM_ERR_INVALID_ARG, "aem_resample_systematic: NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    Workspace w = carve(work, n, n_models);
    split_model_kernel<<<blocks_for(n, 256), 256, 0, s>>>(model, n, n_models, w.kappa, w.lam, ancestor, nullptr);
    group_kernel<<<1, kGroupThreads, n, s>>>(w.kappa, w.lam, n, 1, n_models, w.perm, w.off, w.counts);
    gather_weights_kernel<<<blocks_for(n, 256), 256, 0, s>>>(W, w.perm, w.off, n_models, w.Wg);
    resample_kernel<<<1, kGroupThreads, 0, s>>>(w.Wg, w.perm, w.off, w.counts, n, n_models, u40, 0ull, 0, nullptr,
                                                w.C, ancestor);
    AEM_CUDA_TRY(cudaGetLastError());
    return AEM_OK;
}

extern "C" int aem_philox4x32(const unsigned int *counters, unsigned int key0, unsigned int key1, unsigned int *out,
                              int n, void *stream) {
    if (n < 0 || (n > 0 && (!counters || !out))) return fail(AEM_ERR_INVALID_ARG, "aem_philox4x32: bad arguments");
    if (n == 0) return AEM_OK;
    philox_kernel<<<blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(counters, key0, key1, out, n);
    AEM_CUDA_TRY(cudaGetLastError());
    return AEM_OK;
}

// ------------------------------------------- resampling without allocation
// Scratch for aem_resample_systematic_noalloc: one fixed array per GPU that
// loads the library, sized for the largest accepted problem and kept until the
// process exits.  Host code must not pass the symbol itself to a kernel (on
// the host it names a stand-in, not device memory); it passes the device
// address obtained below.
namespace {
constexpr size_t kNoAllocScratchBytes = 512 * 1024;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (cudaGetSymbolAddress allocates nothing).
int noalloc_scratch(void **out) {
    int dev = 0;
    AEM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(AEM_ERR_UNSUPPORTED, "aem_resample_systematic_noalloc: device index too large");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "aem_resample_systematic_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return AEM_OK;
}
}  // namespace

extern "C" int aem_resample_systematic_noalloc(const double *W, const int *model, int n, int n_models,
                                                const unsigned long long *u40, int *ancestor, void *stream) {
    if (n < 1 || n > AEM_NOALLOC_MAX_PARTICLES || n_models < 1 || n_models > AEM_NOALLOC_MAX_MODELS)
        return fail(AEM_ERR_INVALID_ARG,
                    "aem_resample_systematic_noalloc: n or n_models exceeds the maximum of the static scratch "
                    "(n <= AEM_NOALLOC_MAX_PARTICLES, n_models <= AEM_NOALLOC_MAX_MODELS)");
    if (aem_smc_workspace_bytes(n, n_models) + 64 > kNoAllocScratchBytes)
        return fail(AEM_ERR_INVALID_ARG, "aem_resample_systematic_noalloc: problem exceeds the static scratch");
    if (!W || !model || !u40 || !ancestor)
        return fail(AEM_ERR_INVALID_ARG, "aem_resample_systematic_noalloc: NULL pointer");
    void *work = nullptr;
    int rc = noalloc_scratch(&work);
    if (rc) return rc;
    // every scratch word the kernels read is written earlier in the same call,
    // so nothing has to be cleared between calls
    return aem_resample_systematic(W, model, n, n_models, u40, ancestor, work, kNoAllocScratchBytes, stream);
}
