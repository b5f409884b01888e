// Host-side system precompute: frequency nodes, the K-point Hankel rule and
// the step-off transform matrix, built in double precision once per system
// and uploaded to the device.  (Section 2: layered-earth Hankel-transform
// forward model; Section 2.3.2: off-time dB/dt gates.)
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "aem_internal.h"

namespace aem {

static thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t err, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(err);
    // a failed runtime call leaves its error as the thread's last error; read
    // it off here so that a later call's cudaGetLastError() does not report it
    // again (a sticky error stays set for the context all the same)
    (void)cudaGetLastError();
    return AEM_ERR_CUDA;
}

namespace {

// Gauss-Legendre rule on [-1, 1]: nodes from the Newton iteration on the
// three-term recurrence, started from Tricomi's asymptotic node estimate.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 1; i <= (n + 1) / 2; ++i) {
        double theta = kPi * (4.0 * i - 1.0) / (4.0 * n + 2.0);
        double z = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * std::cos(theta);
        double dp = 0.0;
        for (int it = 0; it < 60; ++it) {
            double pm1 = 1.0, p = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p - (k - 1.0) * pm1) / k;
                pm1 = p;
                p = pk;
            }
            dp = n * (pm1 - z * p) / (1.0 - z * z);
            double step = p / dp;
            z -= step;
            if (std::fabs(step) < 1e-17) break;
        }
        double pm1 = 1.0, p = z;
        for (int k = 2; k <= n; ++k) {
            double pk = ((2.0 * k - 1.0) * z * p - (k - 1.0) * pm1) / k;
            pm1 = p;
            p = pk;
        }
        dp = n * (pm1 - z * p) / (1.0 - z * z);
        x[i - 1] = -z;
        x[n - i] = z;
        w[i - 1] = w[n - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Integral of u^{-1/2} sin(u) over [X, inf): numerical panels up to X0 = 200
// (when X is smaller) and the asymptotic expansion
//   Int_X^inf u^{-a} e^{iu} du ~ i e^{iX} X^{-a} sum_n (-i)^n (a)_n X^{-n}
// (repeated integration by parts) beyond it.
double sine_tail_half(double X, const std::vector<double> &gx, const std::vector<double> &gw) {
    double acc = 0.0;
    double X0 = X;
    if (X < 200.0) {
        X0 = 200.0;
        int panels = (int)std::ceil((X0 - X) / 0.5);
        double width = (X0 - X) / panels;
        for (int p = 0; p < panels; ++p) {
            double lo = X + p * width, c = lo + 0.5 * width, r = 0.5 * width;
            for (size_t i = 0; i < gx.size(); ++i) {
                double u = c + r * gx[i];
                acc += r * gw[i] * std::sin(u) / std::sqrt(u);
            }
        }
    }
    std::complex<double> sum(0.0, 0.0), term(1.0, 0.0);
    const std::complex<double> mi(0.0, -1.0);
    double a = 0.5;
    for (int n = 0; n < 40; ++n) {
        sum += term;
        std::complex<double> next = term * mi * ((a + n) / X0);
        if (std::abs(next) > std::abs(term) || std::abs(next) < 1e-20) break;
        term = next;
    }
    std::complex<double> I = std::complex<double>(0.0, 1.0) * std::exp(std::complex<double>(0.0, X0)) *
                             std::pow(X0, -a) * sum;
    return acc + I.imag();
}

// sin(w t) for large w t: the product is formed exactly as hi + lo with an
// FMA, the nearest multiple of 2 pi is removed with 2 pi split into its double
// value and the residual 2 pi - fl(2 pi), and sin is taken of the reduced
// argument.  This keeps the phase error near 1e-16 rad instead of w t * 1e-16.
double sin_wt(double w, double t) {
    const double two_pi_hi = 6.283185307179586232, two_pi_lo = 2.4492935982947064e-16;
    double hi = w * t;
    if (std::fabs(hi) < 64.0) return std::sin(hi);
    double lo = std::fma(w, t, -hi);
    double k = std::nearbyint(hi / two_pi_hi);
    double r = std::fma(-k, two_pi_hi, hi);
    r = std::fma(-k, two_pi_lo, r) + lo;
    return std::sin(r);
}

}  // namespace

int build_tables(const aem_system_desc *d, SystemTables *t) {
    if (!d) return fail(AEM_ERR_INVALID_ARG, "aem_system_create: desc is NULL");
    if (!(d->loop_radius > 0) || !(d->height > 0) || !(d->current > 0))
        return fail(AEM_ERR_INVALID_ARG, "aem_system_create: loop_radius, height and current must be > 0");
    if (d->n_freq < 2 || d->n_freq > AEM_MAX_FREQ)
        return fail(AEM_ERR_INVALID_ARG, "aem_system_create: n_freq out of range");
    if (d->n_gates < 1 || d->n_gates > AEM_MAX_GATES || !d->gate_times)
        return fail(AEM_ERR_INVALID_ARG, "aem_system_create: n_gates out of range or gate_times NULL");
    if (d->n_hankel < 8 || d->n_hankel > AEM_MAX_HANKEL)
        return fail(AEM_ERR_INVALID_ARG, "aem_system_create: n_hankel out of range");
    if (!(d->f_min_hz > 0) || !(d->f_max_hz > d->f_min_hz))
        return fail(AEM_ERR_INVALID_ARG, "aem_system_create: need 0 < f_min_hz < f_max_hz");
    if (d->cc_form != AEM_CC_PAPER && d->cc_form != AEM_CC_PELTON && d->cc_form != AEM_CC_LITERAL)
        return fail(AEM_ERR_INVALID_ARG, "aem_system_create: unknown cc_form");
    for (int g = 0; g < d->n_gates; ++g) {
        if (!(d->gate_times[g] > 0) || (g > 0 && !(d->gate_times[g] > d->gate_times[g - 1])))
            return fail(AEM_ERR_INVALID_ARG, "aem_system_create: gate_times must be positive and ascending");
    }
    const int F = d->n_freq, G = d->n_gates, K = d->n_hankel;
    t->a = d->loop_radius;
    t->h = d->height;
    t->current = d->current;
    t->F = F;
    t->G = G;
    t->K = K;
    t->cc_form = d->cc_form;
    t->freqs.resize(F);
    t->omega.resize(F);
    const double lf0 = std::log(d->f_min_hz), lf1 = std::log(d->f_max_hz);
    for (int f = 0; f < F; ++f) {
        t->freqs[f] = std::exp(lf0 + (lf1 - lf0) * f / (F - 1));
        t->omega[f] = 2.0 * kPi * t->freqs[f];
    }
    t->times.assign(d->gate_times, d->gate_times + G);

    // Hankel rule: trapezoid in x = ln(lambda) on [ln(1e-5/(2h+a)), ln(20/h)]
    // with the geometry folded into the weights.
    t->lam.resize(K);
    t->hw.resize(K);
    const double a = t->a, h = t->h;
    const double x0 = std::log(1e-5 / (2.0 * h + a)), x1 = std::log(20.0 / h);
    const double dx = (x1 - x0) / (K - 1);
    for (int k = 0; k < K; ++k) {
        double lam = std::exp(x0 + dx * k);
        double wt = dx * ((k == 0 || k == K - 1) ? 0.5 : 1.0);
        t->lam[k] = lam;
        t->hw[k] = wt * 0.5 * t->current * a * lam * lam * std::cyl_bessel_j(1.0, lam * a) * std::exp(-2.0 * lam * h);
    }

    // Clamped cubic spline in x = ln(w): second derivatives M for every unit
    // data vector by the tridiagonal (Thomas) solve.
    std::vector<double> x(F), hh(F - 1);
    for (int f = 0; f < F; ++f) x[f] = std::log(t->omega[f]);
    for (int j = 0; j < F - 1; ++j) hh[j] = x[j + 1] - x[j];
    std::vector<double> sub(F, 0.0), diag(F, 0.0), sup(F, 0.0);
    diag[0] = hh[0] / 3.0;
    sup[0] = hh[0] / 6.0;
    for (int i = 1; i < F - 1; ++i) {
        sub[i] = hh[i - 1] / 6.0;
        diag[i] = (hh[i - 1] + hh[i]) / 3.0;
        sup[i] = hh[i] / 6.0;
    }
    sub[F - 1] = hh[F - 2] / 6.0;
    diag[F - 1] = hh[F - 2] / 3.0;
    // M2[f][i]: second derivative at node i for data e_f
    std::vector<double> M2((size_t)F * F);
    for (int f = 0; f < F; ++f) {
        std::vector<double> rhs(F, 0.0);
        auto y = [&](int i) { return i == f ? 1.0 : 0.0; };
        rhs[0] = (y(1) - y(0)) / hh[0] - y(0);
        for (int i = 1; i < F - 1; ++i) rhs[i] = (y(i + 1) - y(i)) / hh[i] - (y(i) - y(i - 1)) / hh[i - 1];
        rhs[F - 1] = -0.5 * y(F - 1) - (y(F - 1) - y(F - 2)) / hh[F - 2];
        std::vector<double> cp(F), dp(F);
        cp[0] = sup[0] / diag[0];
        dp[0] = rhs[0] / diag[0];
        for (int i = 1; i < F; ++i) {
            double den = diag[i] - sub[i] * cp[i - 1];
            cp[i] = (i < F - 1) ? sup[i] / den : 0.0;
            dp[i] = (rhs[i] - sub[i] * dp[i - 1]) / den;
        }
        std::vector<double> sol(F);
        sol[F - 1] = dp[F - 1];
        for (int i = F - 2; i >= 0; --i) sol[i] = dp[i] - cp[i] * sol[i + 1];
        for (int i = 0; i < F; ++i) M2[(size_t)f * F + i] = sol[i];
    }

    std::vector<double> gx, gw;
    gauss_legendre(16, gx, gw);
    t->T.assign((size_t)G * F, 0.0);
    std::vector<double> row(F);
    for (int g = 0; g < G; ++g) {
        const double tg = t->times[g];
        std::fill(row.begin(), row.end(), 0.0);
        for (int j = 0; j < F - 1; ++j) {
            const double wlo = t->omega[j], whi = t->omega[j + 1];
            // moments Int (x - x_j)^m sin(w t) dw over the piece, composite
            // 16-point Gauss-Legendre on panels of <= pi/4 phase and <= 0.025 in x
            int by_phase = (int)std::ceil((whi - wlo) * tg / (0.25 * kPi));
            int by_x = (int)std::ceil(hh[j] / 0.025);
            double mom[4] = {0, 0, 0, 0};
            if (by_phase > by_x) {
                double width = (whi - wlo) / by_phase;
                for (int p = 0; p < by_phase; ++p) {
                    double c = wlo + (p + 0.5) * width, r = 0.5 * width;
                    for (int i = 0; i < 16; ++i) {
                        double w = c + r * gx[i];
                        double dd = std::log(w) - x[j];
                        double s = r * gw[i] * sin_wt(w, tg);
                        mom[0] += s;
                        mom[1] += s * dd;
                        mom[2] += s * dd * dd;
                        mom[3] += s * dd * dd * dd;
                    }
                }
            } else {
                double width = hh[j] / by_x;
                for (int p = 0; p < by_x; ++p) {
                    double c = x[j] + (p + 0.5) * width, r = 0.5 * width;
                    for (int i = 0; i < 16; ++i) {
                        double xx = c + r * gx[i];
                        double w = std::exp(xx);
                        double dd = xx - x[j];
                        double s = r * gw[i] * w * sin_wt(w, tg);  // dw = w dx
                        mom[0] += s;
                        mom[1] += s * dd;
                        mom[2] += s * dd * dd;
                        mom[3] += s * dd * dd * dd;
                    }
                }
            }
            // spline piece j: S = y_j + b d + (M_j/2) d^2 + (M_{j+1}-M_j)/(6 h) d^3
            for (int f = 0; f < F; ++f) {
                double yj = (f == j) ? 1.0 : 0.0, yj1 = (f == j + 1) ? 1.0 : 0.0;
                double Mj = M2[(size_t)f * F + j], Mj1 = M2[(size_t)f * F + j + 1];
                double b = (yj1 - yj) / hh[j] - hh[j] * (2.0 * Mj + Mj1) / 6.0;
                row[f] += yj * mom[0] + b * mom[1] + 0.5 * Mj * mom[2] + (Mj1 - Mj) / (6.0 * hh[j]) * mom[3];
            }
        }
        // tail below the first node: y_0 w / w_0, exact integral
        {
            double w0 = t->omega[0];
            row[0] += (std::sin(w0 * tg) - w0 * tg * std::cos(w0 * tg)) / (w0 * tg * tg);
        }
        // tail above the last node: y_{F-1} (w / w_F)^{-1/2}
        {
            double wF = t->omega[F - 1];
            row[F - 1] += std::sqrt(wF / tg) * sine_tail_half(wF * tg, gx, gw);
        }
        for (int f = 0; f < F; ++f) t->T[(size_t)g * F + f] = -(2.0 * kMu0 / kPi) * row[f];
    }
    return AEM_OK;
}

}  // namespace aem

using namespace aem;

extern "C" const char *aem_last_error(void) { return g_last_error.c_str(); }

template <class T>
static int upload(T **dst, const std::vector<double> &src) {
    std::vector<T> tmp(src.begin(), src.end());
    AEM_CUDA_TRY(cudaMalloc((void **)dst, tmp.size() * sizeof(T)));
    AEM_CUDA_TRY(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
    return AEM_OK;
}

extern "C" int aem_system_create(const aem_system_desc *desc, aem_system **out) {
    if (!out) return fail(AEM_ERR_INVALID_ARG, "aem_system_create: out is NULL");
    *out = nullptr;
    aem_system *s = new aem_system();
    int rc = build_tables(desc, &s->host);
    if (rc != AEM_OK) {
        delete s;
        return rc;
    }
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "cudaGetDevice");
    }
    e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "cudaDeviceGetAttribute");
    }
    const SystemTables &h = s->host;
    if ((rc = upload(&s->d_omega_f, h.omega)) || (rc = upload(&s->d_lam_f, h.lam)) || (rc = upload(&s->d_hw_f, h.hw)) ||
        (rc = upload(&s->d_T_f, h.T)) || (rc = upload(&s->d_omega_d, h.omega)) || (rc = upload(&s->d_lam_d, h.lam)) ||
        (rc = upload(&s->d_hw_d, h.hw)) || (rc = upload(&s->d_T_d, h.T))) {
        aem_system_destroy(s);
        return rc;
    }
    e = cudaMalloc((void **)&s->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(s->d_status, 0, sizeof(int));
    if (e != cudaSuccess) {
        aem_system_destroy(s);
        return cuda_fail(e, "aem_system_create: status word");
    }
    *out = s;
    return AEM_OK;
}

extern "C" int aem_system_destroy(aem_system *s) {
    if (!s) return AEM_OK;
    void *ptrs[] = {s->d_omega_f, s->d_lam_f, s->d_hw_f, s->d_T_f,
                    s->d_omega_d, s->d_lam_d, s->d_hw_d, s->d_T_d, s->d_status};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete s;
    return AEM_OK;
}

extern "C" int aem_system_tables(const aem_system *s, double *freqs, double *lam, double *hw, double *T) {
    if (!s) return fail(AEM_ERR_INVALID_ARG, "aem_system_tables: sys is NULL");
    const SystemTables &h = s->host;
    if (freqs) std::memcpy(freqs, h.freqs.data(), sizeof(double) * h.F);
    if (lam) std::memcpy(lam, h.lam.data(), sizeof(double) * h.K);
    if (hw) std::memcpy(hw, h.hw.data(), sizeof(double) * h.K);
    if (T) std::memcpy(T, h.T.data(), sizeof(double) * h.G * h.F);
    return AEM_OK;
}
