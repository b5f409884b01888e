// FP64 CPU oracle for the airborne-EM forward model of Davies et al.,
// "Bayesian detectability of induced polarisation in airborne EM data using
// reversible jump sequential Monte Carlo" (arXiv 2109.00661).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
// its Python binding) may link, import or call this file.  It shares no code
// with the GPU path: its Hankel integrals are adaptive quadrature between the
// zeros of J1 (with Wynn epsilon acceleration), its transform matrix is built
// by adaptive quadrature per oscillation, and every formula below is written
// out plainly, in double precision, without blocking, fusion or reordering.
//
// Physics (the paper cites Ward & Hohmann 1988 for the layered-earth model in
// Section 2 but prints no equations; the statements below are the standard
// quasi-static TE formulation, with time dependence exp(+i w t)):
//   * Cole-Cole conductivity (Section 2):  sigma(w) = s_inf (1 - m / (1 + (i w tau)^c)).
//   * Layer wavenumber u_n = sqrt(lambda^2 + i w mu0 sigma_n), Re u_n > 0.
//   * Interface reflection r_{n-1,n} = (u_{n-1}-u_n)/(u_{n-1}+u_n), written as
//     i w mu0 (sigma_{n-1}-sigma_n)/(u_{n-1}+u_n)^2 (air: sigma_0 = 0, u_0 = lambda).
//   * Bottom-up recursion R_{n-1} = (r + R_n e^{-2 u_n h_n})/(1 + r R_n e^{-2 u_n h_n}).
//   * Secondary field at the centre of a loop of radius a carrying I, Tx/Rx at
//     height h: Hz_s(w) = (I a / 2) Int_0^inf R_0(lambda, w) e^{-2 lambda h} lambda J1(lambda a) dlambda.
//   * Step-off response (gates, Section 2.3.2): y(t) = -dBz/dt
//     = -(2 mu0 / pi) Int_0^inf Im Hz_s(w) sin(w t) dw, with Im Hz_s interpolated
//     by a cubic spline in ln w through the F frequency nodes, clamped so that
//     it joins a tail proportional to w below the first node and to w^(-1/2)
//     above the last node.
//   * Gaussian log-likelihood (Section 2.3.2): variance eps_an^2 + (eps_mn * y_model)^2.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

typedef std::complex<double> cd;

static const double PI = 3.14159265358979323846;
static const double MU0 = 4e-7 * PI;

// ---------------------------------------------------------------------------
// Gauss-Legendre nodes on [-1, 1] by Newton iteration on P_n (no tables).
// ---------------------------------------------------------------------------
struct GaussLegendre {
    int n;
    std::vector<double> x, w;
    explicit GaussLegendre(int n_) : n(n_), x(n_), w(n_) {
        for (int i = 0; i < n; ++i) {
            double z = std::cos(PI * (i + 0.75) / (n + 0.5));
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = 0.0;
                for (int k = 1; k <= n; ++k) {
                    double p2 = p1;
                    p1 = p0;
                    p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
                }
                double dp = n * (z * p0 - p1) / (z * z - 1.0);
                double dz = p0 / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-16) {
                    // recompute derivative at the converged node for the weight
                    p0 = 1.0; p1 = 0.0;
                    for (int k = 1; k <= n; ++k) {
                        double p2 = p1;
                        p1 = p0;
                        p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
                    }
                    dp = n * (z * p0 - p1) / (z * z - 1.0);
                    break;
                }
            }
            x[i] = z;
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; ++k) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            double dp = n * (z * p0 - p1) / (z * z - 1.0);
            w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};

static const GaussLegendre &gl10() {
    static GaussLegendre g(10);
    return g;
}

// Adaptive Gauss-Legendre: compare one 10-point panel with two half panels.
template <class V, class Fn>
static V gl_panel(const Fn &f, double lo, double hi) {
    const GaussLegendre &g = gl10();
    double c = 0.5 * (lo + hi), r = 0.5 * (hi - lo);
    V s = V();
    for (int i = 0; i < g.n; ++i) s += g.w[i] * f(c + r * g.x[i]);
    return s * r;
}

static double mag(double v) { return std::fabs(v); }
static double mag(const cd &v) { return std::abs(v); }
struct Moments4;
static double mag(const Moments4 &v);

template <class V, class Fn>
static V adapt(const Fn &f, double lo, double hi, V whole, double rtol, double atol, int depth) {
    double mid = 0.5 * (lo + hi);
    V left = gl_panel<V>(f, lo, mid), right = gl_panel<V>(f, mid, hi);
    V both = left + right;
    if (depth <= 0 || mag(both - whole) <= std::max(rtol * mag(both), atol)) return both;
    return adapt<V>(f, lo, mid, left, rtol, atol, depth - 1) +
           adapt<V>(f, mid, hi, right, rtol, atol, depth - 1);
}

// The depth cap bounds the work when rounding noise in the integrand (for
// instance sin(w t) at w t ~ 1e5) sits near the requested tolerance.
template <class V, class Fn>
static V integrate(const Fn &f, double lo, double hi, double rtol, double atol, int max_depth = 20) {
    V whole = gl_panel<V>(f, lo, hi);
    return adapt<V>(f, lo, hi, whole, rtol, atol, max_depth);
}

// Wynn epsilon extrapolation of a sequence of partial sums (returns the best
// estimate from the last complete even column).
template <class V>
static V wynn_epsilon(const std::vector<V> &s) {
    size_t n = s.size();
    if (n < 3) return s.back();
    std::vector<V> e0(n + 1, V()), e1(s.begin(), s.end());
    // e_{-1} = 0, e_0 = s.  Column k+1: e_{k+1}(i) = e_{k-1}(i+1) + 1/(e_k(i+1)-e_k(i))
    std::vector<V> prev = e0, cur = e1;
    V best = s.back();
    for (size_t k = 1; k < n; ++k) {
        std::vector<V> next(n - k);
        bool ok = true;
        for (size_t i = 0; i + 1 < cur.size(); ++i) {
            V d = cur[i + 1] - cur[i];
            if (mag(d) == 0.0) { ok = false; break; }
            next[i] = prev[i + 1] + V(1.0) / d;
        }
        if (!ok) break;
        prev = cur;
        cur = next;
        if (k % 2 == 0 && !cur.empty()) best = cur.back();
    }
    return best;
}

// ---------------------------------------------------------------------------
// Cole-Cole complex conductivity (Section 2).
// form 0: paper's form   s_inf * (1 - m / (1 + (i w tau)^c))       (sig = s_inf)
// form 1: Pelton (1978)  1 / rho,  rho = (1/s0)(1 - m (1 - 1/(1 + (i w tau)^c)))  (sig = s0)
// form 2: the expression s0 (1 - m (1 - 1/(1 + (i w tau)^c))) taken as a conductivity
// ---------------------------------------------------------------------------
static cd colecole(int form, double sig, double m, double tau, double c, double w) {
    if (m == 0.0) return cd(sig, 0.0);
    cd iwt_c = std::pow(w * tau, c) * std::exp(cd(0.0, 0.5 * PI * c));
    cd one(1.0, 0.0);
    if (form == 0) return sig * (one - m / (one + iwt_c));
    if (form == 2) return sig * (one - m * (one - one / (one + iwt_c)));
    return sig / (one - m * (one - one / (one + iwt_c)));
}

// Principal square root with Re >= 0.
static cd csqrt_p(cd z) {
    cd r = std::sqrt(z);
    if (r.real() < 0) r = -r;
    return r;
}

// R_0(lambda, w) by the reflection-coefficient recursion.
// s[n] = i w mu0 sigma_n for layers n = 0..L-1 (top to bottom, last is the half-space).
static cd r0_reflection(int L, const cd *s, const double *thick, double lam) {
    std::vector<cd> u(L);
    for (int n = 0; n < L; ++n) u[n] = csqrt_p(cd(lam * lam, 0.0) + s[n]);
    auto refl = [&](int n) -> cd {  // reflection at the top of layer n (medium above: n-1 or air)
        cd s_above = (n == 0) ? cd(0.0, 0.0) : s[n - 1];
        cd u_above = (n == 0) ? cd(lam, 0.0) : u[n - 1];
        cd sum = u_above + u[n];
        return (s_above - s[n]) / (sum * sum);
    };
    cd R = refl(L - 1);
    for (int n = L - 2; n >= 0; --n) {
        cd E = std::exp(-2.0 * u[n] * thick[n]);
        cd r = refl(n);
        R = (r + R * E) / (1.0 + r * R * E);
    }
    return R;
}

// R_0(lambda, w) by the impedance (admittance) recursion with tanh, as an
// independent cross-check of r0_reflection.  All admittances share the factor
// 1/(i w mu0), so the wavenumbers u are propagated directly.
static cd r0_admittance(int L, const cd *s, const double *thick, double lam) {
    std::vector<cd> u(L);
    for (int n = 0; n < L; ++n) u[n] = csqrt_p(cd(lam * lam, 0.0) + s[n]);
    cd Y = u[L - 1];
    for (int n = L - 2; n >= 0; --n) {
        cd t = std::tanh(u[n] * thick[n]);
        Y = u[n] * (Y + u[n] * t) / (u[n] + Y * t);
    }
    return (cd(lam, 0.0) - Y) / (cd(lam, 0.0) + Y);
}

// Zeros of J1 (Newton from the McMahon asymptotic guess), cached.
static double j1_zero(int m) {
    static std::vector<double> z;
    if ((int)z.size() >= m) return z[m - 1];
    for (int k = (int)z.size() + 1; k <= m; ++k) {
        double beta = (k + 0.25) * PI;
        double x = beta - 3.0 / (8.0 * beta);
        for (int it = 0; it < 50; ++it) {
            double j1 = std::cyl_bessel_j(1.0, x);
            double dj = std::cyl_bessel_j(0.0, x) - j1 / x;
            double dx = j1 / dj;
            x -= dx;
            if (std::fabs(dx) < 1e-15 * x) break;
        }
        z.push_back(x);
    }
    return z[m - 1];
}

// Secondary Hz by adaptive quadrature: the first J1 lobe is split into
// geometric panels so that structure at small lambda is resolved; then one
// panel per half-oscillation of J1(lambda a) with Wynn extrapolation.
static cd hz_quadrature(int L, const cd *s, const double *thick, double a, double h, double current,
                        int method, double rtol) {
    auto f = [&](double lam) -> cd {
        if (lam <= 0.0) return cd(0.0, 0.0);
        cd R = method == 0 ? r0_reflection(L, s, thick, lam) : r0_admittance(L, s, thick, lam);
        return R * std::exp(-2.0 * lam * h) * lam * std::cyl_bessel_j(1.0, lam * a);
    };
    double atol = 1e-300;
    double z1 = j1_zero(1) / a;
    cd total(0.0, 0.0);
    double lo = 0.0;
    for (int e = -12; e <= 0; ++e) {
        double hi = z1 * std::pow(10.0, (double)e);
        if (e == 0) hi = z1;
        total += integrate<cd>(f, lo, hi, rtol, atol);
        lo = hi;
    }
    std::vector<cd> partial;
    partial.push_back(total);
    int small_run = 0;
    for (int mz = 1; mz < 4000; ++mz) {
        double a0 = j1_zero(mz) / a, a1 = j1_zero(mz + 1) / a;
        cd seg = integrate<cd>(f, a0, a1, rtol, atol);
        total += seg;
        partial.push_back(total);
        if (std::abs(seg) <= 1e-17 * std::abs(total)) {
            if (++small_run >= 3) return total * (0.5 * current * a);
        } else {
            small_run = 0;
        }
        if (partial.size() >= 40 && h == 0.0 && mz % 20 == 0) {
            // slowly converging alternating tail (h = 0): extrapolate and stop
            // once two extrapolations agree
            cd e1 = wynn_epsilon(std::vector<cd>(partial.end() - 30, partial.end()));
            cd e2 = wynn_epsilon(std::vector<cd>(partial.end() - 31, partial.end() - 1));
            if (std::abs(e1 - e2) <= 1e-12 * std::abs(e1)) return e1 * (0.5 * current * a);
        }
    }
    if (h == 0.0) return wynn_epsilon(std::vector<cd>(partial.end() - 30, partial.end())) * (0.5 * current * a);
    return total * (0.5 * current * a);
}

// The fixed K-point Hankel rule (log-spaced trapezoid in ln lambda), built
// here from its definition: lambda_k = exp(x0 + k dx), x0 = ln(1e-5/(2h+a)),
// x_{K-1} = ln(20/h), weight dx (halved at both ends) times the kernel
// (I a / 2) lambda^2 J1(lambda a) e^{-2 lambda h}.
static void hankel_rule(int K, double a, double h, double current, std::vector<double> &lam,
                        std::vector<double> &c) {
    lam.resize(K);
    c.resize(K);
    double x0 = std::log(1e-5 / (2.0 * h + a)), x1 = std::log(20.0 / h);
    double dx = (x1 - x0) / (K - 1);
    for (int k = 0; k < K; ++k) {
        double l = std::exp(x0 + k * dx);
        double wk = (k == 0 || k == K - 1) ? 0.5 * dx : dx;
        lam[k] = l;
        c[k] = wk * 0.5 * current * a * l * l * std::cyl_bessel_j(1.0, l * a) * std::exp(-2.0 * l * h);
    }
}

// ---------------------------------------------------------------------------
// Decoupled-profile merge (Section 2.1, Fig. 2 caption): union of the
// conductive and chargeable interfaces; each merged layer takes sigma from the
// conductive profile and m from the chargeable profile at its depth.
// Interfaces are depths of the top of the layer whose property follows.
// ---------------------------------------------------------------------------
extern "C" int orc_merge(int kappa, const double *zc, const double *logsig /*kappa+1*/, int lam_n,
                         const double *zm, const double *mval /*lam_n (layers below each zm)*/,
                         double *thick_out, double *logsig_out, double *m_out) {
    std::vector<double> z;
    for (int i = 0; i < kappa; ++i) z.push_back(zc[i]);
    for (int j = 0; j < lam_n; ++j) z.push_back(zm[j]);
    std::sort(z.begin(), z.end());
    int L = (int)z.size() + 1;
    for (int n = 0; n < L; ++n) {
        double top = (n == 0) ? 0.0 : z[n - 1];
        double bottom = (n == L - 1) ? top : z[n];
        // property at the layer's top depth: the last interface at or above it
        int ic = 0;
        for (int i = 0; i < kappa; ++i)
            if (zc[i] <= top && n > 0) ic = i + 1;
        int jm = 0;
        for (int j = 0; j < lam_n; ++j)
            if (zm[j] <= top && n > 0) jm = j + 1;
        logsig_out[n] = logsig[ic];
        m_out[n] = (jm == 0) ? 0.0 : mval[jm - 1];
        thick_out[n] = bottom - top;
    }
    return L;
}

// ---------------------------------------------------------------------------
// Transform matrix (Section 2.3.2 gates; step-off reading).  T[g*F + f] maps
// Im Hz_s at node f to y(t_g) = -dBz/dt.  Cubic spline in x = ln w, clamped:
// S'(x_1) = y_1 (tail y_1 w / w_1), S'(x_F) = -y_F / 2 (tail y_F (w/w_F)^-1/2).
// ---------------------------------------------------------------------------
static void spline_basis(int F, const double *x, std::vector<double> &C /*(F-1)*4*F*/) {
    // Unknowns: second derivatives M_0..M_{F-1} (in x) for each unit data vector.
    std::vector<double> A(F * F, 0.0), B(F * F, 0.0);
    std::vector<double> hh(F - 1);
    for (int j = 0; j + 1 < F; ++j) hh[j] = x[j + 1] - x[j];
    for (int i = 1; i + 1 < F; ++i) {
        A[i * F + i - 1] = hh[i - 1] / 6.0;
        A[i * F + i] = (hh[i - 1] + hh[i]) / 3.0;
        A[i * F + i + 1] = hh[i] / 6.0;
        B[i * F + i + 1] += 1.0 / hh[i];
        B[i * F + i] -= 1.0 / hh[i] + 1.0 / hh[i - 1];
        B[i * F + i - 1] += 1.0 / hh[i - 1];
    }
    // S'(x_0) = (y1-y0)/h0 - h0 (2 M0 + M1)/6 = y0
    A[0] = hh[0] / 3.0;
    A[1] = hh[0] / 6.0;
    B[1] += 1.0 / hh[0];
    B[0] += -1.0 / hh[0] - 1.0;
    // S'(x_{F-1}) = (y_{F-1}-y_{F-2})/h + h (M_{F-2} + 2 M_{F-1})/6 = -y_{F-1}/2
    int l = F - 1;
    A[l * F + l] = hh[l - 1] / 3.0;
    A[l * F + l - 1] = hh[l - 1] / 6.0;
    B[l * F + l] += -0.5 - 1.0 / hh[l - 1];
    B[l * F + l - 1] += 1.0 / hh[l - 1];
    // Solve A M = B by Gaussian elimination with partial pivoting (dense).
    std::vector<double> Mm = B;
    std::vector<double> Aw = A;
    for (int col = 0; col < F; ++col) {
        int piv = col;
        for (int r = col + 1; r < F; ++r)
            if (std::fabs(Aw[r * F + col]) > std::fabs(Aw[piv * F + col])) piv = r;
        if (piv != col) {
            for (int k = 0; k < F; ++k) {
                std::swap(Aw[col * F + k], Aw[piv * F + k]);
                std::swap(Mm[col * F + k], Mm[piv * F + k]);
            }
        }
        for (int r = 0; r < F; ++r) {
            if (r == col) continue;
            double fac = Aw[r * F + col] / Aw[col * F + col];
            if (fac == 0.0) continue;
            for (int k = 0; k < F; ++k) {
                Aw[r * F + k] -= fac * Aw[col * F + k];
                Mm[r * F + k] -= fac * Mm[col * F + k];
            }
        }
    }
    for (int r = 0; r < F; ++r) {
        double d = Aw[r * F + r];
        for (int k = 0; k < F; ++k) Mm[r * F + k] /= d;
    }
    // Piece j: S(x) = c0 + c1 d + c2 d^2 + c3 d^3, d = x - x_j.
    C.assign((size_t)(F - 1) * 4 * F, 0.0);
    for (int j = 0; j + 1 < F; ++j) {
        double hj = hh[j];
        for (int f = 0; f < F; ++f) {
            double yj = (f == j) ? 1.0 : 0.0, yj1 = (f == j + 1) ? 1.0 : 0.0;
            double Mj = Mm[j * F + f], Mj1 = Mm[(j + 1) * F + f];
            C[((size_t)j * 4 + 0) * F + f] = yj;
            C[((size_t)j * 4 + 1) * F + f] = (yj1 - yj) / hj - hj * (2.0 * Mj + Mj1) / 6.0;
            C[((size_t)j * 4 + 2) * F + f] = Mj / 2.0;
            C[((size_t)j * 4 + 3) * F + f] = (Mj1 - Mj) / (6.0 * hj);
        }
    }
}

struct Moments4 {
    double m[4];
    Moments4() { m[0] = m[1] = m[2] = m[3] = 0.0; }
    Moments4 &operator+=(const Moments4 &o) { for (int i = 0; i < 4; ++i) m[i] += o.m[i]; return *this; }
    Moments4 operator+(const Moments4 &o) const { Moments4 r = *this; r += o; return r; }
    Moments4 operator-(const Moments4 &o) const { Moments4 r; for (int i = 0; i < 4; ++i) r.m[i] = m[i] - o.m[i]; return r; }
    Moments4 operator*(double s) const { Moments4 r; for (int i = 0; i < 4; ++i) r.m[i] = m[i] * s; return r; }
    friend Moments4 operator*(double s, const Moments4 &a) { return a * s; }
};
static double mag(const Moments4 &a) {
    double s = 0.0;
    for (int i = 0; i < 4; ++i) s = std::max(s, std::fabs(a.m[i]));
    return s;
}

// sin(w t) with the phase reduced modulo 2 pi before rounding: w t can reach
// 1e6 rad, where rounding w t to double alone would cost ~1e-10 rad.  The
// product is split exactly (w t = p + e with an FMA) and p is reduced by the
// nearest multiple of 2 pi using a two-term split of 2 pi.
static double sin_of_product(double w, double t) {
    double p = w * t;
    if (std::fabs(p) < 100.0) return std::sin(p);
    double e = std::fma(w, t, -p);
    const double c1 = 6.283185307179586232;    // fl(2 pi)
    const double c2 = 2.4492935982947064e-16;  // 2 pi - fl(2 pi)
    double n = std::floor(p / c1 + 0.5);
    double red = std::fma(-n, c1, p);
    red = std::fma(-n, c2, red);
    return std::sin(red + e);
}

extern "C" void orc_tmatrix(int F, const double *freqs, int G, const double *times, double *T) {
    std::vector<double> w(F), x(F);
    for (int f = 0; f < F; ++f) {
        w[f] = 2.0 * PI * freqs[f];
        x[f] = std::log(w[f]);
    }
    std::vector<double> C;
    spline_basis(F, x.data(), C);
    for (int g = 0; g < G; ++g) {
        double t = times[g];
        std::vector<double> row(F, 0.0);
        for (int j = 0; j + 1 < F; ++j) {
            auto fm = [&](double om) -> Moments4 {
                Moments4 r;
                double d = std::log(om) - x[j], s = sin_of_product(om, t);
                r.m[0] = s;
                r.m[1] = s * d;
                r.m[2] = s * d * d;
                r.m[3] = s * d * d * d;
                return r;
            };
            // panels of at most a quarter period of sin(w t), and at most
            // 0.05 in ln w, each integrated adaptively
            double lo = w[j], hi = w[j + 1];
            int nph = (int)std::ceil((hi - lo) * t / (0.5 * PI));
            int nx = (int)std::ceil((x[j + 1] - x[j]) / 0.05);
            Moments4 acc;
            if (nph > nx) {
                for (int p = 0; p < nph; ++p) {
                    double a0 = lo + (hi - lo) * p / nph, a1 = lo + (hi - lo) * (p + 1) / nph;
                    acc += integrate<Moments4>(fm, a0, a1, 1e-10, 1e-300, 8);
                }
            } else {
                for (int p = 0; p < nx; ++p) {
                    double a0 = std::exp(x[j] + (x[j + 1] - x[j]) * p / nx);
                    double a1 = std::exp(x[j] + (x[j + 1] - x[j]) * (p + 1) / nx);
                    acc += integrate<Moments4>(fm, a0, a1, 1e-10, 1e-300, 8);
                }
            }
            for (int mm = 0; mm < 4; ++mm)
                for (int f = 0; f < F; ++f) row[f] += acc.m[mm] * C[((size_t)j * 4 + mm) * F + f];
        }
        // low tail: y_0 * (w / w_0) on [0, w_0]
        {
            auto fl = [&](double om) -> double { return (om / w[0]) * std::sin(om * t); };
            row[0] += integrate<double>(fl, 0.0, w[0], 1e-12, 1e-300, 8);
        }
        // high tail: y_{F-1} * (w / w_{F-1})^(-1/2) on [w_{F-1}, inf): half-period
        // panels between zeros of sin(w t), partial sums extrapolated by Wynn epsilon
        {
            double wF = w[F - 1];
            auto fh = [&](double om) -> double { return std::sqrt(wF / om) * sin_of_product(om, t); };
            double first_zero = std::ceil(wF * t / PI) * PI / t;
            if (first_zero <= wF) first_zero += PI / t;
            double total = integrate<double>(fh, wF, first_zero, 1e-10, 1e-300, 8);
            std::vector<double> partial;
            partial.push_back(total);
            double z = first_zero;
            for (int k = 0; k < 60; ++k) {
                total += integrate<double>(fh, z, z + PI / t, 1e-10, 1e-300, 8);
                z += PI / t;
                partial.push_back(total);
            }
            row[F - 1] += wynn_epsilon(partial);
        }
        for (int f = 0; f < F; ++f) T[(size_t)g * F + f] = -(2.0 * MU0 / PI) * row[f];
    }
}

// ---------------------------------------------------------------------------
// Batched forward model on merged layers.
// Model arrays are row-major [P][LMAX]: log10 sigma_inf, log10 thickness (the
// bottom layer's is ignored), m, log10 tau, c.
// hankel_mode: 0 = adaptive quadrature (reflection recursion),
//              1 = adaptive quadrature (admittance recursion),
//              2 = the K-point log-spaced rule.
// Outputs: Im Hz_s per node (P x F) if imh != NULL, gates (P x G) if y != NULL.
// ---------------------------------------------------------------------------
struct OracleModelView {
    int LMAX;
    const int *nlayers;
    const double *logsig, *logh, *m, *logtau, *c;
};

static void forward_one(const OracleModelView &mv, int p, int cc_form, double a, double h, double current,
                        int F, const double *freqs, int G, const double *T, int hankel_mode, int K,
                        double rtol, double *imh_row, double *y_row, double *absh_row) {
    int L = mv.nlayers[p];
    std::vector<double> sig(L), thick(L), mm(L), tau(L), cc(L);
    for (int n = 0; n < L; ++n) {
        sig[n] = std::pow(10.0, mv.logsig[(size_t)p * mv.LMAX + n]);
        thick[n] = (n < L - 1) ? std::pow(10.0, mv.logh[(size_t)p * mv.LMAX + n]) : 0.0;
        mm[n] = mv.m[(size_t)p * mv.LMAX + n];
        tau[n] = std::pow(10.0, mv.logtau[(size_t)p * mv.LMAX + n]);
        cc[n] = mv.c[(size_t)p * mv.LMAX + n];
    }
    std::vector<double> lam, ck;
    if (hankel_mode == 2) hankel_rule(K, a, h, current, lam, ck);
    std::vector<double> imh(F);
    std::vector<cd> s(L);
    for (int f = 0; f < F; ++f) {
        double w = 2.0 * PI * freqs[f];
        for (int n = 0; n < L; ++n) s[n] = cd(0.0, w * MU0) * colecole(cc_form, sig[n], mm[n], tau[n], cc[n], w);
        cd H;
        if (hankel_mode == 2) {
            H = cd(0.0, 0.0);
            double mag = 0.0;  // sum of |term| of the rule: the scale of its rounding error
            for (int k = 0; k < K; ++k) {
                cd R = r0_reflection(L, s.data(), thick.data(), lam[k]);
                H += ck[k] * R;
                mag += std::fabs(ck[k]) * std::abs(R);
            }
            if (absh_row) absh_row[f] = mag;
        } else {
            H = hz_quadrature(L, s.data(), thick.data(), a, h, current, hankel_mode, rtol);
        }
        imh[f] = H.imag();
    }
    if (imh_row) for (int f = 0; f < F; ++f) imh_row[f] = imh[f];
    if (y_row && T) {
        for (int g = 0; g < G; ++g) {
            double acc = 0.0;
            for (int f = 0; f < F; ++f) acc += T[(size_t)g * F + f] * imh[f];
            y_row[g] = acc;
        }
    }
}

extern "C" int orc_forward(int P, int LMAX, const int *nlayers, const double *logsig, const double *logh,
                           const double *m, const double *logtau, const double *c, int cc_form, double a,
                           double h, double current, int F, const double *freqs, int G, const double *T,
                           int hankel_mode, int K, double rtol, double *imh, double *y, int nthreads,
                           double *absh) {
    OracleModelView mv{LMAX, nlayers, logsig, logh, m, logtau, c};
    for (int p = 0; p < P; ++p)
        if (nlayers[p] < 1 || nlayers[p] > LMAX) return -1;
    if (nthreads < 1) nthreads = 1;
    std::vector<std::thread> pool;
    for (int tid = 0; tid < nthreads; ++tid) {
        pool.emplace_back([&, tid]() {
            for (int p = tid; p < P; p += nthreads)
                forward_one(mv, p, cc_form, a, h, current, F, freqs, G, T, hankel_mode, K, rtol,
                            imh ? imh + (size_t)p * F : nullptr, y ? y + (size_t)p * G : nullptr,
                            absh ? absh + (size_t)p * F : nullptr);
        });
    }
    for (auto &th : pool) th.join();
    return 0;
}

// Single-point helpers for the pins.
extern "C" void orc_colecole(int form, double sig, double m, double tau, double c, double w, double *out2) {
    cd z = colecole(form, sig, m, tau, c, w);
    out2[0] = z.real();
    out2[1] = z.imag();
}

extern "C" void orc_r0(int L, const double *sig_re, const double *sig_im, const double *thick, double lam,
                       double w, int method, double *out2) {
    std::vector<cd> s(L);
    for (int n = 0; n < L; ++n) s[n] = cd(0.0, w * MU0) * cd(sig_re[n], sig_im[n]);
    cd R = method == 0 ? r0_reflection(L, s.data(), thick, lam) : r0_admittance(L, s.data(), thick, lam);
    out2[0] = R.real();
    out2[1] = R.imag();
}

extern "C" void orc_hz(int L, const double *sig_re, const double *sig_im, const double *thick, double a,
                       double h, double current, double w, int mode, int K, double rtol, double *out2) {
    std::vector<cd> s(L);
    for (int n = 0; n < L; ++n) s[n] = cd(0.0, w * MU0) * cd(sig_re[n], sig_im[n]);
    cd H;
    if (mode == 2) {
        std::vector<double> lam, ck;
        hankel_rule(K, a, h, current, lam, ck);
        H = cd(0.0, 0.0);
        for (int k = 0; k < K; ++k) H += ck[k] * r0_reflection(L, s.data(), thick, lam[k]);
    } else {
        H = hz_quadrature(L, s.data(), thick, a, h, current, mode, rtol);
    }
    out2[0] = H.real();
    out2[1] = H.imag();
}

extern "C" void orc_hankel_rule(int K, double a, double h, double current, double *lam_out, double *c_out) {
    std::vector<double> lam, ck;
    hankel_rule(K, a, h, current, lam, ck);
    for (int k = 0; k < K; ++k) {
        lam_out[k] = lam[k];
        c_out[k] = ck[k];
    }
}

// Gaussian log-likelihood (Section 2.3.2), one model at a time, summed in order.
extern "C" void orc_loglik(int P, int G, const double *y_model, const double *y_obs, const double *eps_an,
                           double eps_mn, double *ll) {
    for (int p = 0; p < P; ++p) {
        double acc = 0.0;
        for (int g = 0; g < G; ++g) {
            double yhat = y_model[(size_t)p * G + g];
            double v = eps_an[g] * eps_an[g] + (eps_mn * yhat) * (eps_mn * yhat);
            double r = y_obs[g] - yhat;
            acc += r * r / v + std::log(2.0 * PI * v);
        }
        ll[p] = -0.5 * acc;
    }
}
