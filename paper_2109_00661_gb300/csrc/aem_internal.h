// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/aem_rjsmc.h"

namespace aem {

constexpr double kPi = 3.14159265358979323846;
constexpr double kMu0 = 4e-7 * kPi;

// Records the message returned by aem_last_error() and passes the code through.
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t err, const char *what);

#define AEM_CUDA_TRY(expr)                                        \
    do {                                                          \
        cudaError_t _e = (expr);                                  \
        if (_e != cudaSuccess) return ::aem::cuda_fail(_e, #expr); \
    } while (0)

// Host-side tables (double) and their device copies (float and double).
struct SystemTables {
    double a = 0, h = 0, current = 1;
    int F = 0, G = 0, K = 0, cc_form = 0;
    std::vector<double> freqs, omega, times, lam, hw, T;  // T is G x F
};

// Gates (and log-likelihood) from spectra [P][F] by the transform of the
// given aem_gates_mode; y_obs rows advance every obs_per models (gates_tc.cu).
int gates_from_spectrum(const aem_system *sys, const float *imh, int P, int mode, const double *y_obs,
                        int obs_per, const double *eps_an, double eps_mn, float *gates, double *ll,
                        cudaStream_t stream);
}  // namespace aem

struct aem_system {
    aem::SystemTables host;
    int device = 0;
    // device tables: omega[F], lam[K], hw[K], T[G*F] in both precisions
    float *d_omega_f = nullptr, *d_lam_f = nullptr, *d_hw_f = nullptr, *d_T_f = nullptr;
    double *d_omega_d = nullptr, *d_lam_d = nullptr, *d_hw_d = nullptr, *d_T_d = nullptr;
    int num_sms = 0;
    // device status word: kernels record AEM_ERR_TIMEOUT here when a bounded
    // wait gives up (read and cleared by aem_system_status)
    int *d_status = nullptr;
    // diagnostics of the tensor-core transform's bounded wait (aem_debug_bounded_wait):
    // iteration limit (0: the default) and whether CTAs issue nothing for their first tile
    unsigned int wait_spins = 0;
    int wait_skip_mma = 0;
    // launch shape of the FP32 forward kernel per lmax (index into its shape
    // table, 0 = default), set by aem_autotune_forward / aem_forward_shape
    int f32_shape[AEM_MAX_LAYERS + 1] = {};
    // the FP32 forward kernel's depth cutoff (aem_system_set_depth_cutoff):
    // attenuation exponent, 0 = the whole stack always
    float depth_att = 20.f;
};

namespace aem {
// Builds the Hankel rule and the transform matrix on the host (system.cpp).
int build_tables(const aem_system_desc *desc, SystemTables *out);
// FP32 forward + log-likelihood where consecutive blocks of
// models_per_sounding models use consecutive rows of y_obs (forward.cu).
// counter: optional device int the dynamic-scheduled shapes use for model
// claiming instead of a per-launch stream-ordered allocation.  active:
// optional device int; when it holds 0 the launch does nothing (a sweep of a
// captured stage loop that the device-side sweep count switched off).  valid:
// optional per-model device flags; a model whose flag is 0 is skipped and its
// ll left as it was (a proposal that was no move, which the accept step
// ignores).
int loglik_f32_soundings(const aem_system *sys, const aem_models_f32 *models, const double *y_obs,
                         int models_per_sounding, const double *eps_an, double eps_mn, double *ll,
                         cudaStream_t stream, int *counter = nullptr, const int *active = nullptr,
                         const int8_t *valid = nullptr);
// The plain FP64 forward model + log-likelihood with the same per-sounding
// rows of y_obs (forward.cu); active and valid as above.
int loglik_f64_soundings(const aem_system *sys, const aem_models_f64 *models, const double *y_obs,
                         int models_per_sounding, const double *eps_an, double eps_mn, double *ll,
                         cudaStream_t stream, const int *active = nullptr, const int8_t *valid = nullptr);
// Gates [P][G] and log-likelihood (may be NULL) of the FP32 forward kernel
// with per-sounding rows of y_obs (forward.cu); counter and valid as above.
int loglik_gates_f32_soundings(const aem_system *sys, const aem_models_f32 *models, const double *y_obs,
                               int models_per_sounding, const double *eps_an, double eps_mn, double *ll, float *gates,
                               cudaStream_t stream, int *counter = nullptr, const int8_t *valid = nullptr);
// Log-likelihood and its merged-layer gradient [P][lmax][5] with the same
// per-sounding rows of y_obs (adjoint.cu).  work: optional device scratch of
// grad_work_bytes(P, G) bytes (the claim counters and the gates); without it
// the call takes stream-ordered scratch of that size for its duration.  With
// it the call makes no allocation, so it can be captured inside a
// conditional graph body.  valid: optional per-model device flags; a model
// whose flag is 0 is skipped (its ll and gradient left as they were).
size_t grad_work_bytes(int n_models, int G);
int loglik_grad_f32_soundings(const aem_system *sys, const aem_models_f32 *models, const double *y_obs,
                              int models_per_sounding, const double *eps_an, double eps_mn, double *ll, float *grad,
                              cudaStream_t stream, void *work = nullptr, const int8_t *valid = nullptr);
// Gates (and log-likelihood) from spectra [P][F] by the transform of the
// given aem_gates_mode; y_obs rows advance every obs_per models (gates_tc.cu).
int gates_from_spectrum(const aem_system *sys, const float *imh, int P, int mode, const double *y_obs,
                        int obs_per, const double *eps_an, double eps_mn, float *gates, double *ll,
                        cudaStream_t stream);
}  // namespace aem
