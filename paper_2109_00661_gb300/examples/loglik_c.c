/* The forward model and Gaussian log-likelihood through the C ABI alone
 * (include/aem_rjsmc.h), without Python: a 3-layer earth with a chargeable
 * second layer, its FP64 gates taken as the observed data, then the FP32
 * log-likelihood of a batch of perturbed copies of that earth.
 *
 * Build (after the library):
 *   gcc -O2 -I include paper_2109_00661_gb300/examples/loglik_c.c \
 *       -L paper_2109_00661_gb300/_build -laemrjsmc \
 *       -L /usr/local/cuda/lib64 -lcudart -Wl,-rpath,paper_2109_00661_gb300/_build -lm -o loglik_c
 * Run: ./loglik_c [n_models]    (prints the first log-likelihoods; exit status
 * 0 when every call succeeded and the unperturbed copy scores highest). */
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "aem_rjsmc.h"

#define CHECK_AEM(call)                                                              \
    do {                                                                             \
        int rc_ = (call);                                                            \
        if (rc_ != AEM_OK) {                                                         \
            fprintf(stderr, "%s failed (%d): %s\n", #call, rc_, aem_last_error());   \
            return 1;                                                                \
        }                                                                            \
    } while (0)
#define CHECK_CUDA(call)                                                             \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            fprintf(stderr, "%s failed: %s\n", #call, cudaGetErrorString(e_));       \
            return 1;                                                                \
        }                                                                            \
    } while (0)

enum { G = 20, F = 40, K = 120, LMAX = 3 };

int main(int argc, char **argv) {
    const int P = argc > 1 ? atoi(argv[1]) : 1024;
    if (P < 1) return 2;

    /* the single-sounding system: 13 m loop at 30 m, 20 gates 1e-5..1e-2 s */
    double times[G];
    for (int g = 0; g < G; ++g) times[g] = pow(10.0, -5.0 + 3.0 * g / (G - 1));
    aem_system_desc desc = {13.0, 30.0, 1.0, F, 1.0, 1e7, G, times, K, AEM_CC_PAPER};
    aem_system *sys = NULL;
    CHECK_AEM(aem_system_create(&desc, &sys));

    /* host models: copy 0 is the truth, the others are perturbed in log10 sigma */
    const size_t n = (size_t)P * LMAX;
    int8_t *nl = malloc(P);
    float *h32[5];
    double *h64[5];
    for (int q = 0; q < 5; ++q) {
        h32[q] = malloc(n * sizeof(float));
        h64[q] = malloc(n * sizeof(double));
    }
    const double sig[LMAX] = {0.01, 0.1, 0.01}, thick[LMAX] = {20.0, 30.0, 1.0}, mm[LMAX] = {0.0, 0.3, 0.0};
    srand(7);
    for (int p = 0; p < P; ++p) {
        nl[p] = LMAX;
        const double d = p == 0 ? 0.0 : 0.3 * ((double)rand() / RAND_MAX - 0.5);
        for (int j = 0; j < LMAX; ++j) {
            const size_t o = (size_t)p * LMAX + j;
            h64[0][o] = log10(sig[j]) + d;
            h64[1][o] = log10(thick[j]);
            h64[2][o] = mm[j];
            h64[3][o] = -3.0;
            h64[4][o] = 0.5;
            for (int q = 0; q < 5; ++q) h32[q][o] = (float)h64[q][o];
        }
    }

    /* device copies (the caller owns every buffer the library reads or writes) */
    int8_t *d_nl;
    float *d32[5];
    double *d64[5], *d_y, *d_eps, *d_ll, *d_gates64;
    CHECK_CUDA(cudaMalloc((void **)&d_nl, P));
    CHECK_CUDA(cudaMemcpy(d_nl, nl, P, cudaMemcpyHostToDevice));
    for (int q = 0; q < 5; ++q) {
        CHECK_CUDA(cudaMalloc((void **)&d32[q], n * sizeof(float)));
        CHECK_CUDA(cudaMalloc((void **)&d64[q], n * sizeof(double)));
        CHECK_CUDA(cudaMemcpy(d32[q], h32[q], n * sizeof(float), cudaMemcpyHostToDevice));
        CHECK_CUDA(cudaMemcpy(d64[q], h64[q], n * sizeof(double), cudaMemcpyHostToDevice));
    }
    CHECK_CUDA(cudaMalloc((void **)&d_y, G * sizeof(double)));
    CHECK_CUDA(cudaMalloc((void **)&d_eps, G * sizeof(double)));
    CHECK_CUDA(cudaMalloc((void **)&d_ll, (size_t)P * sizeof(double)));
    CHECK_CUDA(cudaMalloc((void **)&d_gates64, (size_t)G * sizeof(double)));

    /* observed data: the truth's FP64 gates (copy 0 only) */
    aem_models_f64 truth = {1, LMAX, d_nl, d64[0], d64[1], d64[2], d64[3], d64[4]};
    CHECK_AEM(aem_forward_f64(sys, &truth, d_gates64, NULL, NULL));
    CHECK_CUDA(cudaMemcpy(d_y, d_gates64, G * sizeof(double), cudaMemcpyDeviceToDevice));
    double eps[G];
    for (int g = 0; g < G; ++g) eps[g] = 1e-13;
    CHECK_CUDA(cudaMemcpy(d_eps, eps, sizeof eps, cudaMemcpyHostToDevice));

    /* the FP32 log-likelihood of the whole batch */
    aem_models_f32 models = {P, LMAX, d_nl, d32[0], d32[1], d32[2], d32[3], d32[4]};
    CHECK_AEM(aem_loglik_f32(sys, &models, d_y, d_eps, 0.03, d_ll, NULL, NULL));
    double *ll = malloc((size_t)P * sizeof(double));
    CHECK_CUDA(cudaMemcpy(ll, d_ll, (size_t)P * sizeof(double), cudaMemcpyDeviceToHost));

    int best = 0;
    for (int p = 1; p < P; ++p)
        if (ll[p] > ll[best]) best = p;
    for (int p = 0; p < (P < 4 ? P : 4); ++p) printf("ll[%d] = %.6f\n", p, ll[p]);
    printf("best model %d of %d\n", best, P);

    for (int q = 0; q < 5; ++q) {
        cudaFree(d32[q]);
        cudaFree(d64[q]);
        free(h32[q]);
        free(h64[q]);
    }
    cudaFree(d_nl);
    cudaFree(d_y);
    cudaFree(d_eps);
    cudaFree(d_ll);
    cudaFree(d_gates64);
    free(nl);
    free(ll);
    CHECK_AEM(aem_system_destroy(sys));
    return best == 0 ? 0 : 3;
}
