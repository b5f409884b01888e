// Gate transform y = T Im H (Section 2.3.2: step-off gates from the
// frequency-domain response) and the Gaussian log-likelihood, from a batch of
// spectra, on the 5th-generation tensor cores.
//
// The transform is the one dense contraction of the path: D[P x G] =
// A[P x F] B[G x F]^T with A the spectra and B the transform matrix.  The
// spectra are FP32 and the transform is ill-conditioned (terms of both signs
// cancel), so each operand is split into a high and a low part in the tensor
// input type and three products are accumulated in FP32:
//   D = A_hi B_hi + A_hi B_lo + A_lo B_hi
// (the dropped A_lo B_lo term is below the split's own rounding).  TF32
// (11-bit significand) leaves a relative residual near 2^-22 per term, BF16
// (8-bit) near 2^-17.
//
// One CTA of four warps per 128-model tile (persistent over tiles): the
// threads stage A_hi / A_lo of the tile and, once per CTA, B_hi / B_lo in
// shared memory in the canonical K-major layout without swizzle (core
// matrices of 8 rows x 16 bytes); one thread issues the tcgen05.mma chain
// into a TMEM accumulator (row m of the tile in TMEM lane m, gate n in column
// n) and commits it to an mbarrier; every warp then reads its 32 lanes with
// tcgen05.ld and forms the gates and the likelihood of its 32 models.  Every
// wait is bounded: on a timeout the CTA records AEM_ERR_TIMEOUT in the
// system's status word, waits (bounded) once more for its own MMAs, frees its
// TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "aem_internal.h"

namespace aem {
namespace {

constexpr int kTM = 128;       // models per tile = MMA M
constexpr int kThreads = 128;  // warp w reads TMEM lanes 32w .. 32w + 31
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (no swizzle): start address, leading
// (K-direction core matrix) byte offset and stride (8-row group) byte offset in
// 16-byte units at bits 0-13, 16-29 and 32-45; descriptor version 1 at bit 46;
// base offset 0, swizzle mode 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor for kind::tf32 / kind::f16: FP32 accumulator (bits
// 4-5 = 1), A and B formats at bits 7-9 and 10-12 (BF16 = 1, TF32 = 2), both
// operands K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

template <int KIND>  // 0: TF32 split, 1: BF16 split
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accumulate) {
    if constexpr (KIND == 0) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
    }
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the given phase parity of the mbarrier.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
    for (uint32_t i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Eight consecutive FP32 columns of this thread's TMEM lane; the wait takes
// the registers as operands so that no use is scheduled before it.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
    uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3), "+r"(r4), "+r"(r5), "+r"(r6), "+r"(r7)::"memory");
    v[0] = __uint_as_float(r0);
    v[1] = __uint_as_float(r1);
    v[2] = __uint_as_float(r2);
    v[3] = __uint_as_float(r3);
    v[4] = __uint_as_float(r4);
    v[5] = __uint_as_float(r5);
    v[6] = __uint_as_float(r6);
    v[7] = __uint_as_float(r7);
}

// High / low split of x in the tensor input type (raw bits).
template <int KIND>
struct Split;
template <>
struct Split<0> {
    using T = uint32_t;
    static constexpr int ES = 4;
    __device__ static void run(float x, uint32_t &hi, uint32_t &lo) {
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
        const float r = x - __uint_as_float(hi);
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
    }
};
template <>
struct Split<1> {
    using T = uint16_t;
    static constexpr int ES = 2;
    __device__ static void run(float x, uint16_t &hi, uint16_t &lo) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(l);
    }
};

// Byte offset of element (row r, k) in the K-major no-swizzle layout with
// K-adjacent core matrices 128 bytes apart and 8-row groups sbo bytes apart.
template <int ES>
__device__ __forceinline__ uint32_t kmajor_offset(int r, int k, uint32_t sbo) {
    constexpr int KC = 16 / ES;
    return (uint32_t)(r >> 3) * sbo + (uint32_t)(k / KC) * 128u + (uint32_t)(r & 7) * 16u + (uint32_t)(k % KC) * ES;
}

struct TcArgs {
    const float *imh;  // [P][F]
    int P, F, G, KP, N, ncols;
    const float *T;  // [G][F]
    const double *y_obs;
    int obs_per;
    const double *eps_an;
    double eps_mn;
    float *gates;  // [P][G] or null
    double *ll;    // [P] or null
    int *status;
};

template <int KIND>
__global__ void __launch_bounds__(kThreads) gates_tc_kernel(TcArgs a) {
    using S = Split<KIND>;
    using E = typename S::T;
    constexpr int ES = S::ES;
    constexpr int KI = 32 / ES;  // K of one MMA: two core matrices
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    unsigned char *base = smem_raw + pad;
    const uint32_t sbo = (uint32_t)(a.KP / (16 / ES)) * 128u;  // same for A and B
    const uint32_t a_bytes = (uint32_t)kTM * a.KP * ES, b_bytes = (uint32_t)a.N * a.KP * ES;
    unsigned char *Ahi = base, *Alo = base + a_bytes, *Bhi = base + 2 * a_bytes, *Blo = Bhi + b_bytes;
    uint64_t *mbar_p = reinterpret_cast<uint64_t *>(Blo + b_bytes);
    uint32_t *slot_p = reinterpret_cast<uint32_t *>(mbar_p + 1);
    int *abort_p = reinterpret_cast<int *>(slot_p + 1);
    const uint32_t mbar = smem_u32(mbar_p);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        mbar_init(mbar, 1);
        *abort_p = 0;
    }
    __syncwarp();
    if (warp == 0) tmem_alloc(smem_u32(slot_p), (uint32_t)a.ncols);
    // B = T (rows: gates, zero-padded to N; columns: frequencies, zero-padded to KP)
    for (int i = tid; i < a.N * a.KP; i += kThreads) {
        const int n = i / a.KP, k = i - (i / a.KP) * a.KP;
        const float x = (n < a.G && k < a.F) ? a.T[n * a.F + k] : 0.f;
        E hi, lo;
        S::run(x, hi, lo);
        const uint32_t o = kmajor_offset<ES>(n, k, sbo);
        *reinterpret_cast<E *>(Bhi + o) = hi;
        *reinterpret_cast<E *>(Blo + o) = lo;
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tbase = *slot_p;
    const uint32_t idesc = instr_desc(KIND == 0 ? 2u : 1u, (uint32_t)kTM, (uint32_t)a.N);
    const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo), bhi = smem_u32(Bhi), blo = smem_u32(Blo);
    const int ntiles = (a.P + kTM - 1) / kTM;
    uint32_t phase = 0;
    bool pending = false;  // an MMA chain committed and not yet observed complete

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // stage the tile's spectra (rows past P and columns past F are zero)
        const size_t row0 = (size_t)tile * kTM;
        for (int i = tid; i < kTM * a.KP; i += kThreads) {
            const int r = i / a.KP, k = i - (i / a.KP) * a.KP;
            const size_t m = row0 + r;
            const float x = (m < (size_t)a.P && k < a.F) ? a.imh[m * a.F + k] : 0.f;
            E hi, lo;
            S::run(x, hi, lo);
            const uint32_t o = kmajor_offset<ES>(r, k, sbo);
            *reinterpret_cast<E *>(Ahi + o) = hi;
            *reinterpret_cast<E *>(Alo + o) = lo;
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        tc_after_sync();
        if (tid == 0) {
            for (int ks = 0; ks < a.KP / KI; ++ks) {
                const uint32_t off = (uint32_t)ks * 256u;
                const uint64_t dah = smem_desc(ahi + off, 128u, sbo), dal = smem_desc(alo + off, 128u, sbo);
                const uint64_t dbh = smem_desc(bhi + off, 128u, sbo), dbl = smem_desc(blo + off, 128u, sbo);
                mma<KIND>(tbase, dah, dbh, idesc, ks > 0 ? 1u : 0u);
                mma<KIND>(tbase, dah, dbl, idesc, 1u);
                mma<KIND>(tbase, dal, dbh, idesc, 1u);
            }
            mma_commit(mbar);
        }
        pending = true;
        const bool done = mbar_wait_bounded(mbar, phase);
        if (!done) atomicExch(abort_p, 1);
        __syncthreads();
        if (*abort_p) break;
        pending = false;
        phase ^= 1u;
        tc_after_sync();
        // epilogue: this thread's model is row 32 warp + lane of the tile
        const size_t m = row0 + (size_t)warp * 32 + lane;
        const bool valid = m < (size_t)a.P;
        const double *y = a.y_obs ? a.y_obs + (valid ? (m / (size_t)a.obs_per) * a.G : 0) : nullptr;
        double acc = 0.0;
        for (int c = 0; c < a.N; c += 8) {
            float v[8];
            tmem_ld8(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int g = c + q;
                if (valid && g < a.G) {
                    if (a.gates) a.gates[m * a.G + g] = v[q];
                    if (y) {
                        const double yh = (double)v[q], ea = a.eps_an[g];
                        const double var = ea * ea + (a.eps_mn * yh) * (a.eps_mn * yh);
                        const double r = y[g] - yh;
                        acc += r * r / var + log(2.0 * kPi * var);
                    }
                }
            }
        }
        if (valid && a.ll) a.ll[m] = -0.5 * acc;
        tc_before_sync();
        __syncthreads();  // every lane read before the next chain overwrites the accumulator
    }
    if (*abort_p) {
        if (tid == 0) atomicExch(a.status, (int)AEM_ERR_TIMEOUT);
        if (pending) mbar_wait_bounded(mbar, phase);  // our own MMAs, once more with a limit
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0) tmem_dealloc(tbase, (uint32_t)a.ncols);
}

// FP32 CUDA-core form of the same transform (for comparison): one thread per
// model, T staged in shared memory.
__global__ void gates_fp32_kernel(TcArgs a) {
    extern __shared__ float Ts[];
    for (int i = threadIdx.x; i < a.G * a.F; i += blockDim.x) Ts[i] = a.T[i];
    __syncthreads();
    for (size_t m = (size_t)blockIdx.x * blockDim.x + threadIdx.x; m < (size_t)a.P; m += (size_t)gridDim.x * blockDim.x) {
        const float *x = a.imh + m * a.F;
        const double *y = a.y_obs ? a.y_obs + (m / (size_t)a.obs_per) * a.G : nullptr;
        double acc = 0.0;
        for (int g = 0; g < a.G; ++g) {
            float s = 0.f;
            for (int k = 0; k < a.F; ++k) s = fmaf(Ts[g * a.F + k], x[k], s);
            if (a.gates) a.gates[m * a.G + g] = s;
            if (y) {
                const double yh = (double)s, ea = a.eps_an[g];
                const double var = ea * ea + (a.eps_mn * yh) * (a.eps_mn * yh);
                const double r = y[g] - yh;
                acc += r * r / var + log(2.0 * kPi * var);
            }
        }
        if (a.ll) a.ll[m] = -0.5 * acc;
    }
}

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

int gates_from_spectrum(const aem_system *sys, const float *imh, int P, int mode, const double *y_obs,
                        int obs_per, const double *eps_an, double eps_mn, float *gates, double *ll,
                        cudaStream_t stream) {
    const SystemTables &h = sys->host;
    TcArgs a{imh, P, h.F, h.G, 0, 0, 0, sys->d_T_f, y_obs, obs_per > 0 ? obs_per : 1, eps_an, eps_mn, gates, ll,
             sys->d_status};
    if (mode == AEM_GATES_FP32) {
        const size_t smem = sizeof(float) * (size_t)h.G * h.F;
        int grid = (int)((P + 255) / 256);
        if (grid > sys->num_sms * 8) grid = sys->num_sms * 8;
        gates_fp32_kernel<<<grid, 256, smem, stream>>>(a);
        AEM_CUDA_TRY(cudaGetLastError());
        return AEM_OK;
    }
    const bool tf32 = mode == AEM_GATES_TF32_SPLIT;
    const int ES = tf32 ? 4 : 2, KI = 32 / ES;
    a.KP = round_up(h.F, KI);
    a.N = round_up(h.G, 16);
    a.ncols = a.N <= 32 ? 32 : 64;
    const size_t smem = (size_t)2 * (kTM + a.N) * a.KP * ES + 1024 + 64;
    auto kern = tf32 ? gates_tc_kernel<0> : gates_tc_kernel<1>;
    AEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    AEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1) return fail(AEM_ERR_UNSUPPORTED, "aem_gates_from_spectrum: tile does not fit in shared memory");
    const int ntiles = (P + kTM - 1) / kTM;
    int grid = sys->num_sms * per_sm;
    if (grid > ntiles) grid = ntiles;
    kern<<<grid, kThreads, smem, stream>>>(a);
    AEM_CUDA_TRY(cudaGetLastError());
    return AEM_OK;
}

}  // namespace aem

using namespace aem;

extern "C" int aem_gates_from_spectrum(const aem_system *sys, const float *imh, int n_models, int mode,
                                       const double *y_obs, const double *eps_an, double eps_mn, float *gates,
                                       double *ll, void *stream) {
    if (!sys) return fail(AEM_ERR_INVALID_ARG, "aem_gates_from_spectrum: sys is NULL");
    if (n_models < 0) return fail(AEM_ERR_INVALID_ARG, "aem_gates_from_spectrum: n_models < 0");
    if (mode != AEM_GATES_FP32 && mode != AEM_GATES_TF32_SPLIT && mode != AEM_GATES_BF16_SPLIT)
        return fail(AEM_ERR_INVALID_ARG, "aem_gates_from_spectrum: unknown mode");
    if (n_models == 0) return AEM_OK;
    if (!imh || (!gates && !ll) || (ll && (!y_obs || !eps_an)))
        return fail(AEM_ERR_INVALID_ARG, "aem_gates_from_spectrum: NULL pointer");
    return gates_from_spectrum(sys, imh, n_models, mode, y_obs, n_models, eps_an, eps_mn, gates, ll,
                               (cudaStream_t)stream);
}

extern "C" int aem_loglik_f32_tc(const aem_system *sys, const aem_models_f32 *models, const double *y_obs,
                                 const double *eps_an, double eps_mn, int mode, float *imh_work, double *ll,
                                 float *gates, void *stream) {
    if (!sys || !models) return fail(AEM_ERR_INVALID_ARG, "aem_loglik_f32_tc: NULL system or models");
    if (models->n_models == 0) return AEM_OK;
    if (!imh_work || !ll || !y_obs || !eps_an) return fail(AEM_ERR_INVALID_ARG, "aem_loglik_f32_tc: NULL pointer");
    int rc = aem_forward_f32(sys, models, nullptr, imh_work, stream);
    if (rc) return rc;
    return aem_gates_from_spectrum(sys, imh_work, models->n_models, mode, y_obs, eps_an, eps_mn, gates, ll, stream);
}

extern "C" int aem_system_status(const aem_system *sys, int *status) {
    if (!sys || !status) return fail(AEM_ERR_INVALID_ARG, "aem_system_status: NULL argument");
    int v = 0;
    AEM_CUDA_TRY(cudaMemcpy(&v, sys->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) AEM_CUDA_TRY(cudaMemset(sys->d_status, 0, sizeof(int)));
    *status = v;
    return AEM_OK;
}
