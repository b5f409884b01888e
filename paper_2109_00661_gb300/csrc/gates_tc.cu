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
// One CTA of eight warps per 128-model tile (persistent over tiles, several
// CTAs per SM so that one CTA's staging overlaps another's MMA and epilogue):
// the threads stage A_hi / A_lo of the tile and, once per CTA, B_hi / B_lo in
// shared memory in the canonical K-major layout without swizzle (core
// matrices of 8 rows x 16 bytes), each lane converting one 16-byte core-matrix
// row so that a warp's stores cover 512 contiguous bytes; one thread issues
// the tcgen05.mma chain into a TMEM accumulator (row m of the tile in TMEM
// lane m, gate n in column n) and commits it to an mbarrier; every warp then
// reads its 32 lanes (warps w and w + 4 the same lanes, each half of the
// columns) with tcgen05.ld and forms the gates and the likelihood terms of
// its 32 models, the two halves' sums meeting in shared memory.  The likelihood terms are FP32 (Section 2.3.2's Gaussian:
// the residual from a float pair holding the FP64 datum, the variance, one
// logarithm and one division per gate) and their sum is carried as an
// unevaluated FP32 pair (Knuth's TwoSum), exact to about 2^-48 of the sum of
// magnitudes, so no FP64 arithmetic is left per gate.  Every wait is bounded:
// on a timeout the CTA records AEM_ERR_TIMEOUT in the system's status word,
// waits (bounded) once more for its own MMAs, frees its TMEM and returns.  If
// that second wait also gives up, the MMAs it issued may still be in flight
// when the TMEM is freed, which the tcgen05 model leaves undefined: the
// recorded timeout then means the device context should be treated as
// unreliable.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "aem_internal.h"

namespace aem {
namespace {

constexpr int kTM = 128;       // models per tile = MMA M
constexpr int kThreads = 256;  // warps w and w + 4 read TMEM lanes 32 (w mod 4) .., one half of the columns each
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr double kLn2Pi = 1.83787706640934548356;  // ln(2 pi)

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
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, uint32_t limit = kSpinLimit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}

// Knuth's TwoSum: s + e == a + b exactly (round to nearest, no overflow).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
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
    uint32_t spins;  // iteration limit of the completion wait
    int skip_mma;    // diagnostics: issue nothing for the first tile (the wait then runs out)
};

// The likelihood terms of one model's gates (Section 2.3.2), FP32 terms
// with the TwoSum-carried sum: for gate g, yh the prediction, (yhi, ylo) the
// float pair of the datum and ea2 = eps_an^2,
//   r = (yhi - yh) + ylo,  v = ea2 + (eps_mn yh)^2,  t = r^2 / v + ln v,
// and ll = -1/2 (sum t + G ln 2 pi) formed in FP64 once per model.
struct LlAcc {
    float s = 0.f, e = 0.f;
    __device__ __forceinline__ void add(float yh, float2 y, float ea2, float em) {
        const float r = (y.x - yh) + y.y;
        const float q = em * yh;
        const float v = fmaf(q, q, ea2);
        const float t = __fdiv_rn(r * r, v) + logf(v);
        float s1, e1;
        two_sum(s, t, s1, e1);
        s = s1;
        e += e1;
    }
    __device__ __forceinline__ double ll(int G) const {
        return -0.5 * (((double)s + (double)e) + (double)G * kLn2Pi);
    }
};

// Converts the 16-byte core-matrix row of element chunk (r, kc) of the tile:
// chunk kc holds elements 16/ES * kc .. of row r.  src: that row's FP32
// values (nullptr: a padding row), zero past F.
template <int KIND>
__device__ __forceinline__ void stage_chunk(const float *__restrict__ src, int F, int kc, bool vec4,
                                            unsigned char *hi_row, unsigned char *lo_row) {
    using S = Split<KIND>;
    constexpr int KC = 16 / S::ES;  // elements per 16-byte core-matrix row
    float x[KC];
    const int k0 = kc * KC;
    if (src && vec4 && k0 + KC <= F) {
#pragma unroll
        for (int q = 0; q < KC; q += 4) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(src + k0 + q));
            x[q] = v.x;
            x[q + 1] = v.y;
            x[q + 2] = v.z;
            x[q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < KC; ++q) x[q] = (src && k0 + q < F) ? __ldg(src + k0 + q) : 0.f;
    }
    typename S::T h[KC], l[KC];
#pragma unroll
    for (int q = 0; q < KC; ++q) S::run(x[q], h[q], l[q]);
    *reinterpret_cast<uint4 *>(hi_row) = *reinterpret_cast<const uint4 *>(h);
    *reinterpret_cast<uint4 *>(lo_row) = *reinterpret_cast<const uint4 *>(l);
}

// Register prefetch of a tile's spectra: thread tid owns chunks
// c = tid + j kThreads (j < JC = kTM NKC / kThreads), each chunk KC / 4 float4
// loads; a tile needs JC KC / 4 <= kPF of them per thread (F <= 64 for both
// splits) and F a multiple of 4 (16-byte rows).  The next tile's loads are
// issued before the current tile's MMA wait and epilogue, so their latency
// overlaps both.  Chunk j's core-matrix index is (tid >> 3) + 32 j: its
// quotient and remainder by NKC (row group, core-matrix column) advance by
// those of 32 with one carry per chunk, from one division per thread.
constexpr int kPF = 8;

template <int KIND>
struct TilePrefetch {
    static constexpr int KC = 16 / Split<KIND>::ES;  // elements per core-matrix row
    static constexpr int Q = KC / 4;                 // float4 loads per chunk
    static constexpr int JMAX = kPF / Q;             // chunks per thread
    float4 v[kPF];
    int nkc;   // NKC
    int pack;  // divmod(tid >> 3, NKC) and divmod(32, NKC), a byte each (all below 64 when the prefetch applies)

    __device__ __forceinline__ void init(int NKC, int tid) {
        nkc = NKC;
        const int q0 = (tid >> 3) / NKC, dq = 32 / NKC;
        pack = q0 | (((tid >> 3) - q0 * NKC) << 8) | (dq << 16) | ((32 - dq * NKC) << 24);
    }

    __device__ __forceinline__ void load(const float *__restrict__ imh, int P, int F, size_t row0) {
        const int jc = nkc * kTM / kThreads, r7 = threadIdx.x & 7;
        const int dq = (pack >> 16) & 0xff, dc = pack >> 24;
        int q = pack & 0xff, kc = (pack >> 8) & 0xff;
#pragma unroll
        for (int j = 0; j < JMAX; ++j) {
            const size_t m = row0 + (size_t)(r7 + 8 * q);
#pragma unroll
            for (int part = 0; part < Q; ++part) {
                const int k0 = kc * KC + part * 4;
                v[j * Q + part] = (j < jc && m < (size_t)P && k0 < F)
                                      ? __ldg(reinterpret_cast<const float4 *>(imh + m * F + k0))
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            q += dq;
            kc += dc;
            if (kc >= nkc) {
                kc -= nkc;
                ++q;
            }
        }
    }

    __device__ __forceinline__ void store(uint32_t sbo, unsigned char *hi, unsigned char *lo) const {
        using S = Split<KIND>;
        const int jc = nkc * kTM / kThreads, r7 = threadIdx.x & 7;
        const int dq = (pack >> 16) & 0xff, dc = pack >> 24;
        int q = pack & 0xff, kc = (pack >> 8) & 0xff;
#pragma unroll
        for (int j = 0; j < JMAX; ++j) {
            if (j < jc) {
                const uint32_t o = (uint32_t)q * sbo + (uint32_t)kc * 128u + (uint32_t)r7 * 16u;
                float x[KC];
#pragma unroll
                for (int p = 0; p < Q; ++p) {
                    x[4 * p] = v[j * Q + p].x;
                    x[4 * p + 1] = v[j * Q + p].y;
                    x[4 * p + 2] = v[j * Q + p].z;
                    x[4 * p + 3] = v[j * Q + p].w;
                }
                typename S::T h[KC], l[KC];
#pragma unroll
                for (int p = 0; p < KC; ++p) S::run(x[p], h[p], l[p]);
                *reinterpret_cast<uint4 *>(hi + o) = *reinterpret_cast<const uint4 *>(h);
                *reinterpret_cast<uint4 *>(lo + o) = *reinterpret_cast<const uint4 *>(l);
            }
            q += dq;
            kc += dc;
            if (kc >= nkc) {
                kc -= nkc;
                ++q;
            }
        }
    }
};

template <int KIND>
__global__ void __launch_bounds__(kThreads, KIND == 0 ? 2 : 3) gates_tc_kernel(TcArgs a) {
    using S = Split<KIND>;
    constexpr int ES = S::ES;
    constexpr int KI = 32 / ES;  // K of one MMA: two core matrices
    constexpr int KC = 16 / ES;  // elements per core-matrix row
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    unsigned char *base = smem_raw + pad;
    const int NKC = a.KP / KC;                // core-matrix columns (16-byte chunks per row)
    const uint32_t sbo = (uint32_t)NKC * 128u;  // same for A and B
    const uint32_t a_bytes = (uint32_t)kTM * a.KP * ES, b_bytes = (uint32_t)a.N * a.KP * ES;
    unsigned char *Ahi = base, *Alo = base + a_bytes, *Bhi = base + 2 * a_bytes, *Blo = Bhi + b_bytes;
    float2 *ysplit = reinterpret_cast<float2 *>(Blo + b_bytes);  // [2][G]: the datum rows of this tile
    float *ea2 = reinterpret_cast<float *>(ysplit + 2 * AEM_MAX_GATES);
    float2 *llp = reinterpret_cast<float2 *>(ea2 + AEM_MAX_GATES);  // [kTM]: the second column half's sums
    uint64_t *mbar_p = reinterpret_cast<uint64_t *>(llp + kTM);
    uint32_t *slot_p = reinterpret_cast<uint32_t *>(mbar_p + 1);
    int *abort_p = reinterpret_cast<int *>(slot_p + 1);
    const uint32_t mbar = smem_u32(mbar_p);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool vec4 = (a.F & 3) == 0 && ((reinterpret_cast<uintptr_t>(a.imh) & 15) == 0);

    if (tid == 0) {
        mbar_init(mbar, 1);
        *abort_p = 0;
    }
    __syncwarp();
    if (warp == 0) tmem_alloc(smem_u32(slot_p), (uint32_t)a.ncols);
    // B = T (rows: gates, zero-padded to N; columns: frequencies, zero-padded to KP)
    for (int c = tid; c < a.N * NKC; c += kThreads) {
        const int r = (c & 7) + 8 * ((c >> 3) / NKC), kc = (c >> 3) % NKC;
        const uint32_t o = (uint32_t)(r >> 3) * sbo + (uint32_t)kc * 128u + (uint32_t)(r & 7) * 16u;
        stage_chunk<KIND>(r < a.G ? a.T + (size_t)r * a.F : nullptr, a.F, kc, false, Bhi + o, Blo + o);
    }
    if (a.eps_an)
        for (int g = tid; g < a.G; g += kThreads) ea2[g] = (float)(a.eps_an[g] * a.eps_an[g]);
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tbase = *slot_p;
    const uint32_t idesc = instr_desc(KIND == 0 ? 2u : 1u, (uint32_t)kTM, (uint32_t)a.N);
    const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo), bhi = smem_u32(Bhi), blo = smem_u32(Blo);
    const int ntiles = (a.P + kTM - 1) / kTM;
    const float em = (float)a.eps_mn;
    uint32_t phase = 0;
    bool pending = false;  // an MMA chain committed and not yet observed complete
    bool first = true;
    const bool pf_ok = vec4 && NKC * kTM / kThreads * TilePrefetch<KIND>::Q <= kPF;
    TilePrefetch<KIND> pf;
    if (pf_ok) pf.init(NKC, tid);
    if (pf_ok && (int)blockIdx.x < ntiles) pf.load(a.imh, a.P, a.F, (size_t)blockIdx.x * kTM);
    // P < 2^31 and obs_per >= 1: the datum row of model m is m / obs_per in 32-bit arithmetic
    const unsigned int obs_per = (unsigned int)a.obs_per;
    const unsigned int last_row = (unsigned int)(a.P - 1) / obs_per;

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const size_t row0 = (size_t)tile * kTM;
        // the datum rows this tile's models use, as float pairs (at most two
        // when models_per_row >= the tile; otherwise the epilogue splits per model)
        const unsigned int s0 = (unsigned int)row0 / obs_per;
        const bool split_rows = a.y_obs && obs_per >= (unsigned int)kTM;
        if (split_rows)
            for (int i = tid; i < 2 * a.G; i += kThreads) {
                const int two = i >= a.G ? 1 : 0;
                const unsigned int srow = s0 + (unsigned int)two;
                const double y = a.y_obs[(size_t)(srow <= last_row ? srow : last_row) * a.G + (i - two * a.G)];
                const float hi = (float)y;
                ysplit[i] = make_float2(hi, (float)(y - (double)hi));
            }
        // stage the tile's spectra (rows past P and columns past F are zero);
        // consecutive lanes fill consecutive 16-byte rows of one core matrix
        if (pf_ok) {
            pf.store(sbo, Ahi, Alo);
        } else {
            for (int c = tid; c < kTM * NKC; c += kThreads) {
                const int r = (c & 7) + 8 * ((c >> 3) / NKC), kc = (c >> 3) % NKC;
                const size_t m = row0 + r;
                const uint32_t o = (uint32_t)(r >> 3) * sbo + (uint32_t)kc * 128u + (uint32_t)(r & 7) * 16u;
                stage_chunk<KIND>(m < (size_t)a.P ? a.imh + m * a.F : nullptr, a.F, kc, vec4, Ahi + o, Alo + o);
            }
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        tc_after_sync();
        const bool issue = !(first && a.skip_mma);
        if (tid == 0 && issue) {
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
        first = false;
        pending = issue;
        // the next tile's loads go out while the MMA runs and the epilogue reads it
        if (pf_ok && tile + (int)gridDim.x < ntiles)
            pf.load(a.imh, a.P, a.F, (size_t)(tile + gridDim.x) * kTM);
        const bool done = mbar_wait_bounded(mbar, phase, a.spins);
        if (!done) atomicExch(abort_p, 1);
        __syncthreads();
        if (*abort_p) break;
        pending = false;
        phase ^= 1u;
        tc_after_sync();
        // epilogue: this thread's model is row 32 (warp mod 4) + lane of the
        // tile; warps 0-3 take the first half of the gate columns, 4-7 the second
        const int quarter = warp & 3, half = warp >> 2;
        const int row = quarter * 32 + lane;
        const size_t m = row0 + (size_t)row;
        const bool valid = m < (size_t)a.P;
        // with split rows the tile spans datum rows s0 and s0 + 1 at most
        const unsigned int srow =
            !valid ? 0u
                   : split_rows ? s0 + ((unsigned int)m >= (s0 + 1u) * obs_per ? 1u : 0u) : (unsigned int)m / obs_per;
        const float2 *yrow = split_rows ? ysplit + (srow - s0) * a.G : nullptr;
        const double *yd = (a.y_obs && !split_rows) ? a.y_obs + (size_t)srow * a.G : nullptr;
        LlAcc acc;
        const int c_lo = half * (a.N / 2), c_hi = c_lo + a.N / 2;
        for (int c = c_lo; c < c_hi; c += 8) {
            float v[8];
            tmem_ld8(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int g = c + q;
                if (valid && g < a.G) {
                    if (a.gates) a.gates[m * a.G + g] = v[q];
                    if (a.y_obs) {
                        float2 y;
                        if (yrow) {
                            y = yrow[g];
                        } else {
                            const double yv = yd[g];
                            y.x = (float)yv;
                            y.y = (float)(yv - (double)y.x);
                        }
                        acc.add(v[q], y, ea2[g], em);
                    }
                }
            }
        }
        if (a.ll) {
            // the two halves' (sum, error) pairs meet in shared memory, added
            // in a fixed order by the first half's thread
            if (half == 1) llp[row] = make_float2(acc.s, acc.e);
            __syncthreads();
            if (half == 0 && valid) {
                const float2 o = llp[row];
                float s1, e1;
                two_sum(acc.s, o.x, s1, e1);
                acc.s = s1;
                acc.e = (acc.e + o.y) + e1;
                a.ll[m] = acc.ll(a.G);
            }
        }
        tc_before_sync();
        __syncthreads();  // every lane read before the next chain overwrites the accumulator
    }
    if (*abort_p) {
        if (tid == 0) atomicExch(a.status, (int)AEM_ERR_TIMEOUT);
        if (pending) mbar_wait_bounded(mbar, phase);  // our own MMAs, once more with the full limit
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0) tmem_dealloc(tbase, (uint32_t)a.ncols);
}

// FP32 CUDA-core form of the same transform (for comparison): one thread per
// model, T staged in shared memory, the same FP32 likelihood terms.
__global__ void gates_fp32_kernel(TcArgs a) {
    extern __shared__ float Ts[];
    __shared__ float ea2[AEM_MAX_GATES];
    for (int i = threadIdx.x; i < a.G * a.F; i += blockDim.x) Ts[i] = a.T[i];
    if (a.eps_an)
        for (int g = threadIdx.x; g < a.G; g += blockDim.x) ea2[g] = (float)(a.eps_an[g] * a.eps_an[g]);
    __syncthreads();
    const float em = (float)a.eps_mn;
    for (size_t m = (size_t)blockIdx.x * blockDim.x + threadIdx.x; m < (size_t)a.P; m += (size_t)gridDim.x * blockDim.x) {
        const float *x = a.imh + m * a.F;
        const double *y = a.y_obs ? a.y_obs + (m / (size_t)a.obs_per) * a.G : nullptr;
        LlAcc acc;
        for (int g = 0; g < a.G; ++g) {
            float s = 0.f;
            for (int k = 0; k < a.F; ++k) s = fmaf(Ts[g * a.F + k], x[k], s);
            if (a.gates) a.gates[m * a.G + g] = s;
            if (y) {
                const float hi = (float)y[g];
                acc.add(s, make_float2(hi, (float)(y[g] - (double)hi)), ea2[g], em);
            }
        }
        if (a.ll) a.ll[m] = acc.ll(a.G);
    }
}

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

int gates_from_spectrum(const aem_system *sys, const float *imh, int P, int mode, const double *y_obs,
                        int obs_per, const double *eps_an, double eps_mn, float *gates, double *ll,
                        cudaStream_t stream) {
    const SystemTables &h = sys->host;
    TcArgs a{imh, P, h.F, h.G, 0, 0, 0, sys->d_T_f, y_obs, obs_per > 0 ? obs_per : 1, eps_an, eps_mn, gates, ll,
             sys->d_status, sys->wait_spins ? sys->wait_spins : kSpinLimit, sys->wait_skip_mma};
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
    const size_t smem = (size_t)2 * (kTM + a.N) * a.KP * ES + 1024 + sizeof(float2) * 2 * AEM_MAX_GATES +
                        sizeof(float) * AEM_MAX_GATES + sizeof(float2) * kTM + 64;
    auto kern = tf32 ? gates_tc_kernel<0> : gates_tc_kernel<1>;
    AEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // all of the SM's unified storage to shared memory, so that several CTAs
    // (two for the TF32 split's 84 KB, five for the BF16 split's 43 KB) stay resident
    AEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    int per_sm = 0;
    AEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1) return fail(AEM_ERR_UNSUPPORTED, "aem_gates_from_spectrum: tile does not fit in shared memory");
    // the occupancy query has reported one CTA per SM for the TF32 tile where
    // two fit (the profiler's shared-memory limit says two); take the count
    // the SM's shared memory, registers and tensor memory allow when it is larger
    {
        int smem_sm = 0, reserved = 0;
        AEM_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, sys->device));
        AEM_CUDA_TRY(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, sys->device));
        cudaFuncAttributes fa{};
        AEM_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
        int by_smem = smem_sm / (int)(smem + (size_t)reserved);
        const int by_regs = fa.numRegs > 0 ? 65536 / (fa.numRegs * kThreads) : 1;
        const int by_tmem = 512 / a.ncols;
        if (by_smem > by_regs) by_smem = by_regs;
        if (by_smem > by_tmem) by_smem = by_tmem;
        if (by_smem > per_sm) per_sm = by_smem;
    }
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

extern "C" int aem_debug_bounded_wait(aem_system *sys, unsigned int spins, int skip_first_mma) {
    if (!sys || (skip_first_mma != 0 && skip_first_mma != 1))
        return fail(AEM_ERR_INVALID_ARG, "aem_debug_bounded_wait: NULL system or skip_first_mma not 0 / 1");
    sys->wait_spins = spins;
    sys->wait_skip_mma = skip_first_mma;
    return AEM_OK;
}

extern "C" int aem_system_status(const aem_system *sys, int *status) {
    if (!sys || !status) return fail(AEM_ERR_INVALID_ARG, "aem_system_status: NULL argument");
    int v = 0;
    AEM_CUDA_TRY(cudaMemcpy(&v, sys->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) AEM_CUDA_TRY(cudaMemset(sys->d_status, 0, sizeof(int)));
    *status = v;
    return AEM_OK;
}
