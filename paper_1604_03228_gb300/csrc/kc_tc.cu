// kc_tc.cu -- tensor-core (tcgen05) distance blocks for the dense n x k
// work: the covering radius of a center set (solution value, Section 7) and
// EIM's prune of R against the sample S (Algorithm 2, the round Section 5.2
// finds dominant).
//
// Operands.  Points and centers are scaled by 2^e (an exact scaling, e chosen
// so that every |coordinate| <= 2^S with d 2^(2S) <= 2^30 and S <= 14) and
// rounded to fp16: x~, c~.  e comes from the largest |coordinate|: a pass over
// packed points, or for row-major points a sample of every 64th row that the
// tile pass checks against every value (a fix-up pass redoes the tiles with
// the true maximum when the sample fell short).  A prep pass writes them once as MMA tiles (128
// point rows or 256 center rows by Kp = d + 3 rounded up to 16) in the
// shared-memory operand layout, with per-row |x~|^2 and error bound
// e = ||x~ - 2^e x|| (FP32, rounded up).  The tiles carry the norm term too:
// a point row is (x~, 2^15, 2^4, 2^-7, 0...), a center row (2 c~, p1, p2, p3,
// 0...) with p1 2^15 + p2 2^4 + p3 2^-7 = -|c~|^2 up to a residual r_c
// (fp16 pieces taken in turn from the FP32 norm, r_c computed exactly), so
// the accumulator itself is v = 2 x~.c~ - |c~|^2 and s~ = |x~|^2 - v
// approximates ||x~ - c~||^2.  Rows past the count are zero (points) or
// carry -inf pieces (centers: v = -inf, never a maximum or within a limit).
//
// Kernel.  One persistent CTA per SM (it holds all 512 TMEM columns).  Warps:
//   8    producer: cp.async.bulk of point tiles (2-stage ring) and center
//        tiles (all of them once when they fit, else a 2-stage ring) into
//        shared memory
//   9    MMA issuer (one thread): tcgen05.mma.kind::f16, M=128 x N=256,
//        Kp/16 instructions per tile pair, FP32 accumulators double-buffered
//        in TMEM (2 x 256 columns)
//   0-7  epilogue: warps w and w+4 own point rows 32(w%4).. (their TMEM
//        lanes) and split the 256 columns; each thread loads its 128 columns
//        as four 32-column loads behind one wait, releases the accumulator
//        after that single round trip, and folds v into a running maximum
//        three values at a time (radius) or compares it with the point's two
//        decision limits (prune).
// With streamed centers (the prune; the radius when the centers do not fit)
// tc_dmin2_kernel takes two point tiles per center tile instead, so that a
// center tile read from L2 feeds two MMAs (see there).
// Shared-memory operand layout: no swizzle, K-major, 8 x 16-byte core
// matrices; core matrix (row block mi, column block ki) of an R-row tile at
// byte ((ki * R/8) + mi) * 128: the descriptor's leading (K) byte offset is
// R/8 * 128 and its stride (M/N) byte offset 128.
//
// Error bound.  fp16 products are exact; the FP32 accumulation (whose terms
// sum in magnitude to at most |x~|^2 + 2 |c~|^2), the norms and the split
// are covered by
//   |s~ - ||x~ - c~||^2| <= eta (|x~|^2 + 2 |c~|^2) + max r_c,
//   eta = g_d + (Kp+16) 2^-21 + 2^-21
// (a deliberately loose model of the tensor core's accumulation).  With the
// triangle inequality ||x - c|| in ||x~ - c~|| -+ (e_x + e_c) (scaled units)
// and the canonical FP32 value within (1 +- g_d) of the exact one, every
// decision is taken on bounds that contain the canonical FP32 value; the
// undecided cases are recomputed exactly from the FP32 coordinates.
#include <cuda_fp16.h>

#include "kc_internal.cuh"

namespace kc {

// Diagnostics of the tensor-core blocks (since the last read): [0] exact pair
// checks of undecided pairs, [1] points processed (prune); clock cycles of
// the MMA-issuing thread, summed over CTAs (radius and prune): [2] waiting
// for a center tile, [3] for a free accumulator, [4] for a point tile, [5] in
// all.
__device__ unsigned long long g_tc_counters[6];

// Cycle counts of an MMA issuer's waits, added to g_tc_counters[2..5] once.
struct MmaClock {
    long long t0, wb, wt, wa;
    __device__ __forceinline__ void start() {
        t0 = clock64();
        wb = wt = wa = 0;
    }
    __device__ __forceinline__ void publish() {
        atomicAdd(&g_tc_counters[2], (unsigned long long)wb);
        atomicAdd(&g_tc_counters[3], (unsigned long long)wt);
        atomicAdd(&g_tc_counters[4], (unsigned long long)wa);
        atomicAdd(&g_tc_counters[5], (unsigned long long)(clock64() - t0));
    }
};

namespace {

constexpr int TC_M = 128;
constexpr int TC_N = 256;
// 8 epilogue warps: with the producer and MMA warps the CTA has 10, at most 3
// per SM sub-partition, which leaves up to 168 registers per thread.
constexpr int TC_EPI_WARPS = 8;                     // epilogue warps 0-7
constexpr int TC_GROUPS = TC_EPI_WARPS / 4;          // column groups per accumulator row
constexpr int TC_COLS = TC_N / TC_GROUPS;            // columns of a tile per epilogue thread
constexpr int TC_PROD = TC_EPI_WARPS;                // producer warp
constexpr int TC_MMA = TC_EPI_WARPS + 1;             // MMA warp
constexpr int TC_THREADS = (TC_EPI_WARPS + 2) * 32;
constexpr int TC_EPI = TC_EPI_WARPS * 32;
static_assert(TC_COLS % 32 == 0, "whole 32-column TMEM loads");
constexpr int TC_KMAX = 128;
constexpr long long TC_SPIN = 1ll << 32;   // wait budget in clock cycles (about two seconds)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version for this architecture; no swizzle
    return d;
}

// kind::f16 instruction descriptor: FP32 accumulate, fp16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(b)),
                 "r"(bytes)
                 : "memory");
}
// Wait for the phase with the given parity; false if the cycle budget ran
// out or another role gave up (*abort set).
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, volatile int *abort) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(smem_u32(b)), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (*abort || clock64() - t0 > TC_SPIN) return false;
    }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                 "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
// One accumulation chain of KS MMAs (K = 16 each) into d: A and B start at
// descriptors ad and bd and advance by ainc / binc (the next K step's start
// address, in the descriptor's 16-byte units; the start field cannot carry:
// shared-memory addresses stay below 2^18 bytes).  The single issuing thread
// does almost nothing between MMAs: rebuilding both 64-bit descriptors per
// MMA in a runtime loop took as long as the MMA itself (a 128 x 256 x 16
// block is about 135 SM clocks) and held the tensor pipe near half its rate.
template <int KS>
__device__ __forceinline__ void umma_chain(uint32_t d, uint64_t ad, uint64_t bd, uint64_t ainc, uint64_t binc,
                                           uint32_t idesc) {
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) umma_f16(d, ad + kk * ainc, bd + kk * binc, idesc, kk > 0 ? 1u : 0u);
}
// The chain for Kp / 16 = ks K steps (1..9: Kp = d + 3 rounded up to 16, d <= 128).
__device__ __forceinline__ void umma_chain_k(int ks, uint32_t d, uint64_t ad, uint64_t bd, uint64_t ainc,
                                             uint64_t binc, uint32_t idesc) {
    switch (ks) {
        case 1: umma_chain<1>(d, ad, bd, ainc, binc, idesc); break;
        case 2: umma_chain<2>(d, ad, bd, ainc, binc, idesc); break;
        case 3: umma_chain<3>(d, ad, bd, ainc, binc, idesc); break;
        case 4: umma_chain<4>(d, ad, bd, ainc, binc, idesc); break;
        case 5: umma_chain<5>(d, ad, bd, ainc, binc, idesc); break;
        case 6: umma_chain<6>(d, ad, bd, ainc, binc, idesc); break;
        case 7: umma_chain<7>(d, ad, bd, ainc, binc, idesc); break;
        case 8: umma_chain<8>(d, ad, bd, ainc, binc, idesc); break;
        default: umma_chain<9>(d, ad, bd, ainc, binc, idesc); break;
    }
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive accumulator columns of this thread's TMEM lane; the
// registers are valid after tmem_wait_ld on them.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
// Wait for this thread's outstanding TMEM loads; r is named as read and
// written so that no use of it moves above the wait.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// After tmem_wait_ld on another array: keeps every use of r below that wait
// (volatile asm statements keep their order).
__device__ __forceinline__ void tmem_pin(uint32_t (&r)[32]) {
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31]));
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Element offset of (row r, coordinate k) in an R-row no-swizzle K-major tile.
__host__ __device__ __forceinline__ int core_off(int R, int r, int k) {
    return ((k >> 3) * (R >> 3) + (r >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// Largest exponent S with d 2^(2S) <= 2^30 (so |c~|^2 <= 2^30 and its first
// fp16 piece fits after the 2^-15 shift), and S <= 14 (2 c~ stays in fp16).
__host__ __device__ __forceinline__ int tc_sexp(int d) {
    int lg = 0;
    while ((1 << lg) < d) ++lg;   // ceil(log2 d)
    const int S = (30 - lg) / 2;
    return S < 14 ? S : 14;
}

// Scale 2^e with max|coordinate| * 2^e <= 2^S (1 for an all-zero input).
__device__ __forceinline__ float tc_scale(const unsigned *absmax, int d) {
    const float m = __uint_as_float(*absmax);
    if (!(m > 0.f)) return 1.f;
    int ex;
    frexpf(m, &ex);                        // m = f 2^ex, f in [0.5, 1): m < 2^ex
    return ldexpf(1.f, tc_sexp(d) - ex);   // m 2^(S-ex) < 2^S
}

// ------------------------------------------------------------------ prep
__global__ void tc_absmax_kernel(const float *__restrict__ pk, int64_t n, int d, unsigned *absmax) {
    float m = 0.f;
    const int64_t total = nblocks(n) * (int64_t)d * BLK;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(pk[e]));   // padding is zero
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(absmax, __float_as_uint(m));
}

// Row-major points: the scale comes from a sample, the largest finite
// |coordinate| of every TC_SAMPLE-th row, doubled (one power of two of
// headroom), into words[1].  The tile pass below checks every value against
// it and a fix-up pass redoes the tiles in the rare case that the sample
// missed a larger magnitude, so the scale always covers every coordinate.
constexpr int TC_SAMPLE = 64;
__global__ void tc_absmax_sample_kernel(const float *__restrict__ rm, int64_t n, int d, unsigned *words) {
    float m = 0.f;
    const int64_t total = (n + TC_SAMPLE - 1) / TC_SAMPLE * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / d;
        const float v = __ldg(rm + r * TC_SAMPLE * d + (e - r * d));
        if (isfinite(v)) m = fmaxf(m, fabsf(v));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&words[1], __float_as_uint(2.f * m));
}

// Checks of one value as the pack performs them: NaN/Inf (KC_ERR_NONFINITE),
// else |v| > 2^54 (KC_ERR_RANGE; squared distances then stay far below
// FLT_MAX); m keeps the largest magnitude.
__device__ __forceinline__ void absmax_check(float v, float &m, bool &bad, bool &nonfin) {
    m = fmaxf(m, fabsf(v));
    if (!(fabsf(v) <= 0x1p54f)) bad = true;   // NaN fails the comparison
    if (!isfinite(v)) nonfin = true;
}

// Does the scale taken from A (tc_scale: 2^(S - e), A < 2^e) keep every
// coordinate of magnitude at most T within 2^S?
__device__ __forceinline__ bool scale_covers(unsigned a_bits, unsigned t_bits) {
    const float A = __uint_as_float(a_bits), T = __uint_as_float(t_bits);
    if (!(T > 0.f)) return true;
    if (!(A > 0.f)) return false;
    int ea, et;
    frexpf(A, &ea);
    frexpf(T, &et);
    return et <= ea;
}

// Point tiles straight from the row-major array (the pack's work folded in):
// a CTA stages a tile's rows, one contiguous span of rm, in shared memory
// (scaled, row stride ld = d | 1, so the per-row reads below are free of bank
// conflicts), then threads 0..127 compute their row's norm and rounding bound
// and all threads write the fp16 tile, one 16-byte core-matrix row per store.
// Values and rounding are those of tc_rows_kernel<TC_M> on the same points.
// words: [0] the scale word every later kernel reads, [1] the sampled one,
// [2] the true largest magnitude.  First pass (FIX false): scale from [1];
// every value checked as the pack does and its magnitude folded into [2].
// Fix-up pass (FIX true): [0] = [1] when it covers [2] (nothing else to
// do), else [0] = [2] and the tiles are redone with that scale.
constexpr int TC_RM_NT = 256;
constexpr int TC_RM_V = 8;   // a 128 x 64 FP32 tile is 8 loads per thread
template <bool FIX>
__global__ void __launch_bounds__(TC_RM_NT) tc_points_rm_kernel(const float *__restrict__ rm, int64_t n, int d,
                                                                 bool vec, int kp, int64_t ntiles, unsigned *words,
                                                                 DevStatus *st, __half *__restrict__ tiles,
                                                                 float *__restrict__ norm, float *__restrict__ err) {
    extern __shared__ float sx[];   // [TC_M][ld]
    const int ld = d | 1;
    const int tid = threadIdx.x;
    if (FIX) {
        const bool covered = scale_covers(words[1], words[2]);
        if (blockIdx.x == 0 && tid == 0) words[0] = covered ? words[1] : words[2];
        if (covered) return;
    }
    const float sc = tc_scale(&words[FIX ? 2 : 1], d);
    float m = 0.f;
    bool bad = false, nonfin = false;
    // f / d as a multiply-high: exact for f < 2^14 (a tile's TC_M * d <= 2^14
    // elements) and d <= 2^7
    const uint64_t dmag = 0xFFFFFFFFull / (uint64_t)d + 1;
    auto row_of = [&](int f) { return (int)(((uint64_t)(uint32_t)f * dmag) >> 32); };
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * TC_M;
        const int rows = (int)((n - p0) < TC_M ? (n - p0) : TC_M);
        const float *base = rm + p0 * (int64_t)d;
        const int total = rows * d;
        const int nv = vec ? total / 4 : 0;
        __syncthreads();   // the previous tile's reads are done
        // TC_RM_V 16-byte loads per thread in flight before any is stored
        for (int q0 = 0; q0 < nv; q0 += TC_RM_V * TC_RM_NT) {
            float4 w[TC_RM_V];
#pragma unroll
            for (int v = 0; v < TC_RM_V; ++v) {
                const int q = q0 + v * TC_RM_NT + tid;
                if (q < nv) w[v] = __ldg(reinterpret_cast<const float4 *>(base) + q);
            }
#pragma unroll
            for (int v = 0; v < TC_RM_V; ++v) {
                const int q = q0 + v * TC_RM_NT + tid;
                if (q >= nv) break;
                const float vv[4] = {w[v].x, w[v].y, w[v].z, w[v].w};
                const int f = 4 * q;
                int r = row_of(f), j = f - r * d;
                if (!FIX) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) absmax_check(vv[u], m, bad, nonfin);
                }
                if ((d & 3) == 0) {   // the four values share a row
                    float *dst = sx + r * ld + j;
#pragma unroll
                    for (int u = 0; u < 4; ++u) dst[u] = __fmul_rn(vv[u], sc);   // exact
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        sx[r * ld + j] = __fmul_rn(vv[u], sc);
                        if (++j == d) {
                            j = 0;
                            ++r;
                        }
                    }
                }
            }
        }
        for (int f = 4 * nv + tid; f < total; f += TC_RM_NT) {
            const int r = row_of(f), j = f - r * d;
            const float v = __ldg(base + f);
            if (!FIX) absmax_check(v, m, bad, nonfin);
            sx[r * ld + j] = __fmul_rn(v, sc);
        }
        for (int f = total + tid; f < TC_M * d; f += TC_RM_NT) {
            const int r = row_of(f), j = f - r * d;
            sx[r * ld + j] = 0.f;
        }
        __syncthreads();
        if (tid < TC_M) {
            const bool valid = tid < rows;
            float nrm = 0.f, e2 = 0.f;
#pragma unroll 8
            for (int k = 0; k < d; ++k) {
                const float x = sx[tid * ld + k];
                const float xq = __half2float(__float2half_rn(x));
                const float df = fabsf(__fsub_rn(x, xq));   // exact (Sterbenz) or x itself
                e2 = __fmaf_ru(df, df, e2);
                nrm = __fmaf_rn(xq, xq, nrm);
            }
            norm[p0 + tid] = valid ? nrm : INFINITY;
            err[p0 + tid] = valid ? __fsqrt_ru(e2) : 0.f;
        }
        __half *tile = tiles + t * (int64_t)TC_M * kp;
        const int chunks = TC_M * (kp / 8);
        for (int c = tid; c < chunks; c += TC_RM_NT) {
            const int r = c % TC_M, k0 = (c / TC_M) * 8;
            uint32_t h[4];
            if (k0 + 8 <= d) {   // coordinates only
                const float *row = sx + r * ld + k0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const __half2 q = __floats2half2_rn(row[2 * u], row[2 * u + 1]);
                    h[u] = *reinterpret_cast<const uint32_t *>(&q);
                }
                *reinterpret_cast<uint4 *>(tile + core_off(TC_M, r, k0)) = make_uint4(h[0], h[1], h[2], h[3]);
                continue;
            }
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                __half q2[2];
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    const int k = k0 + u + v;
                    float x = 0.f;
                    if (k < d) x = sx[r * ld + k];
                    else if (k == d) x = 32768.f;
                    else if (k == d + 1) x = 16.f;
                    else if (k == d + 2) x = 0.0078125f;
                    q2[v] = __float2half_rn(x);
                }
                h[u / 2] = (uint32_t)__half_as_ushort(q2[0]) | ((uint32_t)__half_as_ushort(q2[1]) << 16);
            }
            *reinterpret_cast<uint4 *>(tile + core_off(TC_M, r, k0)) = make_uint4(h[0], h[1], h[2], h[3]);
        }
    }
    if (!FIX) {
#pragma unroll
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        if ((tid & 31) == 0) atomicMax(&words[2], __float_as_uint(m));
        if (nonfin) set_status(st, KC_ERR_NONFINITE, 1, 0);
        else if (bad) set_status(st, KC_ERR_RANGE, 1, 0);
    }
}

// Rows -> fp16 MMA tiles of R rows.  Row i is a point or center: from the
// packed array (pk) when pk != null, else row idx ? idx[i] : i of the
// row-major array rm.  Point tiles (R = TC_M) append the multipliers
// (2^15, 2^4, 2^-7) at columns d, d+1, d+2; center tiles (R = TC_N) store
// 2 c~ and the three fp16 pieces of -|c~|^2 there.  Rows past the count:
// zero coordinates, -inf pieces (centers), norm +inf.  maxes (optional) gets
// the largest e, the largest norm and the largest split residual r_c.  rin
// (optional, with idx and inS): per row, inS[idx[i]] (0 past the count).
template <int R>
__global__ void tc_rows_kernel(const float *__restrict__ pk, const float *__restrict__ rm,
                               const uint32_t *__restrict__ idx, const int32_t *cnt_dev, int64_t cnt_max, int d,
                               int kp, int64_t ntiles, const unsigned *absmax, __half *__restrict__ tiles,
                               float *__restrict__ norm, float *__restrict__ err, unsigned *maxes,
                               const uint8_t *__restrict__ inS, uint8_t *__restrict__ rin) {
    constexpr bool CENTER = R == TC_N;
    const int64_t cnt = dev_count(cnt_dev, cnt_max);
    const float sc = tc_scale(absmax, d);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ntiles * R;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / R;
        const int r = (int)(i % R);
        __half *tile = tiles + t * (int64_t)R * kp;
        const bool valid = i < cnt;
        int64_t g = 0;
        if (valid) g = pk ? i : (idx ? (int64_t)idx[i] : i);
        // coordinates first: norm and rounding bound
        float nrm = 0.f, e2 = 0.f;
        for (int k = 0; k < d; ++k) {
            const float x = valid ? __fmul_rn(pk ? pk[pk_index(g, k, d)] : rm[g * d + k], sc) : 0.f;   // exact
            const float xq = __half2float(__float2half_rn(x));
            const float df = fabsf(__fsub_rn(x, xq));   // exact (Sterbenz) or x itself
            e2 = __fmaf_ru(df, df, e2);
            nrm = __fmaf_rn(xq, xq, nrm);
        }
        // the norm columns
        __half aug[3];
        float resid = 0.f;
        if (!CENTER) {
            aug[0] = __float2half_rn(32768.f);
            aug[1] = __float2half_rn(16.f);
            aug[2] = __float2half_rn(0.0078125f);
        } else if (!valid) {
            aug[0] = aug[1] = aug[2] = __float2half_rn(-INFINITY);
        } else {
            // -|c~|^2 = p1 2^15 + p2 2^4 + p3 2^-7 + residual; each piece is the
            // fp16 rounding of what is left (|c~|^2 <= 2^30, so no piece overflows)
            const double v = -(double)nrm;
            aug[0] = __float2half_rn((float)(v * 0x1p-15));
            const double r1 = v - (double)__half2float(aug[0]) * 0x1p15;
            aug[1] = __float2half_rn((float)(r1 * 0x1p-4));
            const double r2 = r1 - (double)__half2float(aug[1]) * 0x1p4;
            aug[2] = __float2half_rn((float)(r2 * 0x1p7));
            const double r3 = r2 - (double)__half2float(aug[2]) * 0x1p-7;
            resid = __double2float_ru(fabs(r3));
        }
        // one 16-byte core-matrix row (8 columns) per store; consecutive rows
        // of a warp store consecutive 16-byte chunks
        for (int k0 = 0; k0 < kp; k0 += 8) {
            uint32_t w[4];
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                __half q2[2];
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    const int k = k0 + u + v;
                    __half q = __float2half_rn(0.f);
                    if (k < d) {
                        if (valid) {
                            q = __float2half_rn(__fmul_rn(pk ? pk[pk_index(g, k, d)] : rm[g * d + k], sc));
                            if (CENTER) q = __hadd(q, q);   // 2 c~, exact
                        }
                    } else if (k < d + 3) {
                        q = aug[k - d];
                    }
                    q2[v] = q;
                }
                w[u / 2] = (uint32_t)__half_as_ushort(q2[0]) | ((uint32_t)__half_as_ushort(q2[1]) << 16);
            }
            *reinterpret_cast<uint4 *>(tile + core_off(R, r, k0)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        const float e = __fsqrt_ru(e2);
        norm[i] = valid ? nrm : INFINITY;
        err[i] = valid ? e : 0.f;
        if (rin) rin[i] = valid && inS[g] != 0 ? 1 : 0;
        if (maxes && valid) {
            atomicMax(&maxes[0], __float_as_uint(e));
            atomicMax(&maxes[1], __float_as_uint(nrm));
            atomicMax(&maxes[2], __float_as_uint(resid));
        }
    }
}

struct TcArgs {
    int d, kp, kc, ntiles;      // centers: kc real of ntiles * TC_N rows
    int resident;               // all center tiles stay in shared memory (loaded once)
    int64_t npts;               // points (rows of the A tiles)
    const __half *at;           // point tiles [ceil(npts/128)][128 x kp]
    const float *an, *ae;       // point norms and bounds
    const __half *bt;           // center tiles [ntiles][256 x kp]
    const float *cn;            // center norms [ntiles * 256]
    const unsigned *maxes;      // [0] = E (max e_c), [1] = max |c~|^2, [2] = max r_c (float bits), scaled units
    const unsigned *absmax;     // max |coordinate| (float bits), for the scale
    // radius
    float *mlo, *mhi;           // per-point bounds on the canonical minimum (unscaled)
    unsigned *mlo_max;
    // prune
    const float *src;           // row-major FP32 points
    const uint32_t *R;          // point indices of the rows
    const uint8_t *rin;         // per point row: the point is sampled (always removed)
    const float *cen;           // FP32 center rows (exact rechecks)
    const uint32_t *thr;        // threshold (canonical FP32 bits)
    uint32_t *Rn;               // kept points
    unsigned long long *rnn;
    uint2 *pairs;               // undecided (row, center) pairs
    int64_t pcap;
    unsigned long long *npairs;
    uint8_t *pflag;             // per row: bit 0 pairs deferred, bit 1 pair buffer overflowed
    uint32_t *pend;             // rows decided by the pair check
    unsigned long long *npend;
    DevStatus *st;
};

__device__ __forceinline__ float tc_eta(int d, int kp) {
    return (float)(f32_gamma(d) + (double)(kp + 16) * 0x1p-21 + 0x1p-21);
}

// Launch bounds of 384 threads for a 320-thread launch: they cap the
// registers at 168 per thread, so that the SM sub-partition holding three of
// the ten warps has room for them (3 x 32 x 168 <= 16384).
template <int MODE>
__global__ void __launch_bounds__(384, 1) tc_dmin_kernel(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int kp = a.kp;
    const uint32_t a_bytes = (uint32_t)TC_M * kp * 2, b_bytes = (uint32_t)TC_N * kp * 2;
    // point tiles at smem + stage * a_bytes, center tiles after them
    unsigned char *const sAb = smem, *const sBb = smem + 2 * a_bytes;
    __shared__ __align__(8) uint64_t a_full[2], a_empty[2], b_full[2], b_empty[2], t_full[2], t_empty[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    __shared__ float s_part[TC_GROUPS][TC_M];
    __shared__ int s_gone[TC_M];   // prune: the row is surely within the threshold
    __shared__ int s_pend[TC_M];   // prune: another group deferred pairs (bit 0) or overflowed (bit 1)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntile_pts = (a.npts + TC_M - 1) / TC_M;
    volatile int *abort = &s_abort;

    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&a_full[s], 1);
            mbar_init(&a_empty[s], 1);
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1);
            mbar_init(&t_full[s], 1);
            mbar_init(&t_empty[s], TC_EPI);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < TC_M) {
        s_gone[tid] = 0;
        s_pend[tid] = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == TC_PROD) {
        // ------------------------------------------------ producer
        if (lane == 0) {
            uint32_t afill = 0, bfill = 0;   // bit s: parity of stage s's fills so far
            int64_t u = 0, p = 0;
            for (int64_t pt = blockIdx.x; pt < ntile_pts && !*abort; pt += gridDim.x, ++p) {
                const int sa = (int)(p & 1);
                if (!mbar_wait(&a_empty[sa], ((afill >> sa) & 1u) ^ 1u, abort)) {
                    *abort = 1;
                    set_status(a.st, KC_ERR_TIMEOUT, 6, 0);
                    break;
                }
                mbar_expect_tx(&a_full[sa], a_bytes);
                bulk_g2s(sAb + sa * a_bytes, a.at + pt * (int64_t)TC_M * kp, a_bytes, &a_full[sa]);
                afill ^= 1u << sa;
                if (a.resident) {
                    if (p == 0) {   // every center tile, once, behind the first point tile
                        mbar_expect_tx(&b_full[0], (uint32_t)a.ntiles * b_bytes);
                        for (int t = 0; t < a.ntiles; ++t)
                            bulk_g2s(sBb + t * b_bytes, a.bt + (int64_t)t * TC_N * kp, b_bytes, &b_full[0]);
                    }
                    continue;
                }
                for (int t = 0; t < a.ntiles; ++t, ++u) {
                    const int s = (int)(u & 1);
                    if (!mbar_wait(&b_empty[s], ((bfill >> s) & 1u) ^ 1u, abort)) {
                        *abort = 1;
                        set_status(a.st, KC_ERR_TIMEOUT, 6, t);
                        break;
                    }
                    mbar_expect_tx(&b_full[s], b_bytes);
                    bulk_g2s(sBb + s * b_bytes, a.bt + (int64_t)t * TC_N * kp, b_bytes, &b_full[s]);
                    bfill ^= 1u << s;
                }
            }
        }
    } else if (warp == TC_MMA) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = umma_idesc_f16(TC_M, TC_N);
            const uint32_t a_lbo = (TC_M / 8) * 128, b_lbo = (TC_N / 8) * 128;
            // one K step = two core-matrix columns, in 16-byte descriptor units
            const uint64_t ainc = (2 * a_lbo) >> 4, binc = (2 * b_lbo) >> 4;
            uint32_t ause = 0, buse = 0, tuse = 0;   // bit s: parity of stage s's uses so far
            int64_t u = 0, p = 0;
            MmaClock clk;
            clk.start();
            for (int64_t pt = blockIdx.x; pt < ntile_pts && !*abort; pt += gridDim.x, ++p) {
                const int sa = (int)(p & 1);
                long long c0 = clock64();
                if (!mbar_wait(&a_full[sa], (ause >> sa) & 1u, abort)) {
                    *abort = 1;
                    set_status(a.st, KC_ERR_TIMEOUT, 7, 0);
                    break;
                }
                clk.wa += clock64() - c0;
                for (int t = 0; t < a.ntiles; ++t, ++u) {
                    const int s = (int)(u & 1);
                    // resident center tiles: one barrier phase, completed once
                    c0 = clock64();
                    const bool bok = a.resident ? (p > 0 || t > 0 || mbar_wait(&b_full[0], 0u, abort))
                                                : mbar_wait(&b_full[s], (buse >> s) & 1u, abort);
                    const long long c1 = clock64();
                    clk.wb += c1 - c0;
                    const bool tok = mbar_wait(&t_empty[s], ((tuse >> s) & 1u) ^ 1u, abort);
                    clk.wt += clock64() - c1;
                    if (!tok || !bok) {
                        *abort = 1;
                        set_status(a.st, KC_ERR_TIMEOUT, 8, t);
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t ad = umma_desc(smem_u32(sAb + sa * a_bytes), a_lbo, 128);
                    const uint64_t bd = umma_desc(smem_u32(sBb + (a.resident ? t : s) * b_bytes), b_lbo, 128);
                    umma_chain_k(kp / 16, tmem + (uint32_t)(s * TC_N), ad, bd, ainc, binc, idesc);
                    if (!a.resident) umma_commit(&b_empty[s]);
                    umma_commit(&t_full[s]);
                    buse ^= 1u << s;
                    tuse ^= 1u << s;
                }
                umma_commit(&a_empty[sa]);
                ause ^= 1u << sa;
            }
            clk.publish();
        }
    } else {
        // ------------------------------------------------ epilogue warps
        // warp w reads TMEM lanes 32 (w % 4) .. (its accumulator rows) and
        // the columns of group w / 4; each thread owns one row and TC_COLS
        // columns of every tile
        const int row = (warp & 3) * 32 + lane;
        const int grp = warp >> 2;
        const float sc = tc_scale(a.absmax, a.d);
        const float sc2 = sc * sc;                  // exact power of two
        const float isc2 = 1.f / sc2;               // exact power of two
        const float eta = tc_eta(a.d, kp);
        const float g = lp_slack(a.d);
        const float E = __uint_as_float(a.maxes[0]);
        const float cnmax2 = __fmul_ru(2.f, __uint_as_float(a.maxes[1]));
        const float rmax = __uint_as_float(a.maxes[2]);
        uint32_t tuse = 0;   // bit s: parity of TMEM stage s's uses so far
        int64_t u = 0;
        // the row's norm, bound, index and sample flag are loaded one point
        // tile ahead, so that no global load waits at the top of a tile
        float nx_n = 0.f, ae_n = 0.f;
        uint32_t gx_n = 0, in_n = 0;
        auto fetch = [&](int64_t pt) {
            const int64_t pi = pt * TC_M + row;
            if (pt < ntile_pts && pi < a.npts) {
                nx_n = a.an[pi];
                ae_n = a.ae[pi];
                if (MODE == 1) {
                    gx_n = a.R[pi];
                    in_n = a.rin[pi];
                }
            }
        };
        fetch(blockIdx.x);
        float lomax = 0.f;              // radius: largest lower bound of this thread's rows
        unsigned long long nrows = 0;   // prune: rows processed (diagnostics)
        for (int64_t pt = blockIdx.x; pt < ntile_pts; pt += gridDim.x) {
            const int64_t pi = pt * TC_M + row;
            const bool valid = pi < a.npts;
            const float xn = valid ? nx_n : 0.f;
            const float sl = __fadd_ru(valid ? ae_n : 0.f, E);
            const float eps = __fadd_ru(__fmul_ru(eta, __fadd_ru(xn, cnmax2)), rmax);
            int64_t gx = 0;
            bool removed = !valid;
            if (MODE == 1 && valid) {
                gx = (int64_t)gx_n;
                removed = in_n != 0;
            }
            fetch(pt + gridDim.x);
            float vlo = INFINITY, vhi = INFINITY;
            if (MODE == 1 && valid) {
                // s~ = xn - v; v >= vlo: s~ small enough that d(x,c) <= thr
                // surely; v < vhi: d(x,c) > thr surely; between: exact check
                const float thr = __fmul_rn(__uint_as_float(*a.thr), sc2);   // scaled, exact
                const float ra = __fsub_rd(__fsqrt_rd(__fdiv_rd(thr, __fadd_ru(1.f, g))), sl);
                const float lo_lim = ra > 0.f ? __fsub_rd(__fmul_rd(ra, ra), eps) : -1.f;
                const float rb = __fadd_ru(__fsqrt_ru(__fdiv_ru(thr, __fsub_rd(1.f, g))), sl);
                const float hi_lim = __fadd_ru(__fmul_ru(rb, rb), eps);
                vlo = lo_lim >= 0.f ? __fsub_ru(xn, lo_lim) : INFINITY;
                vhi = __fsub_rd(xn, hi_lim);
            }
            float v0 = -INFINITY, v1 = -INFINITY, v2 = -INFINITY, v3 = -INFINITY;
            unsigned long long namb = 0;
            bool emitted = false, ovf = false;
            volatile int *s_gone_v = s_gone;
            int cbase = 0;
            // One 32-column chunk of accumulators v (columns cbase + c0 ..),
            // folded into running maxima three values at a time.
            auto chunk = [&](const uint32_t(&r)[32], int c0) {
                if (MODE == 0) {
#pragma unroll
                    for (int j = 0; j < 32; j += 8) {
                        v0 = max3f(v0, __uint_as_float(r[j]), __uint_as_float(r[j + 1]));
                        v1 = max3f(v1, __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
                        v2 = max3f(v2, __uint_as_float(r[j + 4]), __uint_as_float(r[j + 5]));
                        v3 = max3f(v3, __uint_as_float(r[j + 6]), __uint_as_float(r[j + 7]));
                    }
                } else if (!removed) {
                    // fast pass: the chunk's largest v; only a chunk that can
                    // hold a pair within the threshold is rescanned
                    float m0 = -INFINITY, m1 = -INFINITY;
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        m0 = max3f(m0, __uint_as_float(r[j]), __uint_as_float(r[j + 1]));
                        m1 = max3f(m1, __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
                    }
                    if (fmaxf(m0, m1) >= vhi) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float v = __uint_as_float(r[j]);
                            if (v >= vhi && !removed) {
                                if (v >= vlo) {
                                    removed = true;
                                } else if (!ovf) {
                                    // undecided: deferred to the exact pair check
                                    const int64_t ci = (int64_t)cbase + c0 + j;
                                    if (ci < a.kc) {
                                        const unsigned long long slot = atomicAdd(a.npairs, 1ull);
                                        if (slot < (unsigned long long)a.pcap)
                                            a.pairs[slot] = make_uint2((uint32_t)pi, (uint32_t)ci);
                                        else
                                            ovf = true;
                                        emitted = true;
                                        ++namb;
                                    }
                                }
                            }
                        }
                        if (removed) s_gone_v[row] = 1;
                    }
                }
            };
            for (int t = 0; t < a.ntiles; ++t, ++u) {
                const int s = (int)(u & 1);
                if (!mbar_wait(&t_full[s], (tuse >> s) & 1u, abort)) {
                    set_status(a.st, KC_ERR_TIMEOUT, 10, t);
                    *abort = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                cbase = t * TC_N + grp * TC_COLS;
                if (MODE == 1 && !removed && s_gone_v[row]) removed = true;   // another group decided
                bool released = false;
                if (MODE == 0 || !__all_sync(0xFFFFFFFFu, removed)) {
                    // all four 32-column loads behind one wait: the
                    // accumulator is released after a single TMEM round trip,
                    // then folded (three loads behind one wait and a fourth in
                    // flight took two round trips)
                    static_assert(TC_COLS == 128, "four 32-column chunks per thread");
                    const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(s * TC_N + grp * TC_COLS);
                    uint32_t ra[32], rb[32], rc[32], rd[32];
                    tmem_ld32(taddr, ra);
                    tmem_ld32(taddr + 32, rb);
                    tmem_ld32(taddr + 64, rc);
                    tmem_ld32(taddr + 96, rd);
                    tmem_wait_ld(ra);
                    tmem_pin(rb);
                    tmem_pin(rc);
                    tmem_pin(rd);
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    mbar_arrive(&t_empty[s]);
                    released = true;
                    chunk(ra, 0);
                    chunk(rb, 32);
                    chunk(rc, 64);
                    chunk(rd, 96);
                }
                if (!released) {
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    mbar_arrive(&t_empty[s]);
                }
                tuse ^= 1u << s;
            }
            // combine the column groups of every row in group 0
            const float vmax = fmaxf(fmaxf(v0, v1), fmaxf(v2, v3));
            if (grp > 0) {
                if (MODE == 0) s_part[grp][row] = vmax;
                if (MODE == 1) {
                    if (removed) s_gone[row] = 1;
                    if (emitted || ovf) atomicOr(&s_pend[row], (emitted ? 1 : 0) | (ovf ? 2 : 0));
                }
            }
            asm volatile("bar.sync 1, %0;" ::"n"(TC_EPI) : "memory");
            if (grp == 0 && valid) {
                if (MODE == 0) {
                    // min over centers of s~ = xn - max v, then bounds on the
                    // canonical FP32 minimum (scaled units), then unscaled
                    float vm = vmax;
#pragma unroll
                    for (int q = 1; q < TC_GROUPS; ++q) vm = fmaxf(vm, s_part[q][row]);
                    const float mm_hi = __fsub_ru(xn, vm), mm_lo = __fsub_rd(xn, vm);
                    const float lo_r = __fsub_rd(__fsqrt_rd(fmaxf(__fsub_rd(mm_lo, eps), 0.f)), sl);
                    const float lo = lo_r > 0.f ? __fmul_rd(__fmul_rd(lo_r, lo_r), __fsub_rd(1.f, g)) : 0.f;
                    const float hi_r = __fadd_ru(__fsqrt_ru(__fadd_ru(fmaxf(mm_hi, 0.f), eps)), sl);
                    const float hi = __fmul_ru(__fmul_ru(hi_r, hi_r), __fadd_ru(1.f, g));
                    const float lo_u = __fmul_rd(lo, isc2), hi_u = __fmul_ru(hi, isc2);
                    a.mlo[pi] = lo_u;
                    a.mhi[pi] = hi_u;
                    lomax = fmaxf(lomax, lo_u);
                } else if (!(removed || s_gone[row] != 0)) {
                    const int pf = s_pend[row] | (emitted ? 1 : 0) | (ovf ? 2 : 0);
                    if (pf) {
                        // decided by the pair check (and a full scan on overflow)
                        a.pflag[pi] = (uint8_t)pf;
                        a.pend[atomicAdd(a.npend, 1ull)] = (uint32_t)pi;
                    } else {
                        a.Rn[atomicAdd(a.rnn, 1ull)] = (uint32_t)gx;
                    }
                }
            }
            if (MODE == 1 && grp == 0) {
                s_gone[row] = 0;
                s_pend[row] = 0;
            }
            if (MODE == 1 && namb) atomicAdd(&g_tc_counters[0], namb);
            if (MODE == 1 && grp == 0 && valid) ++nrows;
            asm volatile("bar.sync 1, %0;" ::"n"(TC_EPI) : "memory");   // s_* reused by the next tile
        }
        // one atomic per warp (the lower bounds are non-negative: their bits order as the values)
        if (MODE == 0) {
            const unsigned m = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(lomax));
            if (lane == 0 && grp == 0) atomicMax(a.mlo_max, m);
        } else {
            const unsigned long long r = __reduce_add_sync(0xFFFFFFFFu, (unsigned)nrows);
            if (lane == 0 && r) atomicAdd(&g_tc_counters[1], r);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_N));
    }
}

// Two point tiles per center tile, for streamed centers (the prune; the
// radius when the centers do not fit in shared memory).  tc_dmin_kernel
// reads every center tile from L2 once per point tile; at the MMA's rate that
// is most of the L2 bandwidth (40 KB per 128 x 256 x 80 block, d = 64).  Here
// a center tile feeds two MMAs, one per point tile of a pair, each into its
// own TMEM accumulator (columns 0-255 and 256-511), so every center byte
// serves twice the flops.  While the epilogue drains one accumulator the
// other is being computed: the two accumulators give the overlap of the
// double buffer they replace.  Warps 0-3 own point tile 0's rows, 4-7 tile
// 1's (TMEM lanes 32 (w % 4) ..); each thread holds one row and all 256
// columns of every center tile, so a row's decision needs no exchange
// between warps.  Shared memory: two stages of a tile pair and a two-stage
// center ring (4 A + 2 B bytes).
template <int MODE>
__global__ void __launch_bounds__(384, 1) tc_dmin2_kernel(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int kp = a.kp;
    const uint32_t a_bytes = (uint32_t)TC_M * kp * 2, b_bytes = (uint32_t)TC_N * kp * 2;
    // tile j of pair stage s at smem + (2 s + j) a_bytes, center stage s after them
    unsigned char *const sAb = smem, *const sBb = smem + 4 * a_bytes;
    __shared__ __align__(8) uint64_t a_full[2], a_empty[2], b_full[2], b_empty[2], t_full[2], t_empty[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntile_pts = (a.npts + TC_M - 1) / TC_M;
    const int64_t npairs = (ntile_pts + 1) / 2;
    volatile int *abort = &s_abort;

    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&a_full[s], 1);
            mbar_init(&a_empty[s], 1);
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1);
            mbar_init(&t_full[s], 1);        // accumulator j = s
            mbar_init(&t_empty[s], TC_M);    // its four epilogue warps
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == TC_PROD) {
        // ------------------------------------------------ producer
        if (lane == 0) {
            uint32_t afill = 0, bfill = 0;   // bit s: parity of stage s's fills so far
            int64_t u = 0, p = 0;
            for (int64_t pp = blockIdx.x; pp < npairs && !*abort; pp += gridDim.x, ++p) {
                const int sa = (int)(p & 1);
                const int64_t t0 = 2 * pp;
                const bool has2 = t0 + 1 < ntile_pts;
                if (!mbar_wait(&a_empty[sa], ((afill >> sa) & 1u) ^ 1u, abort)) {
                    *abort = 1;
                    set_status(a.st, KC_ERR_TIMEOUT, 6, 0);
                    break;
                }
                mbar_expect_tx(&a_full[sa], (has2 ? 2u : 1u) * a_bytes);
                bulk_g2s(sAb + (2 * sa) * a_bytes, a.at + t0 * (int64_t)TC_M * kp, a_bytes, &a_full[sa]);
                if (has2)
                    bulk_g2s(sAb + (2 * sa + 1) * a_bytes, a.at + (t0 + 1) * (int64_t)TC_M * kp, a_bytes, &a_full[sa]);
                afill ^= 1u << sa;
                for (int t = 0; t < a.ntiles; ++t, ++u) {
                    const int s = (int)(u & 1);
                    if (!mbar_wait(&b_empty[s], ((bfill >> s) & 1u) ^ 1u, abort)) {
                        *abort = 1;
                        set_status(a.st, KC_ERR_TIMEOUT, 6, t);
                        break;
                    }
                    mbar_expect_tx(&b_full[s], b_bytes);
                    bulk_g2s(sBb + s * b_bytes, a.bt + (int64_t)t * TC_N * kp, b_bytes, &b_full[s]);
                    bfill ^= 1u << s;
                }
            }
        }
    } else if (warp == TC_MMA) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = umma_idesc_f16(TC_M, TC_N);
            const uint32_t a_lbo = (TC_M / 8) * 128, b_lbo = (TC_N / 8) * 128;
            // one K step = two core-matrix columns, in 16-byte descriptor units
            const uint64_t ainc = (2 * a_lbo) >> 4, binc = (2 * b_lbo) >> 4;
            uint32_t ause = 0, buse = 0, tuse = 0;   // bit s: parity of stage (accumulator) s's uses so far
            int64_t u = 0, p = 0;
            MmaClock clk;
            clk.start();
            for (int64_t pp = blockIdx.x; pp < npairs && !*abort; pp += gridDim.x, ++p) {
                const int sa = (int)(p & 1);
                const int nj = 2 * pp + 1 < ntile_pts ? 2 : 1;
                long long c0 = clock64();
                if (!mbar_wait(&a_full[sa], (ause >> sa) & 1u, abort)) {
                    *abort = 1;
                    set_status(a.st, KC_ERR_TIMEOUT, 7, 0);
                    break;
                }
                clk.wa += clock64() - c0;
                for (int t = 0; t < a.ntiles && !*abort; ++t, ++u) {
                    const int s = (int)(u & 1);
                    c0 = clock64();
                    if (!mbar_wait(&b_full[s], (buse >> s) & 1u, abort)) {
                        *abort = 1;
                        set_status(a.st, KC_ERR_TIMEOUT, 8, t);
                        break;
                    }
                    clk.wb += clock64() - c0;
                    const uint64_t bd = umma_desc(smem_u32(sBb + s * b_bytes), b_lbo, 128);
                    for (int j = 0; j < nj; ++j) {
                        c0 = clock64();
                        const bool tok = mbar_wait(&t_empty[j], ((tuse >> j) & 1u) ^ 1u, abort);
                        clk.wt += clock64() - c0;
                        if (!tok) {
                            *abort = 1;
                            set_status(a.st, KC_ERR_TIMEOUT, 8, t);
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint64_t ad = umma_desc(smem_u32(sAb + (2 * sa + j) * a_bytes), a_lbo, 128);
                        umma_chain_k(kp / 16, tmem + (uint32_t)(j * TC_N), ad, bd, ainc, binc, idesc);
                        umma_commit(&t_full[j]);
                        tuse ^= 1u << j;
                    }
                    umma_commit(&b_empty[s]);
                    buse ^= 1u << s;
                }
                umma_commit(&a_empty[sa]);
                ause ^= 1u << sa;
            }
            clk.publish();
        }
    } else {
        // ------------------------------------------------ epilogue warps
        const int j = warp >> 2;                  // the point tile of the pair
        const int row = (warp & 3) * 32 + lane;   // and its row (TMEM lane)
        const float sc = tc_scale(a.absmax, a.d);
        const float sc2 = sc * sc;                // exact power of two
        const float isc2 = 1.f / sc2;             // exact power of two
        const float eta = tc_eta(a.d, kp);
        const float g = lp_slack(a.d);
        const float E = __uint_as_float(a.maxes[0]);
        const float cnmax2 = __fmul_ru(2.f, __uint_as_float(a.maxes[1]));
        const float rmax = __uint_as_float(a.maxes[2]);
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(j * TC_N);
        uint32_t tuse = 0;   // parity of this accumulator's uses so far
        float lomax = 0.f;              // radius: largest lower bound of this thread's rows
        unsigned long long nrows = 0;   // prune: rows processed (diagnostics)
        for (int64_t pp = blockIdx.x; pp < npairs; pp += gridDim.x) {
            const int64_t pt = 2 * pp + j;
            if (pt >= ntile_pts) continue;   // the last pair has one tile (uniform over the warp)
            const int64_t pi = pt * TC_M + row;
            const bool valid = pi < a.npts;
            const float xn = valid ? a.an[pi] : 0.f;
            const float sl = __fadd_ru(valid ? a.ae[pi] : 0.f, E);
            const float eps = __fadd_ru(__fmul_ru(eta, __fadd_ru(xn, cnmax2)), rmax);
            int64_t gx = 0;
            bool removed = !valid;
            if (MODE == 1 && valid) {
                gx = (int64_t)a.R[pi];
                removed = a.rin[pi] != 0;
            }
            float vlo = INFINITY, vhi = INFINITY;
            if (MODE == 1 && valid) {
                // as in tc_dmin_kernel: v >= vlo surely within the threshold,
                // v < vhi surely beyond it, between: the exact pair check
                const float thr = __fmul_rn(__uint_as_float(*a.thr), sc2);   // scaled, exact
                const float ra = __fsub_rd(__fsqrt_rd(__fdiv_rd(thr, __fadd_ru(1.f, g))), sl);
                const float lo_lim = ra > 0.f ? __fsub_rd(__fmul_rd(ra, ra), eps) : -1.f;
                const float rb = __fadd_ru(__fsqrt_ru(__fdiv_ru(thr, __fsub_rd(1.f, g))), sl);
                const float hi_lim = __fadd_ru(__fmul_ru(rb, rb), eps);
                vlo = lo_lim >= 0.f ? __fsub_ru(xn, lo_lim) : INFINITY;
                vhi = __fsub_rd(xn, hi_lim);
            }
            float v0 = -INFINITY, v1 = -INFINITY, v2 = -INFINITY, v3 = -INFINITY;
            unsigned long long namb = 0;
            bool emitted = false, ovf = false;
            int cbase = 0;
            auto chunk = [&](const uint32_t(&r)[32], int c0) {
                if (MODE == 0) {
#pragma unroll
                    for (int q = 0; q < 32; q += 8) {
                        v0 = max3f(v0, __uint_as_float(r[q]), __uint_as_float(r[q + 1]));
                        v1 = max3f(v1, __uint_as_float(r[q + 2]), __uint_as_float(r[q + 3]));
                        v2 = max3f(v2, __uint_as_float(r[q + 4]), __uint_as_float(r[q + 5]));
                        v3 = max3f(v3, __uint_as_float(r[q + 6]), __uint_as_float(r[q + 7]));
                    }
                } else if (!removed) {
                    float m0 = -INFINITY, m1 = -INFINITY;
#pragma unroll
                    for (int q = 0; q < 32; q += 4) {
                        m0 = max3f(m0, __uint_as_float(r[q]), __uint_as_float(r[q + 1]));
                        m1 = max3f(m1, __uint_as_float(r[q + 2]), __uint_as_float(r[q + 3]));
                    }
                    if (fmaxf(m0, m1) >= vhi) {
#pragma unroll
                        for (int q = 0; q < 32; ++q) {
                            const float v = __uint_as_float(r[q]);
                            if (v >= vhi && !removed) {
                                if (v >= vlo) {
                                    removed = true;
                                } else if (!ovf) {
                                    const int64_t ci = (int64_t)cbase + c0 + q;
                                    if (ci < a.kc) {
                                        const unsigned long long slot = atomicAdd(a.npairs, 1ull);
                                        if (slot < (unsigned long long)a.pcap)
                                            a.pairs[slot] = make_uint2((uint32_t)pi, (uint32_t)ci);
                                        else
                                            ovf = true;
                                        emitted = true;
                                        ++namb;
                                    }
                                }
                            }
                        }
                    }
                }
            };
            for (int t = 0; t < a.ntiles; ++t) {
                if (!__all_sync(0xFFFFFFFFu, mbar_wait(&t_full[j], tuse & 1u, abort))) {
                    set_status(a.st, KC_ERR_TIMEOUT, 10, t);
                    *abort = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                cbase = t * TC_N;
                bool released = false;
                if (MODE == 0 || !__all_sync(0xFFFFFFFFu, removed)) {
                    // 256 columns as two batches of four 32-column loads
                    // behind one wait each; the accumulator is released as
                    // soon as the second batch has landed
                    uint32_t ra[32], rb[32], rc[32], rd[32];
#pragma unroll 1
                    for (int h = 0; h < 2; ++h) {
                        const uint32_t ta = taddr + (uint32_t)(h * 128);
                        tmem_ld32(ta, ra);
                        tmem_ld32(ta + 32, rb);
                        tmem_ld32(ta + 64, rc);
                        tmem_ld32(ta + 96, rd);
                        tmem_wait_ld(ra);
                        tmem_pin(rb);
                        tmem_pin(rc);
                        tmem_pin(rd);
                        if (h == 1) {
                            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                            mbar_arrive(&t_empty[j]);
                            released = true;
                        }
                        chunk(ra, h * 128);
                        chunk(rb, h * 128 + 32);
                        chunk(rc, h * 128 + 64);
                        chunk(rd, h * 128 + 96);
                    }
                }
                if (!released) {
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    mbar_arrive(&t_empty[j]);
                }
                tuse ^= 1u;
            }
            if (!valid) continue;
            if (MODE == 0) {
                // min over centers of s~ = xn - max v, then bounds on the
                // canonical FP32 minimum (scaled units), then unscaled
                const float vm = fmaxf(fmaxf(v0, v1), fmaxf(v2, v3));
                const float mm_hi = __fsub_ru(xn, vm), mm_lo = __fsub_rd(xn, vm);
                const float lo_r = __fsub_rd(__fsqrt_rd(fmaxf(__fsub_rd(mm_lo, eps), 0.f)), sl);
                const float lo = lo_r > 0.f ? __fmul_rd(__fmul_rd(lo_r, lo_r), __fsub_rd(1.f, g)) : 0.f;
                const float hi_r = __fadd_ru(__fsqrt_ru(__fadd_ru(fmaxf(mm_hi, 0.f), eps)), sl);
                const float hi = __fmul_ru(__fmul_ru(hi_r, hi_r), __fadd_ru(1.f, g));
                const float lo_u = __fmul_rd(lo, isc2), hi_u = __fmul_ru(hi, isc2);
                a.mlo[pi] = lo_u;
                a.mhi[pi] = hi_u;
                lomax = fmaxf(lomax, lo_u);
            } else {
                if (!removed) {
                    const int pf = (emitted ? 1 : 0) | (ovf ? 2 : 0);
                    if (pf) {
                        // decided by the pair check (and a full scan on overflow)
                        a.pflag[pi] = (uint8_t)pf;
                        a.pend[atomicAdd(a.npend, 1ull)] = (uint32_t)pi;
                    } else {
                        a.Rn[atomicAdd(a.rnn, 1ull)] = (uint32_t)gx;
                    }
                }
                if (namb) atomicAdd(&g_tc_counters[0], namb);
                ++nrows;
            }
        }
        if (MODE == 0) {
            const unsigned m = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(lomax));
            if (lane == 0) atomicMax(a.mlo_max, m);
        } else {
            const unsigned long long r = __reduce_add_sync(0xFFFFFFFFu, (unsigned)nrows);
            if (lane == 0 && r) atomicAdd(&g_tc_counters[1], r);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_N));
    }
}

// Radius, exact part.  T = (largest lower bound) (1 - 3 gamma): a point whose
// upper bound reaches T can hold the maximum (the FP32-to-FP64 margin of the
// CUDA-core path).  Flag pass: those points go to a list (in no particular
// order) and start from an empty minimum; every other point gets 0.
__global__ void tc_flag_kernel(int64_t n, int d, const float *__restrict__ mhi, const unsigned *mlo_max,
                               uint32_t *__restrict__ mind, uint32_t *__restrict__ flist,
                               unsigned long long *fcount, const DevStatus *st) {
    if (ld_volatile_i32(&st->code) != 0) return;
    const double T = (double)__uint_as_float(*mlo_max) * (1.0 - 3.0 * f32_gamma(d));
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    // a warp takes 128 consecutive points per pass, four loads in flight
    for (int64_t base = (blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)) * 128; base < n;
         base += warps * 128) {
        float h[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t x = base + 32 * q + lane;
            h[q] = x < n ? mhi[x] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t x = base + 32 * q + lane;
            const bool flag = x < n && (double)h[q] >= T;
            if (x < n) mind[x] = flag ? 0xFFFFFFFFu : 0u;
            const unsigned b = __ballot_sync(0xFFFFFFFFu, flag);
            if (!b) continue;
            unsigned long long at = 0;
            if (lane == 0) at = atomicAdd(fcount, (unsigned long long)__popc(b));
            at = __shfl_sync(0xFFFFFFFFu, at, 0);
            if (flag) flist[at + __popc(b & ((1u << lane) - 1u))] = (uint32_t)x;
        }
    }
}

// Exact canonical FP32 minima of the listed points: work items are (a group
// of EX_PG listed points, a chunk of EX_CC centers); a CTA stages the chunk
// (row stride d | 1: the lanes' rows fall in distinct banks) and the group's
// coordinates in shared memory, each warp takes points of the group with its
// lanes over the chunk's centers, and the chunk minima meet in atomicMin
// (float bits of non-negative values order as the values).
constexpr int EX_NT = 256, EX_PG = 64, EX_CC = 128;
__global__ void __launch_bounds__(EX_NT) tc_exact_list_kernel(const float *__restrict__ pk, const float *__restrict__ rm,
                                                              int d, const float *__restrict__ cen,
                                                              const int32_t *kc_dev, int kc_max,
                                                              const uint32_t *__restrict__ flist,
                                                              const unsigned long long *fcount,
                                                              uint32_t *__restrict__ mind, const DevStatus *st) {
    extern __shared__ float ex_smem[];
    if (ld_volatile_i32(&st->code) != 0) return;
    const int ld = d | 1;
    float *scen = ex_smem;                  // [EX_CC][ld]
    float *spts = ex_smem + EX_CC * ld;     // [EX_PG][d]
    const int kc = (int)dev_count(kc_dev, kc_max);
    const int64_t F = (int64_t)*fcount;
    const int64_t chunks = (kc + EX_CC - 1) / EX_CC;
    const int64_t items = (F + EX_PG - 1) / EX_PG * chunks;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int64_t p0 = it / chunks * EX_PG;
        const int c0 = (int)(it % chunks) * EX_CC;
        const int ncc = kc - c0 < EX_CC ? kc - c0 : EX_CC;
        const int npg = (int)(F - p0 < EX_PG ? F - p0 : EX_PG);
        __syncthreads();   // the previous item's reads are done
        for (int e = tid; e < ncc * d; e += EX_NT) {
            const int ci = e / d, j = e - ci * d;
            scen[ci * ld + j] = cen[(int64_t)(c0 + ci) * d + j];
        }
        for (int e = tid; e < npg * d; e += EX_NT) {
            const int q = e / d, j = e - q * d;
            spts[q * d + j] = point_at(pk, rm, flist[p0 + q], j, d);
        }
        __syncthreads();
        for (int q = warp; q < npg; q += EX_NT / 32) {
            const float *xp = spts + q * d;
            uint32_t m = 0xFFFFFFFFu;
            for (int ci = lane; ci < ncc; ci += 32) {
                const float *cr = scen + ci * ld;
                float acc = 0.f;
                for (int j = 0; j < d; ++j) acc = sq_step(acc, xp[j], cr[j]);
                m = min(m, __float_as_uint(acc));
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) m = min(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
            if (lane == 0) atomicMin(&mind[flist[p0 + q]], m);
        }
    }
}

// The argmax key over the listed points (everyone else has minimum 0).
__global__ void tc_key_list_kernel(const uint32_t *__restrict__ flist, const unsigned long long *fcount,
                                   const uint32_t *__restrict__ mind, unsigned long long *key32, const DevStatus *st) {
    if (ld_volatile_i32(&st->code) != 0) return;
    const int64_t F = (int64_t)*fcount;
    uint64_t best = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < F; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = flist[i];
        best = umax64(best, make_key(mind[x], x));
    }
    best = warp_max_u64(best);
    if ((threadIdx.x & 31) == 0 && best) atomicMax(key32, (unsigned long long)best);
}

// Canonical FP32 squared distance of rows x and c (d coordinates), with
// 16-byte loads when both rows allow them.
__device__ __forceinline__ float row_dist(const float *__restrict__ x, const float *__restrict__ c, int d, bool v4) {
    float acc = 0.f;
    if (v4) {
        const float4 *x4 = reinterpret_cast<const float4 *>(x), *c4 = reinterpret_cast<const float4 *>(c);
        for (int k = 0; k < d / 4; ++k) {
            const float4 xa = __ldg(x4 + k), ca = __ldg(c4 + k);
            acc = sq_step(acc, xa.x, ca.x);
            acc = sq_step(acc, xa.y, ca.y);
            acc = sq_step(acc, xa.z, ca.z);
            acc = sq_step(acc, xa.w, ca.w);
        }
    } else {
        for (int k = 0; k < d; ++k) acc = sq_step(acc, __ldg(x + k), __ldg(c + k));
    }
    return acc;
}

// Exact check of the deferred pairs: hit[row] once a pair is within the
// threshold (canonical FP32 distance, the same test as the CUDA-core prune).
__global__ void tc_pair_kernel(const float *__restrict__ src, int d, bool v4, const uint32_t *__restrict__ R,
                               const float *__restrict__ cen, const uint2 *__restrict__ pairs,
                               const unsigned long long *npairs, int64_t pcap, const uint32_t *thr, uint8_t *hit) {
    const int64_t np = (int64_t)min(*npairs, (unsigned long long)pcap);
    const uint32_t T = *thr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        const uint2 p = pairs[i];
        if (hit[p.x]) continue;
        const float acc = row_dist(src + (int64_t)R[p.x] * d, cen + (int64_t)p.y * d, d, v4);
        if (__float_as_uint(acc) <= T) hit[p.x] = 1;
    }
}

// Pending rows: removed on a hit; a row whose pairs overflowed the buffer is
// scanned against every center (one warp, lanes over centers); the rest are
// kept.
__global__ void tc_resolve_kernel(const float *__restrict__ src, int d, bool v4, const uint32_t *__restrict__ R,
                                  const float *__restrict__ cen, int64_t sn, const uint32_t *__restrict__ pend,
                                  const unsigned long long *npend, const uint8_t *__restrict__ flag,
                                  const uint8_t *__restrict__ hit, const uint32_t *thr, uint32_t *Rn,
                                  unsigned long long *rnn) {
    const int64_t np = (int64_t)*npend;
    const uint32_t T = *thr;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); j < np; j += warps) {
        const uint32_t pi = pend[j];
        const int64_t gx = (int64_t)R[pi];
        bool rm = hit[pi] != 0;
        if (!rm && (flag[pi] & 2)) {
            for (int64_t cb = 0; cb < sn && !rm; cb += 32) {
                const int64_t ci = cb + lane;
                const bool h = ci < sn && __float_as_uint(row_dist(src + gx * d, cen + ci * d, d, v4)) <= T;
                rm = __any_sync(0xFFFFFFFFu, h);
            }
        }
        if (!rm && lane == 0) Rn[atomicAdd(rnn, 1ull)] = (uint32_t)gx;
    }
}

int sms() {
    int dev = 0, s = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    return s;
}

// K of the MMA tiles: the d coordinates and the three norm columns, rounded
// up to the MMA's K of 16.
int kpad(int d) { return (d + 3 + 15) / 16 * 16; }

// Dynamic shared memory: two point tiles and two center tiles, and at least
// 120 KB so that one CTA (holding all 512 TMEM columns) runs per SM.
// Dynamic shared memory of a launch over ntiles center tiles: a two-stage
// point-tile ring and either every center tile (resident, loaded once) or a
// two-stage center ring; at least 120 KB, so that one CTA holds the SM (and
// all 512 TMEM columns).  A third point stage (when it fits beside resident
// centers) measured slower: the larger shared-memory carve-out leaves less
// L1.
constexpr size_t TC_SMEM_MAX = 220 * 1024;
size_t tc_smem_for(TcArgs &a) {
    const size_t A = (size_t)TC_M * a.kp * 2, B = (size_t)TC_N * a.kp * 2;
    const size_t centers = (size_t)a.ntiles * B;
    a.resident = 2 * A + centers <= TC_SMEM_MAX && !getenv("KC_TC_STREAM_CENTERS") ? 1 : 0;
    const size_t need = 2 * A + (a.resident ? centers : 2 * B);
    const size_t floor1 = 120 * 1024;   // one CTA per SM
    return need > floor1 ? need : floor1;
}

// tc_dmin2_kernel's shared memory (two stages of a point-tile pair, a
// two-stage center ring), or 0 when it does not fit (d above 93) or
// KC_TC_PAIR=0 in the environment.
size_t tc_pair_smem(int kp) {
    const size_t A = (size_t)TC_M * kp * 2, B = (size_t)TC_N * kp * 2;
    if (const char *env = getenv("KC_TC_PAIR"))
        if (atoi(env) == 0) return 0;
    const size_t need = 4 * A + 2 * B;
    return need <= TC_SMEM_MAX ? (need > 120 * 1024 ? need : 120 * 1024) : 0;
}

template <int MODE>
cudaError_t launch_dmin2(const TcArgs &a, size_t smem, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(tc_dmin2_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    const int64_t pairs = ((a.npts + TC_M - 1) / TC_M + 1) / 2;
    const int grid = (int)std::min<int64_t>(pairs, (int64_t)sms());
    if (grid > 0) tc_dmin2_kernel<MODE><<<grid, TC_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <int R>
cudaError_t rows(const float *pk, const float *rm, const uint32_t *idx, const int32_t *cnt_dev, int64_t cnt, int d,
                 const unsigned *absmax, void *tiles, float *norm, float *err, unsigned *maxes, cudaStream_t s,
                 const uint8_t *inS = nullptr, uint8_t *rin = nullptr) {
    const int64_t nt = (cnt + R - 1) / R;
    if (nt == 0) return cudaSuccess;
    const int64_t rowsn = nt * R;
    const int grid = (int)std::min<int64_t>((rowsn + 255) / 256, (int64_t)sms() * 8);
    tc_rows_kernel<R><<<grid, 256, 0, s>>>(pk, rm, idx, cnt_dev, cnt, d, kpad(d), nt, absmax, (__half *)tiles, norm, err,
                                           maxes, inS, rin);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

bool tc_supported(int d) { return d >= 1 && d <= TC_KMAX; }

cudaError_t read_tc_counters(unsigned long long out[6], bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_tc_counters, 6 * sizeof(unsigned long long));
    if (e == cudaSuccess && reset) {
        const unsigned long long z[6] = {0, 0, 0, 0, 0, 0};
        e = cudaMemcpyToSymbol(g_tc_counters, z, sizeof z);
    }
    return e;
}

int tc_center_tiles(int64_t kc) { return (int)((kc + TC_N - 1) / TC_N); }
size_t tc_center_bytes(int64_t kc, int d) { return (size_t)tc_center_tiles(kc) * TC_N * kpad(d) * 2; }
size_t tc_point_bytes(int64_t n, int d) { return (size_t)((n + TC_M - 1) / TC_M) * TC_M * kpad(d) * 2; }
int64_t tc_point_rows(int64_t n) { return (n + TC_M - 1) / TC_M * TC_M; }

cudaError_t launch_tc_absmax(const float *pk, int64_t n, int d, unsigned *absmax, cudaStream_t s) {
    cudaMemsetAsync(absmax, 0, sizeof(unsigned), s);
    const int64_t total = nblocks(n) * (int64_t)d * BLK;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sms() * 8);
    tc_absmax_kernel<<<grid, 256, 0, s>>>(pk, n, d, absmax);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_tc_centers(const float *cen_rows, const int32_t *kc_dev, int64_t kc, int d, const unsigned *absmax,
                              void *bt, float *cn, float *ce, unsigned *maxes, cudaStream_t s) {
    cudaMemsetAsync(maxes, 0, 3 * sizeof(unsigned), s);
    return rows<TC_N>(nullptr, cen_rows, nullptr, kc_dev, kc, d, absmax, bt, cn, ce, maxes, s);
}

cudaError_t launch_tc_points(const float *pk, const float *rm, const uint32_t *idx, int64_t n, int d,
                             const unsigned *absmax, void *at, float *an, float *ae, cudaStream_t s,
                             const uint8_t *inS = nullptr, uint8_t *rin = nullptr) {
    return rows<TC_M>(pk, rm, idx, nullptr, n, d, absmax, at, an, ae, nullptr, s, inS, rin);
}

cudaError_t launch_tc_radius(const float *pk, const float *rm, int64_t n, int d, const float *cen,
                             const int32_t *kc_dev, int kc, const TcBufs &B, uint32_t *mind,
                             unsigned long long *key32, DevStatus *st, cudaStream_t s) {
    cudaError_t e;
    if (pk) {
        if ((e = launch_tc_absmax(pk, n, d, B.absmax, s)) != cudaSuccess) return e;
        if ((e = launch_tc_points(pk, nullptr, nullptr, n, d, B.absmax, B.at, B.an, B.ae, s)) != cudaSuccess)
            return e;
    } else {
        const bool vec = ((uintptr_t)rm & 15) == 0;
        cudaMemsetAsync(B.absmax, 0, 3 * sizeof(unsigned), s);   // final, sampled and true scale words
        const int64_t stotal = (n + TC_SAMPLE - 1) / TC_SAMPLE * d;
        const int ga = (int)std::min<int64_t>((stotal + 255) / 256, (int64_t)sms() * 4);
        tc_absmax_sample_kernel<<<ga, 256, 0, s>>>(rm, n, d, B.absmax);
        const int64_t nt = (n + TC_M - 1) / TC_M;
        const size_t sm = (size_t)TC_M * (d | 1) * sizeof(float);
        if ((e = cudaFuncSetAttribute(tc_points_rm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(tc_points_rm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm)) != cudaSuccess)
            return e;
        const int gp = (int)std::min<int64_t>(nt, (int64_t)sms() * 8);
        tc_points_rm_kernel<false><<<gp, TC_RM_NT, sm, s>>>(rm, n, d, vec, kpad(d), nt, B.absmax, st,
                                                             (__half *)B.at, B.an, B.ae);
        tc_points_rm_kernel<true><<<gp, TC_RM_NT, sm, s>>>(rm, n, d, vec, kpad(d), nt, B.absmax, st,
                                                            (__half *)B.at, B.an, B.ae);
        note_launches(3);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = launch_tc_centers(cen, kc_dev, kc, d, B.absmax, B.bt, B.cn, B.ce, B.maxes, s)) != cudaSuccess) return e;
    TcArgs a{};
    a.d = d;
    a.kp = kpad(d);
    a.kc = kc;
    a.ntiles = tc_center_tiles(kc);
    a.npts = n;
    a.at = (const __half *)B.at;
    a.an = B.an;
    a.ae = B.ae;
    a.bt = (const __half *)B.bt;
    a.cn = B.cn;
    a.maxes = B.maxes;
    a.absmax = B.absmax;
    a.mlo = B.mlo;
    a.mhi = B.mhi;
    a.mlo_max = B.mlomax;
    a.st = st;
    const size_t smem = tc_smem_for(a);
    if ((e = cudaFuncSetAttribute(tc_dmin_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    cudaMemsetAsync(B.mlomax, 0, sizeof(unsigned), s);
    const size_t smem2 = a.resident ? 0 : tc_pair_smem(a.kp);
    if (smem2) {
        // streamed centers: two point tiles per center tile
        if ((e = launch_dmin2<0>(a, smem2, s)) != cudaSuccess) return e;
    } else {
        const int64_t tiles = (n + TC_M - 1) / TC_M;
        const int grid = (int)std::min<int64_t>(tiles, (int64_t)sms());
        tc_dmin_kernel<0><<<grid, TC_THREADS, smem, s>>>(a);
    }
    const int g2 = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms() * 8);
    cudaMemsetAsync(B.fcount, 0, sizeof(unsigned long long), s);
    tc_flag_kernel<<<g2, 256, 0, s>>>(n, d, B.mhi, B.mlomax, mind, B.flist, B.fcount, st);
    const size_t exsm = ((size_t)EX_CC * (d | 1) + (size_t)EX_PG * d) * sizeof(float);
    if ((e = cudaFuncSetAttribute(tc_exact_list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)exsm)) !=
        cudaSuccess)
        return e;
    // the list's length is on the device: the grid covers the largest case
    const int64_t items_max = (n + EX_PG - 1) / EX_PG * ((kc + EX_CC - 1) / EX_CC);
    const int g3 = (int)std::min<int64_t>(items_max, (int64_t)sms() * 8);
    tc_exact_list_kernel<<<g3, EX_NT, exsm, s>>>(pk, rm, d, cen, kc_dev, kc, B.flist, B.fcount, mind, st);
    tc_key_list_kernel<<<g2, 256, 0, s>>>(B.flist, B.fcount, mind, key32, st);
    note_launches(4);
    return cudaGetLastError();
}

cudaError_t launch_tc_prune(const float *src, int d, const uint32_t *R, int64_t rn, const uint8_t *inS, const float *Scen,
                            int64_t sn, const TcBufs &B, const PruneBufs &P, const uint32_t *thr, uint32_t *Rn,
                            unsigned long long *rnn, DevStatus *st, cudaStream_t s) {
    cudaError_t e;
    if ((e = launch_tc_points(nullptr, src, R, rn, d, B.absmax, B.at, B.an, B.ae, s, inS, B.rin)) != cudaSuccess)
        return e;
    if ((e = launch_tc_centers(Scen, nullptr, sn, d, B.absmax, B.bt, B.cn, B.ce, B.maxes, s)) != cudaSuccess) return e;
    cudaMemsetAsync(P.npairs, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(P.npend, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(P.hit, 0, (size_t)rn, s);
    TcArgs a{};
    a.d = d;
    a.kp = kpad(d);
    a.kc = (int)sn;
    a.ntiles = tc_center_tiles(sn);
    a.npts = rn;
    a.at = (const __half *)B.at;
    a.an = B.an;
    a.ae = B.ae;
    a.bt = (const __half *)B.bt;
    a.cn = B.cn;
    a.maxes = B.maxes;
    a.absmax = B.absmax;
    a.src = src;
    a.R = R;
    a.rin = B.rin;
    a.cen = Scen;
    a.thr = thr;
    a.Rn = Rn;
    a.rnn = rnn;
    a.pairs = P.pairs;
    a.pcap = P.pcap;
    a.npairs = P.npairs;
    a.pflag = P.flag;
    a.pend = P.pend;
    a.npend = P.npend;
    a.st = st;
    const size_t smem = tc_smem_for(a);
    const int64_t tiles = (rn + TC_M - 1) / TC_M;
    if (tiles == 0) return cudaGetLastError();
    const size_t smem2 = a.resident ? 0 : tc_pair_smem(a.kp);
    if (smem2) {
        // streamed centers: two point tiles per center tile
        if ((e = launch_dmin2<1>(a, smem2, s)) != cudaSuccess) return e;
    } else {
        if ((e = cudaFuncSetAttribute(tc_dmin_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        const int grid = (int)std::min<int64_t>(tiles, (int64_t)sms());
        tc_dmin_kernel<1><<<grid, TC_THREADS, smem, s>>>(a);
    }
    const bool v4 = (d & 3) == 0 && ((uintptr_t)src & 15) == 0 && ((uintptr_t)Scen & 15) == 0;
    const int g2 = sms() * 8;
    tc_pair_kernel<<<g2, 256, 0, s>>>(src, d, v4, R, Scen, P.pairs, P.npairs, P.pcap, thr, P.hit);
    tc_resolve_kernel<<<g2, 256, 0, s>>>(src, d, v4, R, Scen, sn, P.pend, P.npend, P.flag, P.hit, thr, Rn, rnn);
    note_launches(3);
    return cudaGetLastError();
}

}  // namespace kc
