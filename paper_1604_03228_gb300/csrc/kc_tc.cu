// kc_tc.cu -- tensor-core (tcgen05) distance blocks for the dense n x k
// work: the covering radius of a center set (solution value, Section 7) and
// EIM's prune of R against the sample S (Algorithm 2, the round Section 5.2
// finds dominant).
//
// A CTA owns a tile of 128 points (the MMA's M) and streams the centers in
// tiles of 256 (N).  Points and centers are rounded to bf16; one
// tcgen05.mma.kind::f16 per 16 coordinates accumulates the 128 x 256 dot
// products x~.c~ in FP32 in tensor memory (two accumulators, 512 columns),
// while bulk copies stage the next center tile in shared memory.  Warps:
//   0-7  epilogue: warps w and w+4 own point rows 32(w%4).. (their TMEM
//        lanes) and split the 256 accumulator columns; each thread forms
//        s~ = |x~|^2 + |c~|^2 - 2 x~.c~ per center from tcgen05.ld values
//   8    producer: cp.async.bulk of pre-laid-out center tiles
//   9    MMA issuer (one thread)
// Operand layout in shared memory: no swizzle, K-major, 8x16-byte core
// matrices; core matrix (row block mi, column block ki) of an R-row tile at
// byte ((ki * R/8) + mi) * 128, so the descriptor's leading (K) byte offset
// is R/8 * 128 and its stride (M/N) byte offset is 128.
//
// Error bound.  With e_x = ||x~ - x|| (and E = max over centers of e_c), the
// products of bf16 values are exact and the FP32 accumulation, the norms and
// the two epilogue operations are covered by
//   |s~ - ||x~ - c~||^2| <= eta (|x~|^2 + |c~|^2),  eta = g_d + (K+16) 2^-21 + 2^-21,
// a deliberately loose model of the tensor core's accumulation.  With the
// triangle inequality ||x - c|| in [||x~-c~|| - e_x - e_c, ||x~-c~|| + e_x + e_c]
// and the canonical FP32 value within (1 +- g_d) of the exact one, every
// decision below is taken on bounds that contain the canonical FP32 value;
// undecided cases are recomputed exactly.
#include <cuda_bf16.h>

#include "kc_internal.cuh"

namespace kc {

namespace {

constexpr int TC_M = 128;
constexpr int TC_N = 256;
constexpr int TC_THREADS = 320;   // warps 0-7 epilogue, 8 producer, 9 MMA
constexpr int TC_EPI = 256;
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

// kind::f16 instruction descriptor: FP32 accumulate, bf16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
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

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                 "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t r[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Element offset of (row r, coordinate k) in an R-row no-swizzle K-major tile.
__host__ __device__ __forceinline__ int core_off(int R, int r, int k) {
    return ((k >> 3) * (R >> 3) + (r >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// ------------------------------------------------------------ center prep
// Centers (FP32 rows [kc][d]) -> bf16 tiles of TC_N rows in the core layout,
// |c~|^2 per center (+inf for padding rows), and the maxima of e_c and |c~|^2.
__global__ void tc_prep_kernel(const float *__restrict__ cen, const int32_t *kc_dev, int kc_max, int d, int kp,
                               int ntiles, __nv_bfloat16 *__restrict__ bt, float *__restrict__ cn,
                               unsigned *__restrict__ maxes) {
    const int kc = kc_dev ? *kc_dev : kc_max;
    const int tile_elems = TC_N * kp;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < (int64_t)ntiles * TC_N;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(c / TC_N), r = (int)(c % TC_N);
        __nv_bfloat16 *tile = bt + (int64_t)t * tile_elems;
        float nrm = 0.f, e2 = 0.f;
        for (int k = 0; k < kp; ++k) {
            const float x = (c < kc && k < d) ? cen[c * d + k] : 0.f;
            const __nv_bfloat16 q = __float2bfloat16_rn(x);
            const float xq = __bfloat162float(q);
            const float df = fabsf(__fsub_rn(x, xq));
            e2 = __fmaf_ru(df, df, e2);
            nrm = __fmaf_rn(xq, xq, nrm);
            tile[core_off(TC_N, r, k)] = q;
        }
        cn[c] = c < kc ? nrm : INFINITY;
        if (c < kc) {
            atomicMax(&maxes[0], __float_as_uint(__fsqrt_ru(e2)));
            atomicMax(&maxes[1], __float_as_uint(nrm));
        }
    }
}

struct TcArgs {
    int mode;                   // 0: radius (per-point bounds), 1: EIM prune
    int d, kp, kc, ntiles;
    int64_t npts;               // points (radius: n; prune: |R|)
    const float *pk;            // radius: packed FP32 points
    const float *src;           // prune: row-major FP32 points
    const uint32_t *R;          // prune: point indices
    const uint8_t *inS;         // prune: sampled points (always removed)
    const __nv_bfloat16 *bt;    // center tiles
    const float *cn;            // [ntiles * TC_N]
    const unsigned *maxes;      // [0] = E (max e_c), [1] = max |c~|^2 (float bits)
    const float *cen;           // FP32 center rows (exact rechecks)
    float *mlo, *mhi;           // radius: per-point bounds on the canonical minimum
    unsigned *mlo_max;          // radius: max of mlo (float bits)
    const uint32_t *thr;        // prune: threshold (canonical FP32 bits)
    uint32_t *Rn;               // prune: kept points
    unsigned long long *rnn;
    unsigned long long *amb;    // prune diagnostics: exact pair checks
    DevStatus *st;
};

__device__ __forceinline__ float tc_eta(int d, int kp) {
    return (float)(f32_gamma(d) + (double)(kp + 16) * 0x1p-21 + 0x1p-21);
}

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_dmin_kernel(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int kp = a.kp;
    const uint32_t a_bytes = (uint32_t)TC_M * kp * 2, b_bytes = (uint32_t)TC_N * kp * 2;
    __nv_bfloat16 *sA = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *sB0 = reinterpret_cast<__nv_bfloat16 *>(smem + a_bytes);
    __nv_bfloat16 *sB1 = reinterpret_cast<__nv_bfloat16 *>(smem + a_bytes + b_bytes);
    __shared__ __align__(8) uint64_t b_full[2], b_empty[2], t_full[2], t_empty[2], a_full, a_empty;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    __shared__ float s_xn[TC_M], s_ex[TC_M], s_part[TC_M];
    __shared__ int s_gone[TC_M], s_gone2[TC_M];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntile_pts = (a.npts + TC_M - 1) / TC_M;
    volatile int *abort = &s_abort;

    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1);
            mbar_init(&t_full[s], 1);
            mbar_init(&t_empty[s], TC_EPI);
        }
        mbar_init(&a_full, TC_M);
        mbar_init(&a_empty, 1);
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

    if (warp == 8) {
        // ------------------------------------------------ producer
        if (lane == 0) {
            uint32_t fills[2] = {0, 0};
            int64_t u = 0;
            for (int64_t pt = blockIdx.x; pt < ntile_pts && !*abort; pt += gridDim.x) {
                for (int t = 0; t < a.ntiles; ++t, ++u) {
                    const int s = (int)(u & 1);
                    if (!mbar_wait(&b_empty[s], (fills[s] & 1u) ^ 1u, abort)) {
                        *abort = 1;
                        set_status(a.st, KC_ERR_TIMEOUT, 6, t);
                        break;
                    }
                    mbar_expect_tx(&b_full[s], b_bytes);
                    bulk_g2s(s ? sB1 : sB0, a.bt + (int64_t)t * TC_N * kp, b_bytes, &b_full[s]);
                    ++fills[s];
                }
            }
        }
    } else if (warp == 9) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = umma_idesc_bf16(TC_M, TC_N);
            const uint32_t a_lbo = (TC_M / 8) * 128, b_lbo = (TC_N / 8) * 128;
            uint32_t uses_b[2] = {0, 0}, uses_t[2] = {0, 0}, pts = 0;
            int64_t u = 0;
            for (int64_t pt = blockIdx.x; pt < ntile_pts && !*abort; pt += gridDim.x, ++pts) {
                if (!mbar_wait(&a_full, pts & 1u, abort)) {
                    *abort = 1;
                    set_status(a.st, KC_ERR_TIMEOUT, 7, 0);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int t = 0; t < a.ntiles; ++t, ++u) {
                    const int s = (int)(u & 1);
                    if (!mbar_wait(&t_empty[s], (uses_t[s] & 1u) ^ 1u, abort) ||
                        !mbar_wait(&b_full[s], uses_b[s] & 1u, abort)) {
                        *abort = 1;
                        set_status(a.st, KC_ERR_TIMEOUT, 8, t);
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t abase = smem_u32(sA), bbase = smem_u32(s ? sB1 : sB0);
                    for (int kk = 0; kk < kp / 16; ++kk) {
                        const uint64_t ad = umma_desc(abase + kk * 2 * a_lbo, a_lbo, 128);
                        const uint64_t bd = umma_desc(bbase + kk * 2 * b_lbo, b_lbo, 128);
                        umma_bf16(tmem + (uint32_t)(s * TC_N), ad, bd, idesc, kk > 0 ? 1u : 0u);
                    }
                    umma_commit(&b_empty[s]);
                    umma_commit(&t_full[s]);
                    ++uses_b[s];
                    ++uses_t[s];
                }
                umma_commit(&a_empty);
            }
        }
    } else {
        // ------------------------------------------------ epilogue warps 0-7
        // Warps w and w+4 share TMEM lanes 32(w%4)..: row = point of the tile;
        // warp w < 4 takes accumulator columns 0..127, warp w+4 columns 128..255.
        const int row = (warp & 3) * 32 + lane;
        const int half = warp >> 2;
        const float eta = tc_eta(a.d, kp);
        const float g = lp_slack(a.d);
        const float E = __uint_as_float(a.maxes[0]);
        const float cnmax = __uint_as_float(a.maxes[1]);
        uint32_t uses_t[2] = {0, 0}, pts = 0;
        int64_t u = 0;
        for (int64_t pt = blockIdx.x; pt < ntile_pts; pt += gridDim.x, ++pts) {
            const int64_t pi = pt * TC_M + row;
            const bool valid = pi < a.npts;
            int64_t gx = 0;
            if (valid) gx = MODE == 0 ? pi : (int64_t)a.R[pi];
            if (half == 0) {
                // A tile: this thread's point, rounded to bf16, into the core layout
                if (!mbar_wait(&a_empty, (pts & 1u) ^ 1u, abort)) {
                    set_status(a.st, KC_ERR_TIMEOUT, 9, 0);
                    *abort = 1;
                }
                float xn = 0.f, e2 = 0.f;
                for (int k = 0; k < kp; ++k) {
                    float x = 0.f;
                    if (valid && k < a.d) x = MODE == 0 ? a.pk[pk_index(gx, k, a.d)] : a.src[gx * a.d + k];
                    const __nv_bfloat16 q = __float2bfloat16_rn(x);
                    const float xq = __bfloat162float(q);
                    const float df = fabsf(__fsub_rn(x, xq));
                    e2 = __fmaf_ru(df, df, e2);
                    xn = __fmaf_rn(xq, xq, xn);
                    sA[core_off(TC_M, row, k)] = q;
                }
                s_xn[row] = xn;
                s_ex[row] = __fsqrt_ru(e2);
                s_gone[row] = (!valid || (MODE == 1 && a.inS[gx])) ? 1 : 0;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&a_full);
            }
            asm volatile("bar.sync 1, %0;" ::"n"(TC_EPI) : "memory");
            const float xn = s_xn[row];
            const float sl = __fadd_ru(s_ex[row], E);
            const float eps = __fmul_ru(eta, __fadd_ru(xn, cnmax));
            bool removed = s_gone[row] != 0;
            float lo_lim = 0.f, hi_lim = 0.f;
            if (MODE == 1) {
                const float thr = __uint_as_float(*a.thr);
                const float ra = __fsub_rd(__fsqrt_rd(__fdiv_rd(thr, __fadd_ru(1.f, g))), sl);
                lo_lim = ra > 0.f ? __fsub_rd(__fmul_rd(ra, ra), eps) : -1.f;   // s~ <= lo_lim: within thr
                const float rb = __fadd_ru(__fsqrt_ru(__fdiv_ru(thr, __fsub_rd(1.f, g))), sl);
                hi_lim = __fadd_ru(__fmul_ru(rb, rb), eps);                    // s~ > hi_lim: beyond thr
            }
            float m0 = INFINITY, m1 = INFINITY, m2 = INFINITY, m3 = INFINITY;
            unsigned long long namb = 0;
            for (int t = 0; t < a.ntiles; ++t, ++u) {
                const int s = (int)(u & 1);
                if (!mbar_wait(&t_full[s], uses_t[s] & 1u, abort)) {
                    set_status(a.st, KC_ERR_TIMEOUT, 10, t);
                    *abort = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const float *cnt = a.cn + (int64_t)t * TC_N + half * (TC_N / 2);
                for (int c0 = 0; c0 < TC_N / 2; c0 += 32) {
                    uint32_t r[32];
                    tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(s * TC_N + half * (TC_N / 2) + c0),
                              r);
                    if (MODE == 0) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {
                            m0 = fminf(m0, __fadd_rn(__fmaf_rn(-2.f, __uint_as_float(r[j]), xn), __ldg(cnt + c0 + j)));
                            m1 = fminf(m1, __fadd_rn(__fmaf_rn(-2.f, __uint_as_float(r[j + 1]), xn), __ldg(cnt + c0 + j + 1)));
                            m2 = fminf(m2, __fadd_rn(__fmaf_rn(-2.f, __uint_as_float(r[j + 2]), xn), __ldg(cnt + c0 + j + 2)));
                            m3 = fminf(m3, __fadd_rn(__fmaf_rn(-2.f, __uint_as_float(r[j + 3]), xn), __ldg(cnt + c0 + j + 3)));
                        }
                    } else if (!removed) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float sv = __fadd_rn(__fmaf_rn(-2.f, __uint_as_float(r[j]), xn), __ldg(cnt + c0 + j));
                            if (sv <= lo_lim) {
                                removed = true;
                            } else if (sv <= hi_lim && !removed) {
                                // undecided: the canonical FP32 distance decides
                                const int64_t ci = (int64_t)t * TC_N + half * (TC_N / 2) + c0 + j;
                                if (ci < a.kc) {
                                    float acc = 0.f;
                                    for (int k = 0; k < a.d; ++k)
                                        acc = sq_step(acc, a.src[gx * a.d + k], a.cen[ci * a.d + k]);
                                    ++namb;
                                    if (__float_as_uint(acc) <= *a.thr) removed = true;
                                }
                            }
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&t_empty[s]);
                ++uses_t[s];
            }
            // combine the two column halves of every row
            const float mmin = fminf(fminf(m0, m1), fminf(m2, m3));
            if (half == 1) {
                s_part[row] = mmin;
                s_gone2[row] = removed ? 1 : 0;
            }
            asm volatile("bar.sync 1, %0;" ::"n"(TC_EPI) : "memory");
            if (half == 0) {
                if (MODE == 0) {
                    const float mm = fminf(mmin, s_part[row]);
                    if (valid) {
                        // bounds on the canonical FP32 minimum over all centers
                        const float lo_r = __fsub_rd(__fsqrt_rd(fmaxf(__fsub_rd(mm, eps), 0.f)), sl);
                        const float lo = lo_r > 0.f ? __fmul_rd(__fmul_rd(lo_r, lo_r), __fsub_rd(1.f, g)) : 0.f;
                        const float hi_r = __fadd_ru(__fsqrt_ru(__fadd_ru(mm, eps)), sl);
                        const float hi = __fmul_ru(__fmul_ru(hi_r, hi_r), __fadd_ru(1.f, g));
                        a.mlo[gx] = lo;
                        a.mhi[gx] = hi;
                        atomicMax(a.mlo_max, __float_as_uint(lo));
                    }
                } else {
                    const bool gone = removed || s_gone2[row] != 0;
                    if (valid && !gone) a.Rn[atomicAdd(a.rnn, 1ull)] = (uint32_t)gx;
                }
            }
            if (MODE == 1 && namb) atomicAdd(a.amb, namb);
            asm volatile("bar.sync 1, %0;" ::"n"(TC_EPI) : "memory");   // s_* reused by the next tile
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_N));
    }
}

// Radius: points whose upper bound can reach the largest lower bound (less
// the FP32-to-FP64 margin) get their exact canonical FP32 minimum (one warp
// per point, lanes over centers); everyone else gets 0.  The key of the
// maximum then equals the one the CUDA-core path produces.
__global__ void tc_exact_kernel(const float *__restrict__ pk, int64_t n, int d, const float *__restrict__ cen,
                                const int32_t *kc_dev, int kc_max, const float *__restrict__ mhi,
                                const unsigned *mlo_max, uint32_t *__restrict__ mind, unsigned long long *key32,
                                const DevStatus *st) {
    if (ld_volatile_i32(&st->code) != 0) return;
    const int kc = kc_dev ? *kc_dev : kc_max;
    const double T = (double)__uint_as_float(*mlo_max) * (1.0 - 3.0 * f32_gamma(d));
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    uint64_t best = 0;
    for (int64_t base = (blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n;
         base += warps * 32) {
        const int64_t x = base + lane;
        const bool flag = x < n && (double)mhi[x] >= T;
        if (x < n && !flag) mind[x] = 0u;
        unsigned todo = __ballot_sync(0xFFFFFFFFu, flag);
        while (todo) {
            const int srcl = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t xs = base + srcl;
            uint32_t m = 0xFFFFFFFFu;
            for (int ci = lane; ci < kc; ci += 32) {
                float acc = 0.f;
                for (int j = 0; j < d; ++j) acc = sq_step(acc, pk[pk_index(xs, j, d)], cen[(int64_t)ci * d + j]);
                m = min(m, __float_as_uint(acc));
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) m = min(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
            if (lane == srcl) {
                mind[xs] = m;
                best = umax64(best, make_key(m, (uint32_t)xs));
            }
        }
    }
    best = warp_max_u64(best);
    if (lane == 0 && best) atomicMax(key32, (unsigned long long)best);
}

int sms() {
    int dev = 0, s = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    return s;
}

// Dynamic shared memory: the A tile and two center tiles, and at least
// 120 KB so that one CTA (holding all 512 TMEM columns) runs per SM.
size_t tc_smem(int kp) {
    const size_t need = (size_t)TC_M * kp * 2 + (size_t)2 * TC_N * kp * 2;
    return need > 120 * 1024 ? need : 120 * 1024;
}

}  // namespace

bool tc_supported(int d) { return d >= 1 && d <= TC_KMAX; }

size_t tc_center_bytes(int kc, int d) {
    const int kp = (d + 15) / 16 * 16;
    const int ntiles = (kc + TC_N - 1) / TC_N;
    return (size_t)ntiles * TC_N * kp * 2;
}

int tc_center_tiles(int kc) { return (kc + TC_N - 1) / TC_N; }

cudaError_t launch_tc_prep(const float *cen, const int32_t *kc_dev, int kc, int d, void *bt, float *cn, unsigned *maxes,
                           cudaStream_t s) {
    const int kp = (d + 15) / 16 * 16;
    const int ntiles = tc_center_tiles(kc);
    cudaMemsetAsync(maxes, 0, 2 * sizeof(unsigned), s);
    const int64_t rows = (int64_t)ntiles * TC_N;
    const int grid = (int)std::min<int64_t>((rows + 255) / 256, (int64_t)sms() * 8);
    tc_prep_kernel<<<grid, 256, 0, s>>>(cen, kc_dev, kc, d, kp, ntiles, (__nv_bfloat16 *)bt, cn, maxes);
    note_launches(1);
    return cudaGetLastError();
}

// Radius bounds for all n points of a packed array; then exact canonical
// minima for the points that can reach the maximum.
cudaError_t launch_tc_radius(const float *pk, int64_t n, int d, const float *cen, const int32_t *kc_dev, int kc,
                             const void *bt, const float *cn, const unsigned *maxes, float *mlo, float *mhi,
                             unsigned *mlo_max, uint32_t *mind, unsigned long long *key32, DevStatus *st,
                             cudaStream_t s) {
    TcArgs a{};
    a.mode = 0;
    a.d = d;
    a.kp = (d + 15) / 16 * 16;
    a.kc = kc;
    a.ntiles = tc_center_tiles(kc);
    a.npts = n;
    a.pk = pk;
    a.bt = (const __nv_bfloat16 *)bt;
    a.cn = cn;
    a.maxes = maxes;
    a.cen = cen;
    a.mlo = mlo;
    a.mhi = mhi;
    a.mlo_max = mlo_max;
    a.st = st;
    const size_t smem = tc_smem(a.kp);
    cudaError_t e = cudaFuncSetAttribute(tc_dmin_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(mlo_max, 0, sizeof(unsigned), s);
    const int64_t tiles = (n + TC_M - 1) / TC_M;
    const int grid = (int)std::min<int64_t>(tiles, (int64_t)sms());
    tc_dmin_kernel<0><<<grid, TC_THREADS, smem, s>>>(a);
    const int g2 = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms() * 8);
    tc_exact_kernel<<<g2, 256, 0, s>>>(pk, n, d, cen, kc_dev, kc, mhi, mlo_max, mind, key32, st);
    note_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_tc_prune(const float *src, int d, const uint32_t *R, int64_t rn, const uint8_t *inS, const float *Scen,
                            int64_t sn, const void *bt, const float *cn, const unsigned *maxes, const uint32_t *thr,
                            uint32_t *Rn, unsigned long long *rnn, unsigned long long *amb, DevStatus *st,
                            cudaStream_t s) {
    TcArgs a{};
    a.mode = 1;
    a.d = d;
    a.kp = (d + 15) / 16 * 16;
    a.kc = (int)sn;
    a.ntiles = tc_center_tiles((int)sn);
    a.npts = rn;
    a.src = src;
    a.R = R;
    a.inS = inS;
    a.bt = (const __nv_bfloat16 *)bt;
    a.cn = cn;
    a.maxes = maxes;
    a.cen = Scen;
    a.thr = thr;
    a.Rn = Rn;
    a.rnn = rnn;
    a.amb = amb;
    a.st = st;
    const size_t smem = tc_smem(a.kp);
    cudaError_t e = cudaFuncSetAttribute(tc_dmin_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (rn + TC_M - 1) / TC_M;
    const int grid = (int)std::min<int64_t>(tiles, (int64_t)sms());
    if (grid > 0) tc_dmin_kernel<1><<<grid, TC_THREADS, smem, s>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace kc
