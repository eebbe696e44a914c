// kc_gon.cu -- persistent Gonzalez kernels: all k farthest-point steps of GON
// (Section 3.1; O(k n) distance evaluations, Section 5.1) in one launch.
//
// An instance is a contiguous index range [lo, lo + n) of a packed point
// array, solved by a group of G CTAs (group mode, cooperative launch) or by
// one CTA that takes instances from a queue (queue mode).  Single GON is one
// instance over the whole array; MRG round 1 (Algorithm 1) is m instances,
// one per part, run side by side with CTA groups sized to the parts; the
// batched many-instance form uses the queue.
//
// Each step, every CTA of the group
//   1. sweeps its blocks of the range (a warp streams one 128-point block:
//      lane l owns points 4l..4l+3 with one 16-byte load per coordinate):
//      squared distance to the newest center (staged in shared memory), the
//      running minimum (written back only where it fell) and the running
//      (value, lowest local index) maximum as a 64-bit key;
//   2. reduces the key over the CTA (shuffles, shared memory, one barrier);
//   3. warp 0 publishes the CTA's key in its slot for this step, polls the
//      group's slots of this step (relaxed loads, all of a lane's slots in
//      flight at once, bounded by a cycle budget), reduces them to the group
//      key, and loads the winner's coordinates for the next step;
//   4. one more barrier hands the key and the new center to the CTA.
// Slots are per step and zeroed before the launch, so a non-zero slot always
// belongs to the current step; the key itself is the payload, so relaxed
// accesses suffice (no other data crosses CTAs).
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "kc_internal.cuh"

namespace kc {

// Diagnostic counters (since the last read):
// [0] exact FP32 rechecks of candidates, [1] candidate-buffer overflows,
// [2] rechecks whose memo was more than a few centers behind (done by a
// whole warp); clock cycles of the mixed-precision GON kernels' phases (CTA
// groups only), summed over CTAs:
// [3] sweep (to the first barrier of a step), [4] exact rechecks (mixed
// precision only), [5] group exchange and center load; the largest of any
// CTA: [6] sweep total, [7] sweep + recheck total.
__device__ unsigned long long g_counters[8];

// Per-CTA phase clock, kept in shared memory (c[0] the last mark, c[1..3]
// the phase totals) and driven by thread 0: mark() adds the cycles since the
// last mark to one phase; publish() adds the totals to g_counters once.
__device__ __forceinline__ void pc_start(long long *c) {
    c[0] = clock64();
    c[1] = c[2] = c[3] = 0;
}
__device__ __forceinline__ void pc_mark(long long *c, int ph) {
    const long long now = clock64();
    c[1 + ph] += now - c[0];
    c[0] = now;
}
__device__ __forceinline__ void pc_publish(const long long *c) {
    for (int i = 0; i < 3; ++i)
        if (c[1 + i] > 0) atomicAdd(&g_counters[3 + i], (unsigned long long)c[1 + i]);
    atomicMax(&g_counters[6], (unsigned long long)c[1]);
    atomicMax(&g_counters[7], (unsigned long long)(c[1] + c[2]));
}

namespace {

constexpr int GROUP_NT = 1024;   // group mode: one CTA per SM
constexpr int QUEUE_NT = 256;    // queue mode: several CTAs per SM

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<int32_t> { using type = int4; };

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <typename T, int DC>
__device__ __forceinline__ void dist4(const T *__restrict__ blk, int d, const T *cs, int lane,
                                      typename AccOf<T>::type acc[4]) {
    using V4 = typename Vec4<T>::type;
    using A = typename AccOf<T>::type;
    const V4 *src = reinterpret_cast<const V4 *>(blk) + lane;
    A a0 = A(0), a1 = A(0), a2 = A(0), a3 = A(0);
    if constexpr (DC > 0) {
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            const V4 v = __ldg(src + j * (BLK / 4));
            const T c = cs[j];
            a0 = sq_step(a0, v.x, c);
            a1 = sq_step(a1, v.y, c);
            a2 = sq_step(a2, v.z, c);
            a3 = sq_step(a3, v.w, c);
        }
    } else {
#pragma unroll 4
        for (int j = 0; j < d; ++j) {
            const V4 v = __ldg(src + j * (BLK / 4));
            const T c = cs[j];
            a0 = sq_step(a0, v.x, c);
            a1 = sq_step(a1, v.y, c);
            a2 = sq_step(a2, v.z, c);
            a3 = sq_step(a3, v.w, c);
        }
    }
    acc[0] = a0;
    acc[1] = a1;
    acc[2] = a2;
    acc[3] = a3;
}

// The blocks of CTA r (of G, W warps each) over [b0, b1] are
// b(i) = b0 + r W + i % W + (i / W) G W for i = 0, 1, ... (increasing in i).
// Within a step the CTA's warps take i from a counter in shared memory (ctr;
// the next index is claimed while the current block is processed), so a warp
// whose loads came back sooner takes more blocks and the CTA's share is done
// when its blocks are, not when its slowest warp's fixed list is.  A block's
// minima stay with the CTA, which orders every step's accesses with its
// barriers.  ctr null: the fixed assignment i = warp + j W.
__device__ __forceinline__ int64_t cta_block(int64_t b0, int r, int G, int W, int i) {
    return b0 + (int64_t)r * W + (i % W) + (int64_t)(i / W) * G * W;
}
__device__ __forceinline__ int claim_block(int *ctr, int lane) {
    int v = 0;
    if (lane == 0) v = atomicAdd(ctr, 1);
    return __shfl_sync(0xFFFFFFFFu, v, 0);
}

// First block of the group's shared tail: with a tail counter, the CTAs own
// the blocks below it (7/8 of the range, whole rounds of G W blocks) and any
// warp of the group claims the rest, two blocks at a time, from a per-step
// counter in global memory, so the group's step ends when its blocks are done
// rather than when the CTA that got the least bandwidth is.  Blocks of the
// tail change CTA from step to step: their minima are read past L1 and every
// step's writes are fenced before the step's slot is published (gon_solve).
__device__ __forceinline__ int64_t tail_start(int64_t b0, int64_t b1, int G, int W, bool tail) {
    if (!tail) return b1 + 1;
    const int64_t GW = (int64_t)G * W;
    const int64_t rounds = (b1 - b0 + 1) * 7 / 8 / GW;
    return rounds >= 2 ? b0 + rounds * GW : b1 + 1;
}

// One step's sweep of this CTA's share (rank r of G) of [lo, lo + n).
template <typename T, int DC, int NT>
__device__ __forceinline__ uint64_t sweep(const T *__restrict__ pk, uint32_t *__restrict__ mind,
                                          int64_t lo, int64_t n, int d, const T *cs, bool first_step,
                                          int r, int G, int *ctr, int *gtail) {
    constexpr int W = NT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t hi = lo + n;
    const int64_t b0 = lo / BLK, b1 = (hi - 1) / BLK;
    uint64_t best = 0;
    // one block: distances to the newest center, the running minima, the key
    auto block = [&](int64_t b) {
        const int64_t g0 = b * BLK + lane * 4;
        const bool full = g0 >= lo && g0 + 3 < hi;
        uint4 *mp = reinterpret_cast<uint4 *>(mind + b * BLK) + lane;
        uint32_t o[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
        if (!first_step) {
            if (full) {
                // past L1 only when tail blocks move between CTAs; a small
                // instance's minima otherwise stay in L1 from step to step
                const uint4 ov = gtail ? __ldcg(mp) : *mp;
                o[0] = ov.x;
                o[1] = ov.y;
                o[2] = ov.z;
                o[3] = ov.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (g0 + q >= lo && g0 + q < hi) o[q] = gtail ? __ldcg(mind + g0 + q) : mind[g0 + q];
            }
        }
        typename AccOf<T>::type acc[4];
        dist4<T, DC>(pk + b * d * BLK, d, cs, lane, acc);
        uint32_t m[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) m[q] = min(o[q], acc_bits(acc[q]));
        if (full) {
            if (first_step || m[0] != o[0] || m[1] != o[1] || m[2] != o[2] || m[3] != o[3])
                *mp = make_uint4(m[0], m[1], m[2], m[3]);
#pragma unroll
            for (int q = 0; q < 4; ++q) best = umax64(best, make_key(m[q], (uint32_t)(g0 + q - lo)));
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t g = g0 + q;
                if (g >= lo && g < hi) {
                    if (first_step || m[q] != o[q]) mind[g] = m[q];
                    best = umax64(best, make_key(m[q], (uint32_t)(g - lo)));
                }
            }
        }
    };
    if (!ctr && !gtail) {
        // the fixed assignment: warp w of CTA r takes blocks b0 + r W + w + j G W
        for (int64_t b = b0 + (int64_t)r * W + warp; b <= b1; b += (int64_t)G * W) block(b);
        return best;
    }
    const int64_t ts = tail_start(b0, b1, G, W, gtail != nullptr);
    int nxt = ctr ? claim_block(ctr, lane) : warp;
    int64_t pend = -1;   // second block of a claimed tail pair
    for (;;) {
        int64_t b = cta_block(b0, r, G, W, nxt);
        if (b < ts) {
            nxt = ctr ? claim_block(ctr, lane) : nxt + W;
        } else if (ts > b1) {
            break;
        } else if (pend >= 0) {
            b = pend;
            pend = -1;
        } else {
            int t = 0;
            if (lane == 0) t = atomicAdd(gtail, 2);
            t = __shfl_sync(0xFFFFFFFFu, t, 0);
            b = ts + t;
            if (b > b1) break;
            if (b + 1 <= b1) pend = b + 1;
        }
        block(b);
    }
    return best;
}

// Warp 0: wait for all G slots of this step and return their maximum.
__device__ uint64_t poll_slots(const uint64_t *slots, int G, long long timeout, DevStatus *st,
                               int step, bool *abort_out) {
    const int lane = threadIdx.x & 31;
    uint64_t g = 0;
    bool ab = false;
    for (int s0 = 0; s0 < G && !ab; s0 += 128) {
        uint64_t v[4];
        unsigned pend = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (s0 + q * 32 + lane < G) pend |= 1u << q;
        const long long t0 = clock64();
        while (pend) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (pend >> q & 1u) v[q] = ld_relaxed_u64(slots + s0 + q * 32 + lane);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if ((pend >> q & 1u) && v[q] != 0) {
                    g = umax64(g, v[q]);
                    pend &= ~(1u << q);
                }
            if (pend && (clock64() - t0 > timeout || ld_volatile_i32(&st->code) != 0)) {
                set_status(st, KC_ERR_TIMEOUT, 3, step);
                ab = true;
                break;
            }
        }
    }
    *abort_out = __any_sync(0xFFFFFFFFu, ab);
    return warp_max_u64(g);
}

__device__ __forceinline__ int64_t out_index(const GonInst &I, int64_t local) {
    return I.map ? I.map[local] : I.base + local;
}

struct Shared {
    uint64_t red[32];
    uint64_t key;
    int abort;
    int ctr[2];   // block counters of even and odd steps
};

// All k steps of one instance by this CTA (rank r of a group of G).  DYN:
// the instance is large enough for claimed blocks and the shared tail (a
// separate instantiation, so that small instances run the plain loop).
template <typename T, int DC, int NT, bool DYN = false>
__device__ void gon_solve(const GonInst &I, int r, int G, T *cs, Shared &sh, DevStatus *st,
                          long long timeout, int withhold = 0, bool bad_index = false) {
    constexpr int W = NT / 32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int d = DC > 0 ? DC : I.d;
    const T *pk = (const T *)I.pk;
    if (warp == 0) {
        for (int j = lane; j < d; j += 32) cs[j] = pk[pk_index(I.lo + I.first, j, d)];
        if (lane == 0) {
            sh.abort = 0;
            sh.ctr[0] = sh.ctr[1] = 0;
        }
    }
    if (r == 0 && tid == 0) I.centers[0] = out_index(I, I.first);
    __syncthreads();
    const bool claim = DYN && NT == GROUP_NT && (I.lo + I.n - 1) / BLK - I.lo / BLK + 1 >= 4 * (int64_t)G * W;
    const bool tail = DYN && G > 1 && I.tail != nullptr;

    int it;
    uint64_t K = 0;
    for (it = 0; it < I.k; ++it) {
        // claimed blocks in the 1024-thread group CTAs when every warp has
        // several (measured: GON on 8M x 64, k = 1024, 313 -> 308 ms); the
        // fixed assignment in the 256-thread queue CTAs (MRG round 1 on
        // 10M x 16 was 5% slower with claims) and for small instances
        uint64_t best = sweep<T, DC, NT>(pk, I.mind, I.lo, I.n, d, cs, it == 0, r, G,
                                         claim ? &sh.ctr[it & 1] : nullptr, tail ? I.tail + it : nullptr);
        best = warp_max_u64(best);
        if (lane == 0) sh.red[warp] = best;
        __syncthreads();
        if (DYN && tid == 0) sh.ctr[(it + 1) & 1] = 0;   // the next step's counter (last used a step ago)
        if (warp == 0) {
            uint64_t v = lane < W ? sh.red[lane] : 0;
            v = warp_max_u64(v);
            uint64_t g = v;
            bool ab = false;
            if (G > 1) {
                const int64_t row = (int64_t)it * slot_stride(G);
                const bool held = withhold == it + 1 && r == G - 1;
                // with a shared tail, the step's minima (written by this
                // CTA's threads before the barrier) are made visible to the
                // group before the slot is, and the other CTAs' after it is
                // seen (the release / acquire pattern of a grid barrier)
                if (tail) __threadfence();
                if (lane == 0 && !held) st_relaxed_u64(&I.slots[row + r], v ? v : 1);
                g = poll_slots(I.slots + row, G, timeout, st, it, &ab);
                if (tail) __threadfence();
            }
            if (!ab && key_val(g) != 0 && it + 1 < I.k) {
#ifdef KC_CHECKS
                // testing hook of the checked build: a winner index one past
                // the instance, which the check below must catch
                const int64_t c = (bad_index && it == 0) ? I.n : (int64_t)key_idx(g);
#else
                const int64_t c = key_idx(g);
#endif
                if (KC_IN_RANGE(st, c, I.n, KC_AT_CENTER_LOAD)) {
                    for (int j = lane; j < d; j += 32) cs[j] = pk[pk_index(I.lo + c, j, d)];
                    if (r == 0 && lane == 0) I.centers[it + 1] = out_index(I, c);
                } else {
                    ab = true;
                }
            }
            if (lane == 0) {
                sh.key = g;
                sh.abort = ab;
            }
        }
        __syncthreads();
        if (sh.abort) return;
        K = sh.key;
        if (key_val(K) == 0) {   // every point is at distance 0: stop early
            ++it;
            break;
        }
    }
    if (r == 0 && tid == 0) {
        *I.k_out = it;
        *I.final_key = K;
    }
}

// ------------------------------------------------- mixed-precision sweep
//
// The sweep streams the low-precision words instead of FP32 coordinates and
// keeps m~(x), the running minimum of the FP32-evaluated squared distance
// between decoded(x) and decoded(c).  With u = 2^-24, g = (d+2)u/(1-(d+2)u)
// + 2^-20, e_x the point's bound (its block's maximum) and E the largest
// bound of any center so far, the canonical FP32 minimum m32(x) satisfies
//   L(x) = (1-g)(sqrt(m~)(1-g) - e_x - E) <= sqrt(m32(x)) <= U(x)
//        = (1+g)(sqrt(m~)(1+g) + e_x + E)
// (triangle inequality on ||.||_2, both FP32 evaluations within (1 +- g));
// U and L are evaluated with directed rounding.  A CTA takes T = max L over
// its points; a point with U(x) < T cannot be the CTA's exact argmax (nor tie
// with it), so only points with U(x) >= T are recomputed exactly (canonical
// FP32 against every center so far, from the FP32 points and the centers'
// FP32 coordinates) and the CTA key is the exact maximum over them, equal to
// the FP32 sweep's.  Candidates are collected during the sweep in a per-warp
// buffer against the warp's running max L; if it overflows, the warp
// rescans its running minima instead.
template <int KIND> struct LPDec;
template <> struct LPDec<KC_SWEEP_BF16> {
    __device__ static __forceinline__ void dec(uint32_t w, const float *, float o[2]) {
        o[0] = __uint_as_float(w << 16);
        o[1] = __uint_as_float(w & 0xFFFF0000u);
    }
};
// fp16 codes decode to their fp16 values, in the pack's scaled units (the
// sweep never leaves them).
template <> struct LPDec<KC_SWEEP_FP16> {
    __device__ static __forceinline__ void dec(uint32_t w, const float *, float o[2]) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w));
        o[0] = f.x;
        o[1] = f.y;
    }
};
template <> struct LPDec<KC_SWEEP_FP8> {
    __device__ static __forceinline__ void dec(uint32_t w, const float *sc, float o[4]) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)((w >> (8 * t)) & 0xFFu), __NV_E4M3);
            o[t] = __fmul_rn(__half2float(__half(h)), sc[t]);
        }
    }
};

struct Cand {
    uint32_t idx;   // local index
    float U;
};
constexpr int LP_CAP = 128;   // candidates per warp

struct ShLP {
    uint64_t red[32];
    uint64_t key;
    unsigned Lcta;     // largest positive lower bound L published by a warp this step (float bits)
    float Tg;          // the group's largest L this step
    long long pc[4];
    float Lw[32];
    int ovf[32];
    int cnt[32];
    float ecmax;
    int abort;
};


// Canonical FP32 minimum of point gx over the first ncen centers (cenT is
// [d][kcap]), from the memo: m32[gx] holds the exact minimum over centers
// [0, stamp[gx]), so only centers [stamp, ncen) are evaluated; the memo is
// then advanced to ncen.  A point is rechecked by the one warp that owns its
// block (the same in every step), so the memo needs no atomics.
constexpr int MEMO_LANE_GAP = 4;   // gaps up to this many centers: one lane per point

// Canonical FP32 squared distance of packed point gx and center i of cenT,
// loads issued four coordinates at a time (coordinates past d are zero
// pairs, whose term fma(0, 0, acc) leaves acc unchanged).  row: the point's
// FP32 row when the instance has one (then read with 16-byte loads, all of
// them in flight at once, when d % 4 == 0 and the row is aligned).
template <bool VEC>
__device__ __forceinline__ float memo_dist(const float *__restrict__ pk, int64_t gx, int d,
                                           const float *__restrict__ cenT, int kcap, int i,
                                           const float *__restrict__ row) {
    float acc = 0.f;
    if (row) {
        if (VEC && (d & 3) == 0 && ((uintptr_t)row & 15) == 0) {
            const float4 *r4 = reinterpret_cast<const float4 *>(row);
            for (int q0 = 0; q0 < d / 4; q0 += 4) {
                float4 xv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (q0 + u < d / 4) xv[u] = __ldg(r4 + q0 + u);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (q0 + u < d / 4) {
                        const int j = 4 * (q0 + u);
                        acc = sq_step(acc, xv[u].x, cenT[(int64_t)j * kcap + i]);
                        acc = sq_step(acc, xv[u].y, cenT[(int64_t)(j + 1) * kcap + i]);
                        acc = sq_step(acc, xv[u].z, cenT[(int64_t)(j + 2) * kcap + i]);
                        acc = sq_step(acc, xv[u].w, cenT[(int64_t)(j + 3) * kcap + i]);
                    }
            }
        } else {
            for (int j = 0; j < d; ++j) acc = sq_step(acc, __ldg(row + j), cenT[(int64_t)j * kcap + i]);
        }
        return acc;
    }
    for (int j0 = 0; j0 < d; j0 += 4) {
        float xv[4], cv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + u;
            xv[u] = j < d ? pk[pk_index(gx, j, d)] : 0.f;
            cv[u] = j < d ? cenT[(int64_t)j * kcap + i] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc = sq_step(acc, xv[u], cv[u]);
    }
    return acc;
}

// One lane, centers [stamp, ncen) in order.
template <bool VEC>
__device__ __forceinline__ uint32_t memo_min_lane(const float *__restrict__ pk, int64_t gx, int d,
                                                  const float *__restrict__ cenT, int kcap, int ncen,
                                                  uint32_t *__restrict__ m32, uint32_t *__restrict__ stamp,
                                                  const float *__restrict__ row) {
    const int s0 = (int)stamp[gx];
    uint32_t m = s0 ? m32[gx] : 0xFFFFFFFFu;
    for (int i = s0; i < ncen; ++i) m = min(m, __float_as_uint(memo_dist<VEC>(pk, gx, d, cenT, kcap, i, row)));
    m32[gx] = m;
    stamp[gx] = (uint32_t)ncen;
    return m;
}

// The whole warp: lane l takes centers stamp + l, stamp + l + 32, ...
template <bool VEC>
__device__ uint32_t memo_min_warp(const float *__restrict__ pk, int64_t gx, int d, const float *__restrict__ cenT,
                                  int kcap, int ncen, uint32_t *__restrict__ m32, uint32_t *__restrict__ stamp,
                                  int lane, const float *__restrict__ row) {
    const int s0 = (int)stamp[gx];
    uint32_t m = s0 ? m32[gx] : 0xFFFFFFFFu;
    for (int i = s0 + lane; i < ncen; i += 32)
        m = min(m, __float_as_uint(memo_dist<VEC>(pk, gx, d, cenT, kcap, i, row)));
#pragma unroll
    for (int o = 16; o; o >>= 1) m = min(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    __syncwarp();
    if (lane == 0) {
        m32[gx] = m;
        stamp[gx] = (uint32_t)ncen;
    }
    __syncwarp();
    return m;
}

// Exact values of the points lanes flag (want; local index idx): small gaps
// lane by lane, the rest one at a time by the whole warp.  Updates the lane's
// best key and recheck count.
template <bool VEC>
__device__ __forceinline__ void memo_recheck(const GonInst &I, const float *__restrict__ pk, int d, int ncen,
                                             bool want, uint32_t idx, int lane, uint64_t &best, unsigned &nre,
                                             DevStatus *st) {
    want = want && KC_IN_RANGE(st, idx, I.n, KC_AT_RECHECK);
    const int64_t gx = I.lo + idx;
    const bool small = want && ncen - (int)I.stamp[gx] <= MEMO_LANE_GAP;
    if (small) {
        const uint32_t mm = memo_min_lane<VEC>(pk, gx, d, I.cenT, I.kcap, ncen, I.m32, I.stamp,
                                          I.rm ? I.rm + (int64_t)idx * d : nullptr);
        best = umax64(best, make_key(mm, idx));
        ++nre;
    }
    unsigned big = __ballot_sync(0xFFFFFFFFu, want && !small);
    if (big && lane == 0) atomicAdd(&g_counters[2], (unsigned long long)__popc(big));
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        const uint32_t bidx = __shfl_sync(0xFFFFFFFFu, idx, src);
        const uint32_t mm = memo_min_warp<VEC>(pk, I.lo + bidx, d, I.cenT, I.kcap, ncen, I.m32, I.stamp, lane,
                                          I.rm ? I.rm + (int64_t)bidx * d : nullptr);
        if (lane == src) {
            best = umax64(best, make_key(mm, bidx));
            ++nre;
        }
    }
}

// In-place removal of buffer entries with U < lim (warp-cooperative).
__device__ __forceinline__ int lp_compact(Cand *buf, int cnt, float lim, int lane) {
    int out = 0;
    for (int e0 = 0; e0 < cnt; e0 += 32) {
        const int e = e0 + lane;
        Cand c = {0u, 0.f};
        const bool keep = e < cnt && (c = buf[e]).U >= lim;
        __syncwarp();
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
        if (keep) buf[out + __popc(bal & ((1u << lane) - 1u))] = c;
        out += __popc(bal);
        __syncwarp();
    }
    return out;
}

// Order-preserving 64-bit code of a float lower bound for the slot exchange
// (non-zero, so a published slot is never mistaken for an empty one).
__device__ __forceinline__ uint64_t enc_bound(float T) {
    const uint32_t u = __float_as_uint(T);
    return (1ull << 32) | (uint64_t)((u & 0x80000000u) ? ~u : (u | 0x80000000u));
}
__device__ __forceinline__ float dec_bound(uint64_t v) {
    const uint32_t o = (uint32_t)v;
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}

// The decoded low-precision center, its bound, and its FP32 coordinates
// appended to cenT (every CTA of the group writes the same values).
template <int KIND>
__device__ __forceinline__ void lp_load_center(const GonInst &I, int64_t c, int d, int ng, float *cl, const float *scs,
                                               int slot, int lane, float *ec) {
    constexpr int LG = lp_group(KIND);
    const float *__restrict__ pk = (const float *)I.pk;
    const int64_t g = I.lo + c;
    // every load first (one memory round trip for all of them), then the
    // stores: the winner's words, FP32 coordinates (d <= 32 * 8 per lane
    // here, the rest in a second pass) and bound
    constexpr int NW = 4, NX = 8;
    uint32_t w[NW];
    float xv[NX];
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        const int jg = lane + 32 * q;
        w[q] = jg < ng ? __ldg(I.lp + ((g / BLK) * ng + jg) * BLK + g % BLK) : 0u;
    }
#pragma unroll
    for (int q = 0; q < NX; ++q) {
        const int j = lane + 32 * q;
        xv[q] = j < d ? __ldg(pk + pk_index(g, j, d)) : 0.f;
    }
    const float e = __ldg(I.ept + g);
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        const int jg = lane + 32 * q;
        if (jg < ng) {
            float v[LG];
            LPDec<KIND>::dec(w[q], scs + jg * LG, v);
#pragma unroll
            for (int t = 0; t < LG; ++t) cl[jg * LG + t] = v[t];
        }
    }
    for (int jg = lane + 32 * NW; jg < ng; jg += 32) {
        float v[LG];
        LPDec<KIND>::dec(I.lp[((g / BLK) * ng + jg) * BLK + g % BLK], scs + jg * LG, v);
#pragma unroll
        for (int t = 0; t < LG; ++t) cl[jg * LG + t] = v[t];
    }
#pragma unroll
    for (int q = 0; q < NX; ++q) {
        const int j = lane + 32 * q;
        if (j < d) I.cenT[(int64_t)j * I.kcap + slot] = xv[q];
    }
    for (int j = lane + 32 * NX; j < d; j += 32) I.cenT[(int64_t)j * I.kcap + slot] = pk[pk_index(g, j, d)];
    *ec = e;
}

template <int KIND, int DC, int NT>
__device__ void gon_solve_lp(const GonInst &I, int r, int G, float *smem, ShLP &sh, DevStatus *st, long long timeout,
                             int withhold = 0, bool local_t = false) {
    constexpr int W = NT / 32;
    constexpr int LG = lp_group(KIND);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int d = DC > 0 ? DC : I.d;
    const int ng = (d + LG - 1) / LG;
    const int dp = ng * LG;
    float *cl = smem;                                  // [dp] decoded center
    float *scs = smem + dp;                            // [dp] fp8 scales
    Cand *buf = reinterpret_cast<Cand *>(smem + 2 * ((dp + 1) & ~1)) + warp * LP_CAP;
    const float *pk = (const float *)I.pk;
    const bool clk = G > 1;   // phase clocks for CTA groups (queue instances are too short to time)
    const float g1 = lp_slack(d);
    const float opg = __fadd_ru(1.f, g1), omg = __fsub_rd(1.f, g1);
    const int64_t lo = I.lo, hi = I.lo + I.n, b1 = (hi - 1) / BLK;

    for (int j = tid; j < dp; j += NT) scs[j] = (KIND == KC_SWEEP_FP8) ? I.scale[j] : 1.f;
    __syncthreads();
    // fixed assignment of the CTA's blocks to its warps (claiming them from a
    // counter, as the FP32 sweep does, measured slower here: 183 -> 188 ms
    // per solve on 8M x 64, k = 1024)
    const int64_t b0 = lo / BLK;
    if (warp == 0) {
        float ec;
        lp_load_center<KIND>(I, I.first, d, ng, cl, scs, 0, lane, &ec);
        if (lane == 0) {
            sh.ecmax = ec;
            sh.abort = 0;
            sh.Lcta = 0u;
        }
    }
    if (r == 0 && tid == 0) I.centers[0] = out_index(I, I.first);
    __syncthreads();

    int it;
    uint64_t K = 0;
    if (clk && tid == 0) pc_start(sh.pc);
    volatile unsigned *Lcta = &sh.Lcta;
    for (it = 0; it < I.k; ++it) {
        const float ecmax = sh.ecmax;
        float Lrun = -INFINITY;
        int cnt = 0;
        bool ovf = false;
        for (int bi = warp;; bi += W) {
            const int64_t b = cta_block(b0, r, G, W, bi);
            if (b > b1) break;
            const int64_t g0 = b * BLK + lane * 4;
            const uint4 *src = reinterpret_cast<const uint4 *>(I.lp + b * ng * BLK) + lane;
            float a[4] = {0.f, 0.f, 0.f, 0.f};
            if constexpr (DC > 0) {
#pragma unroll 4
                for (int jg = 0; jg < (DC + LG - 1) / LG; ++jg) {
                    const uint4 w = __ldg(src + jg * (BLK / 4));
                    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float v[LG];
                        LPDec<KIND>::dec(ws[q], scs + jg * LG, v);
#pragma unroll
                        for (int t = 0; t < LG; ++t) {
                            const float df = __fsub_rn(v[t], cl[jg * LG + t]);
                            a[q] = __fmaf_rn(df, df, a[q]);
                        }
                    }
                }
            } else {
                for (int jg = 0; jg < ng; ++jg) {
                    const uint4 w = __ldg(src + jg * (BLK / 4));
                    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float v[LG];
                        LPDec<KIND>::dec(ws[q], scs + jg * LG, v);
#pragma unroll
                        for (int t = 0; t < LG; ++t) {
                            const float df = __fsub_rn(v[t], cl[jg * LG + t]);
                            a[q] = __fmaf_rn(df, df, a[q]);
                        }
                    }
                }
            }
            // Running minimum of the approximate values, kept in 16 bits: the
            // float bits shifted right by 16 (bf16 rounded toward zero).
            // Truncation commutes with min, so the stored code t satisfies
            // lo(t) <= m~ < hi(t) with lo(t) = t << 16, hi(t) = (t + 1) << 16.
            const bool full = g0 >= lo && g0 + 3 < hi;
            uint32_t o[4] = {0xFFFFu, 0xFFFFu, 0xFFFFu, 0xFFFFu};
            uint16_t *m16 = reinterpret_cast<uint16_t *>(I.mind);
            uint2 *mp = reinterpret_cast<uint2 *>(m16 + b * BLK) + lane;
            if (it > 0) {
                if (full) {
                    const uint2 ov = *mp;
                    o[0] = ov.x & 0xFFFFu;
                    o[1] = ov.x >> 16;
                    o[2] = ov.y & 0xFFFFu;
                    o[3] = ov.y >> 16;
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (g0 + q >= lo && g0 + q < hi) o[q] = m16[g0 + q];
                }
            }
            uint32_t m[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) m[q] = min(o[q], __float_as_uint(a[q]) >> 16);
            if (full) {
                if (it == 0 || m[0] != o[0] || m[1] != o[1] || m[2] != o[2] || m[3] != o[3])
                    *mp = make_uint2(m[0] | (m[1] << 16), m[2] | (m[3] << 16));
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (g0 + q >= lo && g0 + q < hi && (it == 0 || m[q] != o[q])) m16[g0 + q] = (uint16_t)m[q];
            }
            // Bounds.  L and U increase with m~ and delta is per block, so the
            // block's largest L comes from its largest code, and U(x) >= Lrun
            // holds iff hi(x) >= tau with tau = ((Lrun/(1+g) - delta)/(1+g))^2;
            // tau is rounded down (admitting a superset), so no per-point
            // square root is needed.  U is evaluated only for admitted points.
            const float delta = __fadd_ru(I.eblk[b], ecmax);
            uint32_t mmax = 0;
            bool anyv = false;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (g0 + q >= lo && g0 + q < hi) {
                    mmax = max(mmax, m[q]);
                    anyv = true;
                }
            float bl = anyv ? lp_lower(mmax << 16, delta, omg) : -INFINITY;
#pragma unroll
            for (int o2 = 16; o2; o2 >>= 1) bl = fmaxf(bl, __shfl_xor_sync(0xFFFFFFFFu, bl, o2));
            Lrun = fmaxf(Lrun, bl);
            // admission against the CTA's largest L so far (<= the final T)
            if (lane == 0 && Lrun > 0.f) atomicMax(&sh.Lcta, __float_as_uint(Lrun));
            const float Lc = fmaxf(Lrun, __uint_as_float(*Lcta));
            if (!ovf) {
                const float a0 = __fsub_rd(__fdiv_rd(Lc, opg), delta);
                const float t0 = a0 > 0.f ? __fdiv_rd(a0, opg) : 0.f;
                const uint32_t tau = __float_as_uint(__fmul_rd(t0, t0));
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t hib = (m[q] + 1u) << 16;
                    const bool pred = g0 + q >= lo && g0 + q < hi && hib >= tau;
                    const unsigned bal = __ballot_sync(0xFFFFFFFFu, pred);
                    const int nq = __popc(bal);
                    if (nq == 0) continue;
                    if (cnt + nq > LP_CAP) {
                        cnt = lp_compact(buf, cnt, Lc, lane);
                        if (cnt + nq > LP_CAP) {
                            ovf = true;
                            break;
                        }
                    }
                    if (pred && KC_IN_RANGE(st, cnt + __popc(bal & ((1u << lane) - 1u)), LP_CAP, KC_AT_CANDIDATE))
                        buf[cnt + __popc(bal & ((1u << lane) - 1u))] =
                            Cand{(uint32_t)(g0 + q - lo), lp_upper(hib, delta, opg)};
                    cnt += nq;
                }
            }
        }
        if (lane == 0) {
            sh.Lw[warp] = Lrun;
            sh.ovf[warp] = ovf;
            sh.cnt[warp] = cnt;
        }
        __syncthreads();
        if (clk && tid == 0) pc_mark(sh.pc, 0);
        float T = -INFINITY;
        for (int w = 0; w < W; ++w) T = fmaxf(T, sh.Lw[w]);
        if (G > 1 && !local_t) {
            // The group's largest lower bound: a point whose upper bound is
            // below it is strictly below that point's exact value, so only
            // candidates reaching it are rechecked (slots [k G, 2 k G)).
            if (warp == 0) {
                bool ab = false;
                uint64_t *ts = I.slots + ((int64_t)I.k + it) * slot_stride(G);
                if (lane == 0) st_relaxed_u64(ts + r, enc_bound(T));
                const uint64_t tg = poll_slots(ts, G, timeout, st, it, &ab);
                if (lane == 0) {
                    sh.Tg = dec_bound(tg);
                    if (ab) sh.abort = 1;
                }
            }
            __syncthreads();
            if (clk && tid == 0) pc_mark(sh.pc, 2);
            if (sh.abort) break;
            T = sh.Tg;
        }
        // exact recheck of this warp's candidates with U >= T
        uint64_t best = 0;
        const int ncen = it + 1;
        unsigned nre = 0;
        if (!ovf) {
            __syncwarp();
            for (int e0 = 0; e0 < cnt; e0 += 32) {
                const int e = e0 + lane;
                Cand c = {0u, -INFINITY};
                if (e < cnt) c = buf[e];
                memo_recheck<(DC > 0)>(I, pk, d, ncen, e < cnt && c.U >= T, c.idx, lane, best, nre, st);
            }
        } else {
            // the buffer overflowed: rescan the warp's running minima against
            // the final T, buffering the survivors and rechecking them 32 at a
            // time
            if (lane == 0) atomicAdd(&g_counters[1], 1ull);
            int c2 = 0;
            __syncwarp();
            for (int bi = warp;; bi += W) {
                const int64_t b = cta_block(b0, r, G, W, bi);
                if (b > b1) break;
                const float delta = __fadd_ru(I.eblk[b], ecmax);
#pragma unroll 1
                for (int q = 0; q < 4; ++q) {
                    const int64_t g = b * BLK + lane * 4 + q;
                    const bool pred =
                        g >= lo && g < hi &&
                        lp_upper(((uint32_t)reinterpret_cast<const uint16_t *>(I.mind)[g] + 1u) << 16, delta, opg) >=
                            T;
                    const unsigned bal = __ballot_sync(0xFFFFFFFFu, pred);
                    if (pred && KC_IN_RANGE(st, c2 + __popc(bal & ((1u << lane) - 1u)), LP_CAP, KC_AT_CANDIDATE))
                        buf[c2 + __popc(bal & ((1u << lane) - 1u))] = Cand{(uint32_t)(g - lo), 0.f};
                    c2 += __popc(bal);
                    if (c2 > LP_CAP - 32) {
                        __syncwarp();
                        for (int e0 = 0; e0 < c2; e0 += 32)
                            memo_recheck<(DC > 0)>(I, pk, d, ncen, e0 + lane < c2, e0 + lane < c2 ? buf[e0 + lane].idx : 0u,
                                         lane, best, nre, st);
                        c2 = 0;
                        __syncwarp();
                    }
                }
            }
            __syncwarp();
            for (int e0 = 0; e0 < c2; e0 += 32)
                memo_recheck<(DC > 0)>(I, pk, d, ncen, e0 + lane < c2, e0 + lane < c2 ? buf[e0 + lane].idx : 0u, lane, best,
                             nre, st);
        }
        nre = __reduce_add_sync(0xFFFFFFFFu, nre);
        if (lane == 0 && nre) atomicAdd(&g_counters[0], (unsigned long long)nre);
        best = warp_max_u64(best);
        if (lane == 0) sh.red[warp] = best;
        __syncthreads();
        if (clk && tid == 0) pc_mark(sh.pc, 1);
        if (warp == 0) {
            uint64_t v = lane < W ? sh.red[lane] : 0;
            v = warp_max_u64(v);
            uint64_t g = v;
            bool ab = false;
            if (G > 1) {
                const int64_t row = (int64_t)it * slot_stride(G);
                const bool held = withhold == it + 1 && r == G - 1;
                if (lane == 0 && !held) st_relaxed_u64(&I.slots[row + r], v ? v : 1);
                g = poll_slots(I.slots + row, G, timeout, st, it, &ab);
            }
            if (lane == 0) sh.Lcta = 0u;   // next step's admission bound starts over
            if (!ab && key_val(g) != 0 && it + 1 < I.k) {
                const int64_t c = key_idx(g);
                if (KC_IN_RANGE(st, c, I.n, KC_AT_CENTER_LOAD) && KC_IN_RANGE(st, it + 1, I.kcap, KC_AT_CENTER_COPY)) {
                    float ec;
                    lp_load_center<KIND>(I, c, d, ng, cl, scs, it + 1, lane, &ec);
                    if (lane == 0) sh.ecmax = fmaxf(sh.ecmax, ec);
                    if (r == 0 && lane == 0) I.centers[it + 1] = out_index(I, c);
                } else {
                    ab = true;
                }
            }
            if (lane == 0) {
                sh.key = g;
                sh.abort = ab;
            }
        }
        __syncthreads();
        if (clk && tid == 0) pc_mark(sh.pc, 2);
        if (sh.abort) break;
        K = sh.key;
        if (key_val(K) == 0) {
            ++it;
            break;
        }
    }
    if (clk && tid == 0) pc_publish(sh.pc);
    if (sh.abort) return;
    if (r == 0 && tid == 0) {
        *I.k_out = it;
        *I.final_key = K;
        if (I.ecmax_out) *I.ecmax_out = sh.ecmax;
    }
}

template <typename T>
__device__ bool instance_ok(const GonInst &I, DevStatus *st) {
    if constexpr (std::is_same<T, int32_t>::value) {
        if (!int_range_ok(I.range2, I.d)) {
            set_status(st, KC_ERR_RANGE, 2, 0);
            return false;
        }
    }
    return true;
}

// Last instance of insts[0, m) whose CTA group starts at or before this CTA.
__device__ __forceinline__ void find_group(const GonInst *insts, int m, GonInst &I) {
    int lo = 0, hi = m - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (insts[mid].cta0 <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    I = insts[lo];
}

template <typename T, int DC, bool DYN>
__global__ void __launch_bounds__(GROUP_NT, 1) gon_group_kernel(GonArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *cs = reinterpret_cast<T *>(smem_raw);
    __shared__ GonInst I;
    __shared__ Shared sh;
    if (threadIdx.x == 0) {
        if (a.insts) find_group(a.insts, a.ninst, I);
        else I = a.single;
    }
    __syncthreads();
    const int r = (int)blockIdx.x - I.cta0;
    if (r < 0 || r >= I.G) return;
    if (ld_volatile_i32(&a.st->code) != 0) return;
    if (!instance_ok<T>(I, a.st)) return;
    gon_solve<T, DC, GROUP_NT, DYN>(I, r, I.G, cs, sh, a.st, a.timeout_cycles, a.withhold, a.bad_index != 0);
}

// Queue mode, optionally with heavy instances in front: insts[0, nheavy)
// are solved by CTA groups [cta0, cta0 + G) of the first gheavy CTAs (the
// launch is then cooperative, so the groups are co-resident); every CTA then
// takes the remaining instances insts[nheavy, ninst) one at a time, in order.
template <typename T, int DC>
__global__ void __launch_bounds__(QUEUE_NT) gon_queue_kernel(GonArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *cs = reinterpret_cast<T *>(smem_raw);
    __shared__ GonInst I;
    __shared__ Shared sh;
    __shared__ int s_i;
    if ((int)blockIdx.x < a.gheavy) {
        if (threadIdx.x == 0) find_group(a.insts, a.nheavy, I);
        __syncthreads();
        const int r = (int)blockIdx.x - I.cta0;
        if (r >= 0 && r < I.G && ld_volatile_i32(&a.st->code) == 0 && instance_ok<T>(I, a.st))
            gon_solve<T, DC, QUEUE_NT>(I, r, I.G, cs, sh, a.st, a.timeout_cycles);
        __syncthreads();
    }
    for (;;) {
        if (threadIdx.x == 0) {
            s_i = a.nheavy + atomicAdd(a.counter, 1);
            if (s_i < a.ninst) I = a.insts[s_i];
        }
        __syncthreads();
        if (s_i >= a.ninst) return;
        if (ld_volatile_i32(&a.st->code) != 0) return;
        if (instance_ok<T>(I, a.st)) gon_solve<T, DC, QUEUE_NT>(I, 0, 1, cs, sh, a.st, a.timeout_cycles);
        __syncthreads();
    }
}

__device__ __forceinline__ void find_instance(const GonArgs &a, GonInst &I) {
    if (a.insts) find_group(a.insts, a.ninst, I);
    else I = a.single;
}

template <int KIND, int DC>
__global__ void __launch_bounds__(GROUP_NT, 1) gon_group_lp_kernel(GonArgs a) {
    extern __shared__ __align__(16) float smem_f[];
    __shared__ GonInst I;
    __shared__ ShLP sh;
    if (threadIdx.x == 0) find_instance(a, I);
    __syncthreads();
    const int r = (int)blockIdx.x - I.cta0;
    if (r < 0 || r >= I.G) return;
    if (ld_volatile_i32(&a.st->code) != 0) return;
    gon_solve_lp<KIND, DC, GROUP_NT>(I, r, I.G, smem_f, sh, a.st, a.timeout_cycles, a.withhold, a.lp_local_t != 0);
}

template <int KIND, int DC>
__global__ void __launch_bounds__(QUEUE_NT, 4) gon_queue_lp_kernel(GonArgs a) {
    extern __shared__ __align__(16) float smem_f[];
    __shared__ GonInst I;
    __shared__ ShLP sh;
    __shared__ int s_i;
    if ((int)blockIdx.x < a.gheavy) {
        if (threadIdx.x == 0) find_group(a.insts, a.nheavy, I);
        __syncthreads();
        const int r = (int)blockIdx.x - I.cta0;
        if (r >= 0 && r < I.G && ld_volatile_i32(&a.st->code) == 0)
            gon_solve_lp<KIND, DC, QUEUE_NT>(I, r, I.G, smem_f, sh, a.st, a.timeout_cycles, 0, a.lp_local_t != 0);
        __syncthreads();
    }
    for (;;) {
        if (threadIdx.x == 0) {
            s_i = a.nheavy + atomicAdd(a.counter, 1);
            if (s_i < a.ninst) I = a.insts[s_i];
        }
        __syncthreads();
        if (s_i >= a.ninst) return;
        if (ld_volatile_i32(&a.st->code) != 0) return;
        gon_solve_lp<KIND, DC, QUEUE_NT>(I, 0, 1, smem_f, sh, a.st, a.timeout_cycles);
        __syncthreads();
    }
}

// ------------------------------------------------ resident single GON
//
// For one instance whose points fit on chip across the grid (one CTA per SM),
// every CTA keeps its contiguous share [lo_r, hi_r) of the rows for all k
// steps: local point t + j * 1024 belongs to thread t; j = 0 sits in the
// thread's registers, j >= 1 in shared memory, coordinate-major (column i of
// coordinate c at c * cap + i - 1024, so a warp's loads hit 32 banks); the
// running minima stay in registers and go to global memory once, at the end.
// The rows are read where they lie (no packed copy), with the pack's checks
// (NaN/Inf and magnitude for floats; the int32 range, checked after the
// launch).  Each step's exchange slot carries the CTA's candidate with its
// coordinates (one 64-bit word each: a non-zero tag over the value bits):
// warp 0 polls the keys (up to five slots per lane, all loads in flight),
// then reads the winner's coordinates from its slot, still in L2, waiting for
// each tag (every wait bounded by the cycle budget).
constexpr int RES_PPT = 8;   // points per thread (1 in registers + 7 in shared memory)

__host__ __device__ constexpr int res_slot_words(int d) { return 1 + d; }

struct ShRes {
    uint64_t red[32];
    uint32_t cand[32][12];   // each warp's candidate coordinates (value bits)
    uint64_t pkey[1];        // the step's winning key
    uint32_t pc[1][12];      // and its coordinates: the next center
    int abort;
};

template <typename T>
__device__ __forceinline__ uint32_t val_bits(T v) {
    if constexpr (std::is_same<T, float>::value) return __float_as_uint(v);
    else return (uint32_t)v;
}
template <typename T>
__device__ __forceinline__ T bits_val(uint32_t b) {
    if constexpr (std::is_same<T, float>::value) return __uint_as_float(b);
    else return (T)(int32_t)b;
}

template <typename T>
__device__ __forceinline__ void res_check(T v, bool &bad, bool &nonfin, uint32_t &lo, uint32_t &hi) {
    if constexpr (std::is_same<T, float>::value) {
        if (!(fabsf(v) <= 0x1p54f)) bad = true;
        if (!isfinite(v)) nonfin = true;
    } else {
        const uint32_t bv = (uint32_t)v ^ 0x80000000u;
        lo = max(lo, 0xFFFFFFFFu - bv);
        hi = max(hi, bv);
    }
}

template <typename T, int DC>
__global__ void __launch_bounds__(GROUP_NT, 1) gon_resident_kernel(GonArgs a) {
    using A = typename AccOf<T>::type;
    constexpr int NT = GROUP_NT, W = NT / 32, SW = res_slot_words(DC);
    static_assert(DC <= 12, "candidate coordinates are staged in 12 words");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ ShRes sh;
    const GonInst &I = a.single;
    const T *__restrict__ rows = (const T *)I.pk;   // row-major [n][DC]
    const int G = gridDim.x, r = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t lo_r = I.n * r / G, hi_r = I.n * (r + 1) / G;
    const int np = (int)(hi_r - lo_r);
    const int cap = a.res_cap;
    T *sp = reinterpret_cast<T *>(smem_raw);

    // load this CTA's rows, with the pack's checks
    T xr[DC];
    {
        bool bad = false, nonfin = false;
        uint32_t lo = 0, hi = 0;
#pragma unroll
        for (int c = 0; c < DC; ++c) {
            xr[c] = T(0);
            if (tid < np) {
                xr[c] = rows[(lo_r + tid) * DC + c];
                res_check(xr[c], bad, nonfin, lo, hi);
            }
        }
        const int64_t ns = np > NT ? (int64_t)(np - NT) * DC : 0;
        const T *src = rows + (lo_r + NT) * DC;
        for (int64_t e = tid; e < ns; e += NT) {
            const int i = (int)(e / DC), c = (int)(e - (int64_t)i * DC);
            const T v = src[e];
            res_check(v, bad, nonfin, lo, hi);
            sp[c * cap + i] = v;
        }
        if constexpr (std::is_same<T, float>::value) {
            if (nonfin) set_status(a.st, KC_ERR_NONFINITE, 1, 0);
            else if (bad) set_status(a.st, KC_ERR_RANGE, 1, 0);
        } else {
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                lo = max(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
                hi = max(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
            }
            if (lane == 0 && (lo | hi)) {
                atomicMax((uint32_t *)&I.range2[0], lo);
                atomicMax((uint32_t *)&I.range2[1], hi);
            }
        }
    }
    if (tid == 0) {
        sh.abort = 0;
        sh.pkey[0] = make_key(1u, (uint32_t)I.first);
    }
    if (warp == 0 && lane < DC) sh.pc[0][lane] = val_bits(rows[I.first * DC + lane]);
    if (r == 0 && tid == 0) I.centers[0] = out_index(I, I.first);
    __syncthreads();

    uint32_t mm[RES_PPT];
#pragma unroll
    for (int j = 0; j < RES_PPT; ++j) mm[j] = 0xFFFFFFFFu;
    int it;
    uint64_t K = 0;
    for (it = 0; it < I.k; ++it) {
        T cc[DC];
#pragma unroll
        for (int c = 0; c < DC; ++c) cc[c] = bits_val<T>(sh.pc[0][c]);
        uint64_t best = 0;
#pragma unroll
        for (int j = 0; j < RES_PPT; ++j) {
            const int i = tid + j * NT;
            if (i < np) {
                A acc = A(0);
#pragma unroll
                for (int c = 0; c < DC; ++c) acc = sq_step(acc, j == 0 ? xr[c] : sp[c * cap + (i - NT)], cc[c]);
                mm[j] = min(mm[j], acc_bits(acc));
                best = umax64(best, make_key(mm[j], (uint32_t)(lo_r + i)));
            }
        }
        // the warp's candidate and its coordinates
        const uint64_t wb = warp_max_u64(best);
        const unsigned own = __ballot_sync(0xFFFFFFFFu, wb != 0 && best == wb);
        if (own && lane == __ffs(own) - 1) {
            const int i = (int)((int64_t)key_idx(wb) - lo_r);
            if (i < NT || KC_IN_RANGE(a.st, i - NT, cap, KC_AT_RESIDENT_SMEM)) {
#pragma unroll
                for (int c = 0; c < DC; ++c) sh.cand[warp][c] = val_bits(i < NT ? xr[c] : sp[c * cap + (i - NT)]);
            }
        }
        if (lane == 0) sh.red[warp] = wb;
        __syncthreads();
        if (warp == 0) {
            const uint64_t v = lane < W ? sh.red[lane] : 0;
            const uint64_t g = warp_max_u64(v);
            const unsigned ow = __ballot_sync(0xFFFFFFFFu, lane < W && g != 0 && v == g);
            const int wsrc = ow ? __ffs(ow) - 1 : 0;
            if (G > 1) {
                // publish the CTA's candidate: coordinates (tagged) and key
                uint64_t *mine = I.slots + ((int64_t)it * G + r) * SW;
                if (!(a.withhold == it + 1 && r == G - 1)) {
                    if (lane < DC) st_relaxed_u64(mine + 1 + lane, (1ull << 32) | sh.cand[wsrc][lane]);
                    if (lane == 0) st_relaxed_u64(mine, g ? g : 1);
                }
                // poll the keys of the step's slots (lane: slots lane + 32 q)
                const uint64_t *row = I.slots + (int64_t)it * G * SW;
                uint64_t kv[5] = {0, 0, 0, 0, 0};
                unsigned pend = 0;
#pragma unroll
                for (int q = 0; q < 5; ++q)
                    if (lane + 32 * q < G) pend |= 1u << q;
                bool ab = false;
                const long long t0 = clock64();
                while (pend) {
#pragma unroll
                    for (int q = 0; q < 5; ++q)
                        if (pend >> q & 1u) kv[q] = ld_relaxed_u64(row + (int64_t)(lane + 32 * q) * SW);
#pragma unroll
                    for (int q = 0; q < 5; ++q)
                        if ((pend >> q & 1u) && kv[q] != 0) pend &= ~(1u << q);
                    if (pend && (clock64() - t0 > a.timeout_cycles || ld_volatile_i32(&a.st->code) != 0)) {
                        set_status(a.st, KC_ERR_TIMEOUT, 3, it);
                        ab = true;
                        break;
                    }
                }
                ab = __any_sync(0xFFFFFFFFu, ab);
                uint64_t lk = 0;
                int ls = 0;
#pragma unroll
                for (int q = 0; q < 5; ++q)
                    if (kv[q] > lk) {
                        lk = kv[q];
                        ls = lane + 32 * q;
                    }
                const uint64_t gg = warp_max_u64(lk);
                const unsigned wl = __ballot_sync(0xFFFFFFFFu, gg != 0 && lk == gg);
                const int win = __shfl_sync(0xFFFFFFFFu, ls, wl ? __ffs(wl) - 1 : 0);
                // the winner's coordinates from its slot (each tag set once written)
                if (!ab && !KC_IN_RANGE(a.st, win, G, KC_AT_SLOT)) ab = true;
                if (!ab && lane < DC) {
                    const uint64_t *wp = row + (int64_t)win * SW + 1 + lane;
                    uint64_t w = ld_relaxed_u64(wp);
                    while ((w >> 32) == 0) {
                        if (clock64() - t0 > a.timeout_cycles || ld_volatile_i32(&a.st->code) != 0) {
                            set_status(a.st, KC_ERR_TIMEOUT, 3, it);
                            ab = true;
                            break;
                        }
                        w = ld_relaxed_u64(wp);
                    }
                    sh.pc[0][lane] = (uint32_t)w;
                }
                ab = __any_sync(0xFFFFFFFFu, ab);
                if (lane == 0) {
                    sh.pkey[0] = gg;
                    if (ab) sh.abort = 1;
                }
            } else {
                if (lane == 0) sh.pkey[0] = g;
                if (lane < DC) sh.pc[0][lane] = sh.cand[wsrc][lane];
            }
        }
        __syncthreads();
        if (sh.abort) return;
        const uint64_t g = sh.pkey[0];
        K = g;
        if (key_val(K) == 0) {   // every point is at distance 0: stop early
            ++it;
            break;
        }
        if (r == 0 && tid == 0 && it + 1 < I.k && KC_IN_RANGE(a.st, key_idx(g), I.n, KC_AT_CENTER_LOAD))
            I.centers[it + 1] = out_index(I, key_idx(g));
    }
    // the running minima, for the radius recheck
#pragma unroll
    for (int j = 0; j < RES_PPT; ++j) {
        const int i = tid + j * NT;
        if (i < np) I.mind[lo_r + i] = mm[j];
    }
    if (r == 0 && tid == 0) {
        *I.k_out = it;
        *I.final_key = K;
    }
}

template <typename T, int DC> void *resident_fn() { return (void *)gon_resident_kernel<T, DC>; }

// Specialisations d = 8 and 10 (float), 10 (int32).  Below d = 8 the
// streaming kernel's sweep from L2 is already short, and measured as fast or
// faster (d = 2: 1M points 0.42 against 0.44 ms, 100k 0.28 against 0.32 ms
// at k = 100); from d = 8 on the resident kernel wins (d = 10: 1M points 0.44
// against 0.72 ms, 200k 0.36 against 0.47 ms; d = 8, 500k: 0.38 against 0.53).
void *pick_resident(int dtype, int d) {
    if (dtype == KC_F32) {
        switch (d) {
            case 8: return resident_fn<float, 8>();
            case 10: return resident_fn<float, 10>();
            default: return nullptr;
        }
    }
    return d == 10 ? resident_fn<int32_t, 10>() : nullptr;
}

template <typename T, int DC, bool DYN = false> void *group_fn() { return (void *)gon_group_kernel<T, DC, DYN>; }
template <typename T, int DC> void *queue_fn() { return (void *)gon_queue_kernel<T, DC>; }
template <int KIND, int DC> void *group_lp_fn() { return (void *)gon_group_lp_kernel<KIND, DC>; }
template <int KIND, int DC> void *queue_lp_fn() { return (void *)gon_queue_lp_kernel<KIND, DC>; }

void *pick_group_lp(int kind, int dc) {
    if (kind == KC_SWEEP_FP8) {
        switch (dc) {
            case 16: return group_lp_fn<KC_SWEEP_FP8, 16>();
            default: return group_lp_fn<KC_SWEEP_FP8, 0>();
        }
    }
    if (kind == KC_SWEEP_FP16) {
        switch (dc) {
            case 10: return group_lp_fn<KC_SWEEP_FP16, 10>();
            case 16: return group_lp_fn<KC_SWEEP_FP16, 16>();
            case 64: return group_lp_fn<KC_SWEEP_FP16, 64>();
            default: return group_lp_fn<KC_SWEEP_FP16, 0>();
        }
    }
    switch (dc) {
        case 10: return group_lp_fn<KC_SWEEP_BF16, 10>();
        case 16: return group_lp_fn<KC_SWEEP_BF16, 16>();
        case 64: return group_lp_fn<KC_SWEEP_BF16, 64>();
        default: return group_lp_fn<KC_SWEEP_BF16, 0>();
    }
}

void *pick_queue_lp(int kind, int dc) {
    if (kind == KC_SWEEP_FP8) return queue_lp_fn<KC_SWEEP_FP8, 0>();
    if (kind == KC_SWEEP_FP16) return queue_lp_fn<KC_SWEEP_FP16, 0>();
    switch (dc) {
        case 3: return queue_lp_fn<KC_SWEEP_BF16, 3>();
        case 8: return queue_lp_fn<KC_SWEEP_BF16, 8>();
        case 32: return queue_lp_fn<KC_SWEEP_BF16, 32>();
        default: return queue_lp_fn<KC_SWEEP_BF16, 0>();
    }
}

size_t lp_smem_bytes(int kind, int dmax, int nt) {
    const int dp = lp_ngroups(kind, dmax) * lp_group(kind);
    return (size_t)2 * ((dp + 1) & ~1) * sizeof(float) + (size_t)(nt / 32) * LP_CAP * sizeof(Cand);
}

void *pick_group(int dtype, int dc, bool dyn = false) {
    if (dtype == KC_F32 && dyn) {
        switch (dc) {
            case 2: return group_fn<float, 2, true>();
            case 3: return group_fn<float, 3, true>();
            case 8: return group_fn<float, 8, true>();
            case 10: return group_fn<float, 10, true>();
            case 16: return group_fn<float, 16, true>();
            case 32: return group_fn<float, 32, true>();
            case 64: return group_fn<float, 64, true>();
            default: return group_fn<float, 0, true>();
        }
    }
    if (dtype == KC_F32) {
        switch (dc) {
            case 2: return group_fn<float, 2>();
            case 3: return group_fn<float, 3>();
            case 8: return group_fn<float, 8>();
            case 10: return group_fn<float, 10>();
            case 16: return group_fn<float, 16>();
            case 32: return group_fn<float, 32>();
            case 64: return group_fn<float, 64>();
            default: return group_fn<float, 0>();
        }
    }
    switch (dc) {
        case 2: return group_fn<int32_t, 2>();
        case 10: return group_fn<int32_t, 10>();
        default: return group_fn<int32_t, 0>();
    }
}

void *pick_queue(int dtype, int dc) {
    if (dtype == KC_F32) {
        switch (dc) {
            case 3: return queue_fn<float, 3>();
            case 8: return queue_fn<float, 8>();
            case 16: return queue_fn<float, 16>();
            case 32: return queue_fn<float, 32>();
            default: return queue_fn<float, 0>();
        }
    }
    return queue_fn<int32_t, 0>();
}

}  // namespace

cudaError_t read_counters(unsigned long long out[8], bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_counters, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess && reset) {
        const unsigned long long z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        e = cudaMemcpyToSymbol(g_counters, z, sizeof z);
    }
    return e;
}

int gon_threads() { return GROUP_NT; }
int gon_queue_warps() { return QUEUE_NT / 32; }
int gon_warps_per_cta() { return GROUP_NT / 32; }

static void *pick_fn(int dtype, int lp, int dc, bool queue, bool dyn = false) {
    if (dtype == KC_F32 && lp) return queue ? pick_queue_lp(lp, dc) : pick_group_lp(lp, dc);
    return queue ? pick_queue(dtype, dc) : pick_group(dtype, dc, dyn);
}

static size_t smem_for(int dtype, int lp, int dmax, bool queue) {
    if (dtype == KC_F32 && lp) return lp_smem_bytes(lp, dmax, queue ? QUEUE_NT : GROUP_NT);
    return (size_t)(dmax > 0 ? dmax : 1) * 4;
}

// Occupancy of a GON kernel with its dynamic shared memory (opted in first
// when above the default 48 KB).
static int gon_occupancy(void *fn, int nt, size_t smem) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, nt, smem) != cudaSuccess) {
        cudaGetLastError();
        occ = 0;
    }
    return occ;
}

int gon_max_grid(int dtype, int d, int lp) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return gon_occupancy(pick_fn(dtype, lp, d, false), GROUP_NT, smem_for(dtype, lp, d, false)) * sms;
}

int gon_queue_grid(int dtype, int d, int lp) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return gon_occupancy(pick_fn(dtype, lp, d, true), QUEUE_NT, smem_for(dtype, lp, d, true)) * sms;
}

int gon_resident_plan(int dtype, int d, int64_t n, int *cap, int *slot_words) {
    if (const char *env = getenv("KC_GON_RESIDENT"))
        if (atoi(env) == 0) return 0;
    void *fn = pick_resident(dtype, d);
    if (!fn || n < 1) return 0;
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // One CTA per 4096 points (four per thread; measured best of 1024, 4096
    // and 8192 on sets of 10k to 1M points in d = 2..10), at most one per SM,
    // and at least as many as the shares need to fit (at most RES_PPT points
    // per thread, the rest of a share within the shared memory one CTA may
    // take).  KC_GON_RESIDENT_PTS sets the points per CTA.
    const int64_t cap_pts = (int64_t)((size_t)optin - sizeof(ShRes) - 1024) / (4 * d) + GROUP_NT;
    const int64_t per = std::min<int64_t>((int64_t)RES_PPT * GROUP_NT, cap_pts);
    int64_t target = 4096;
    if (const char *env = getenv("KC_GON_RESIDENT_PTS")) target = std::max<int64_t>(atoll(env), 1);
    const int64_t gmin = (n + per - 1) / per;
    if (gmin > sms || gmin > 160) return 0;   // warp 0 polls at most five slots per lane
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(gmin, (n + target - 1) / target),
                                                             std::min(sms, 160)));
    const int64_t npmax = (n + G - 1) / G;
    if (npmax > per) return 0;
    const int64_t c = npmax > GROUP_NT ? npmax - GROUP_NT : 1;
    const size_t smem = (size_t)c * d * 4;
    if (smem + sizeof(ShRes) + 1024 > (size_t)optin) return 0;
    if (smem > 48 * 1024 && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, GROUP_NT, smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return 0;
    }
    *cap = (int)c;
    *slot_words = res_slot_words(d);
    return G;
}

cudaError_t launch_gon(GonArgs &a, cudaStream_t s) {
    if (a.res_cap > 0) {
        // resident single instance: one CTA per SM, all co-resident
        void *fn = pick_resident(a.dtype, a.dc);
        if (!fn) return cudaErrorInvalidValue;
        const size_t smem = (size_t)a.res_cap * a.dc * 4;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        note_launches(1);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(a.grid);
        cfg.blockDim = dim3(GROUP_NT);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        void *args[] = {&a};
        return cudaLaunchKernelExC(&cfg, fn, args);
    }
    const size_t smem = smem_for(a.dtype, a.lp_kind, a.dmax, a.queue != 0);
    void *fn = pick_fn(a.dtype, a.lp_kind, a.dc, a.queue != 0, a.dyn != 0);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    note_launches(1);
    // Groups that wait on one another need a cooperative launch (all CTAs
    // co-resident); the attribute form is also accepted by stream capture.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.grid);
    cfg.blockDim = dim3(a.queue ? QUEUE_NT : GROUP_NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = (!a.queue || a.gheavy > 0) ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {&a};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace kc
