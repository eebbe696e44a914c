// kc_radius.cu -- covering radius of a center set (the solution value of
// Section 7): max over points of the distance to the nearest center.
//
//   gather      center coordinates -> scratch [kc][d] (indices validated)
//   min         canonical FP32 (or exact int32) minimum over centers per
//               point, plus the (value, lowest index) maximum key
//   recheck     float only: every point whose FP32 minimum can still reach
//               the FP64 maximum (within the FP32 error bound) gets its FP64
//               minimum over all centers; the largest FP64 value wins, then
//               the lowest index holding it
//   finalize    radius = sqrt(value), argmax index
// The FP32 bound: a canonical FP32 squared distance is within a factor
// (1 +- gamma), gamma = (d+2) 2^-24 / (1 - (d+2) 2^-24), of the exact one, and
// the FP64 value within (1 +- ~d 2^-53).  So the FP64 maximiser x* satisfies
// m32(x*) >= M32 (1 - gamma)(1 - g64) / ((1 + gamma)(1 + g64)) > M32 (1 - 3 gamma):
// flagging m32 >= M32 (1 - 3 gamma) can never miss it.
#include <type_traits>

#include "kc_internal.cuh"

namespace kc {

namespace {

constexpr int RAD_NT = 256;
constexpr int RAD_W = RAD_NT / 32;
constexpr int RAD_TILE_BYTES = 32 * 1024;

// Center rows from the packed array, or (float, pk null) the row-major one.
template <typename T>
__global__ void gather_kernel(const T *__restrict__ pk, const T *__restrict__ rm, int64_t n, int d,
                              const int64_t *__restrict__ centers, const int32_t *kc_dev, int kc_max,
                              T *__restrict__ cen, DevStatus *st) {
    if (ld_volatile_i32(&st->code) != 0) return;
    const int kc = (int)dev_count(kc_dev, kc_max);
    const int64_t total = (int64_t)kc * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / d), j = (int)(e - (int64_t)i * d);
        const int64_t c = centers[i];
        if (c < 0 || c >= n) {
            set_status(st, KC_ERR_ARG, 4, i);
            cen[e] = T(0);
            continue;
        }
        cen[e] = pk ? pk[pk_index(c, j, d)] : rm[c * d + j];
    }
}

// Minimum over all centers for the 4 points of each lane.  Centers are staged
// through shared memory in tiles with a row stride of DR >= d coordinates,
// zero-padded (a zero term leaves the canonical sum unchanged), and the
// lane's points are held in registers when d <= DR.  The points come from the
// packed array pk, or (pk null, float) straight from the row-major array rm:
// a lane's 4 points are 4d consecutive floats, 16-byte aligned when rm is,
// and every coordinate is checked as the pack would check it (NaN/Inf, then
// magnitude above 2^54), so no packed copy is made.
template <typename T, int DR>
__global__ void __launch_bounds__(RAD_NT) radius_min_kernel(
    const T *__restrict__ pk, const T *__restrict__ rm, int64_t n, int d, const T *__restrict__ cen,
    const int32_t *kc_dev, int kc_max, uint32_t *__restrict__ mind, unsigned long long *key32, DevStatus *st) {
    using A = typename AccOf<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *cs = reinterpret_cast<T *>(smem_raw);
    if (ld_volatile_i32(&st->code) != 0) return;
    const int kc = (int)dev_count(kc_dev, kc_max);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t nb = nblocks(n);
    const int tile = RAD_TILE_BYTES / (DR * (int)sizeof(T));
    uint64_t best = 0;
    for (int64_t g = blockIdx.x; g * RAD_W < nb; g += gridDim.x) {
        const int64_t b = g * RAD_W + warp;
        const bool active = b < nb;
        T x[DR][4];
        if (pk || !std::is_same<T, float>::value) {
#pragma unroll
            for (int j = 0; j < DR; ++j) {
                x[j][0] = x[j][1] = x[j][2] = x[j][3] = T(0);
                if (active && j < d) {
                    const T *p = pk + (b * d + j) * BLK + lane * 4;
                    x[j][0] = p[0];
                    x[j][1] = p[1];
                    x[j][2] = p[2];
                    x[j][3] = p[3];
                }
            }
        } else if constexpr (std::is_same<T, float>::value) {
            const int64_t i0 = b * BLK + lane * 4;
            bool bad = false, nonfin = false;
            if (active && d == DR && i0 + 3 < n && ((uintptr_t)rm & 15) == 0) {
                // 4 rows of DR floats: DR 16-byte loads
                T v[4 * DR];
#pragma unroll
                for (int t = 0; t < DR; ++t) {
                    const float4 w = __ldg(reinterpret_cast<const float4 *>(rm + i0 * DR) + t);
                    v[4 * t] = w.x;
                    v[4 * t + 1] = w.y;
                    v[4 * t + 2] = w.z;
                    v[4 * t + 3] = w.w;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int j = 0; j < DR; ++j) x[j][q] = v[q * DR + j];
            } else {
#pragma unroll
                for (int j = 0; j < DR; ++j)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        x[j][q] = (active && j < d && i0 + q < n) ? __ldg(rm + (i0 + q) * d + j) : T(0);
            }
#pragma unroll
            for (int j = 0; j < DR; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float av = fabsf((float)x[j][q]);
                    if (!(av <= 0x1p54f)) bad = true;   // NaN fails the comparison
                    if (!isfinite((float)x[j][q])) nonfin = true;
                }
            if (nonfin) set_status(st, KC_ERR_NONFINITE, 1, 0);
            else if (bad) set_status(st, KC_ERR_RANGE, 1, 0);
        }
        uint32_t m[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
        for (int t0 = 0; t0 < kc; t0 += tile) {
            const int tc = (kc - t0) < tile ? (kc - t0) : tile;
            __syncthreads();
            for (int e = tid; e < tc * DR; e += RAD_NT) {
                const int ci = e / DR, j = e - ci * DR;
                cs[e] = j < d ? cen[(int64_t)(t0 + ci) * d + j] : T(0);
            }
            __syncthreads();
            if (active) {
                for (int ci = 0; ci < tc; ++ci) {
                    const T *cc = cs + ci * DR;
                    A a0 = A(0), a1 = A(0), a2 = A(0), a3 = A(0);
#pragma unroll
                    for (int j = 0; j < DR; ++j) {
                        const T c = cc[j];
                        a0 = sq_step(a0, x[j][0], c);
                        a1 = sq_step(a1, x[j][1], c);
                        a2 = sq_step(a2, x[j][2], c);
                        a3 = sq_step(a3, x[j][3], c);
                    }
                    m[0] = min(m[0], acc_bits(a0));
                    m[1] = min(m[1], acc_bits(a1));
                    m[2] = min(m[2], acc_bits(a2));
                    m[3] = min(m[3], acc_bits(a3));
                }
            }
        }
        if (active) {
            reinterpret_cast<uint4 *>(mind + b * BLK)[lane] = make_uint4(m[0], m[1], m[2], m[3]);
            const int64_t i0 = b * BLK + lane * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (i0 + q < n) best = umax64(best, make_key(m[q], (uint32_t)(i0 + q)));
        }
    }
    best = warp_max_u64(best);
    if (lane == 0 && best) atomicMax(key32, (unsigned long long)best);
}

// Generic version for d > 16: one point per thread, coordinates re-read from
// the packed layout for every center (cache-resident).
template <typename T>
__global__ void __launch_bounds__(RAD_NT) radius_min_generic_kernel(
    const T *__restrict__ pk, int64_t n, int d, const T *__restrict__ cen, const int32_t *kc_dev,
    int kc_max, uint32_t *__restrict__ mind, unsigned long long *key32, const DevStatus *st) {
    using A = typename AccOf<T>::type;
    if (ld_volatile_i32(&st->code) != 0) return;
    const int kc = (int)dev_count(kc_dev, kc_max);
    uint64_t best = 0;
    for (int64_t x = blockIdx.x * (int64_t)RAD_NT + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * RAD_NT) {
        uint32_t m = 0xFFFFFFFFu;
        for (int ci = 0; ci < kc; ++ci) {
            A a = A(0);
            for (int j = 0; j < d; ++j) a = sq_step(a, pk[pk_index(x, j, d)], cen[(int64_t)ci * d + j]);
            m = min(m, acc_bits(a));
        }
        mind[x] = m;
        best = umax64(best, make_key(m, (uint32_t)x));
    }
    best = warp_max_u64(best);
    if ((threadIdx.x & 31) == 0 && best) atomicMax(key32, (unsigned long long)best);
}

__device__ __forceinline__ double flag_threshold(const unsigned long long *key32, int d) {
    const float M32 = __uint_as_float(key_val(*key32));
    return (double)M32 * (1.0 - 3.0 * f32_gamma(d));
}

// Can point x reach the FP64 maximum?  FP32 minima: m32(x) >= thr.  After a
// mixed-precision sweep mind holds approximate minima m~; then U(x)^2 >= thr
// with U(x) >= sqrt of the exact minimum (kc_gon.cu), which also bounds the
// FP64 value within the same (1 - 3 gamma) margin.
__device__ __forceinline__ bool can_reach(const uint32_t *mind, int64_t x, double thr, const float *eblk,
                                          const float *ecmax, float opg, double sc) {
    if (!eblk) return (double)__uint_as_float(mind[x]) >= thr;
    // mixed precision: 16-bit truncated codes, upper end of the code's
    // interval; sc: the fp16 sweep's power-of-two unit (exact in double)
    const uint32_t hi = ((uint32_t)reinterpret_cast<const uint16_t *>(mind)[x] + 1u) << 16;
    const double U = (double)lp_upper(hi, __fadd_ru(eblk[x / BLK], *ecmax), opg) * sc;
    return U * U >= thr;
}

// FP64 minimum over all centers of point x, computed by the whole warp (lane
// l takes centers l, l+32, ...).  FP64 is slow on this part, so a canonical
// FP32 pass goes first: with g the FP32 bound (d+2)u/(1-(d+2)u) and m32 the
// FP32 minimum, a center whose FP32 value exceeds m32 (1+g)/(1-g) (1+eps64)
// has an exact distance above the FP32 argmin's by more than FP64's own
// rounding (eps64 = 4 (d+2) 2^-53), so its FP64 value cannot be the minimum;
// only the remaining centers (usually one or two) are evaluated in FP64,
// each sum in coordinate order.  m32: the canonical FP32 minimum when the
// caller holds it (0xFFFFFFFF: computed here first).
__device__ double min64_warp(const float *__restrict__ pk, const float *__restrict__ rm, int64_t x, int d,
                             const float *__restrict__ cen, int kc, int lane, uint32_t m32) {
    const bool v4 = (d & 3) == 0 && ((uintptr_t)cen & 15) == 0 && (pk || ((uintptr_t)rm & 15) == 0);
    if (m32 == 0xFFFFFFFFu) {
        for (int ci = lane; ci < kc; ci += 32)
            m32 = min(m32, __float_as_uint(point_row_dist(pk, rm, x, d, cen + (int64_t)ci * d, v4)));
#pragma unroll
        for (int o = 16; o; o >>= 1) m32 = min(m32, __shfl_xor_sync(0xFFFFFFFFu, m32, o));
    }
    const double g = f32_gamma(d);
    const double lim = (double)__uint_as_float(m32) * ((1.0 + g) / (1.0 - g)) * (1.0 + 4.0 * (d + 2) * 0x1p-53);
    double m = INFINITY;
    for (int ci = lane; ci < kc; ci += 32) {
        const float s = point_row_dist(pk, rm, x, d, cen + (int64_t)ci * d, v4);
        if ((double)s > lim) continue;
        double s64 = 0.0;
        for (int j = 0; j < d; ++j) s64 = sq_step64(s64, point_at(pk, rm, x, j, d), cen[(int64_t)ci * d + j]);
        m = fmin(m, s64);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmin(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    return m;
}

// Each warp scans 32 points at a time; the flagged ones (ballot) are
// recomputed one after another by the whole warp.  list (optional, with its
// device count): only the listed points can be flagged (every other point's
// minimum is 0), so only they are scanned.
__global__ void recheck_max_kernel(const float *__restrict__ pk, const float *__restrict__ rm, int64_t n, int d,
                                   const float *__restrict__ cen, const int32_t *kc_dev, int kc_max,
                                   const uint32_t *__restrict__ mind, const unsigned long long *key32,
                                   unsigned long long *max64, double *m64, const DevStatus *st,
                                   const float *eblk, const float *ecmax, const float *lpscale,
                                   const uint32_t *__restrict__ list, const unsigned long long *lcount) {
    if (ld_volatile_i32(&st->code) != 0) return;
    if (key_val(*key32) == 0) return;   // every minimum is exactly 0
    const double sc = lpscale ? (double)*lpscale : 1.0;
    const int kc = (int)dev_count(kc_dev, kc_max);
    const double thr = flag_threshold(key32, d);
    const float opg = __fadd_ru(1.f, lp_slack(d));
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t cnt = list ? (int64_t)*lcount : n;
    for (int64_t base = (blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < cnt;
         base += warps * 32) {
        const int64_t i = base + lane;
        int64_t x = i < cnt ? (list ? (int64_t)list[i] : i) : 0;
        if (i < cnt && !KC_IN_RANGE((DevStatus *)st, x, n, KC_AT_RADIUS_LIST)) x = -1;
        const bool flag = i < cnt && x >= 0 && can_reach(mind, x, thr, eblk, ecmax, opg, sc);
        unsigned todo = __ballot_sync(0xFFFFFFFFu, flag);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t xs = __shfl_sync(0xFFFFFFFFu, x, src);
            // FP32 minima: mind holds the canonical one; mixed precision: not
            const double v = min64_warp(pk, rm, xs, d, cen, kc, lane, eblk ? 0xFFFFFFFFu : mind[xs]);
            if (lane == src) {
                m64[xs] = v;
                atomicMax(max64, (unsigned long long)__double_as_longlong(v));
            }
        }
    }
}

__global__ void recheck_arg_kernel(int64_t n, int d, const uint32_t *__restrict__ mind,
                                   const unsigned long long *key32, const unsigned long long *max64,
                                   const double *__restrict__ m64, unsigned long long *arg64,
                                   const DevStatus *st, const float *eblk, const float *ecmax,
                                   const float *lpscale, const uint32_t *__restrict__ list,
                                   const unsigned long long *lcount) {
    if (ld_volatile_i32(&st->code) != 0) return;
    if (key_val(*key32) == 0) return;
    const double sc = lpscale ? (double)*lpscale : 1.0;
    const double thr = flag_threshold(key32, d);
    const float opg = __fadd_ru(1.f, lp_slack(d));
    const double M = __longlong_as_double((long long)*max64);
    const int64_t cnt = list ? (int64_t)*lcount : n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = list ? (int64_t)list[i] : i;
        if (can_reach(mind, x, thr, eblk, ecmax, opg, sc) && m64[x] == M)
            atomicMax(arg64, 0xFFFFFFFFFFFFFFFFull - (unsigned long long)x);
    }
}

// Float points, one launch for the FP64 recheck and the result: every CTA
// scans its share of the points (the list, or all n) as recheck_max_kernel
// does and also appends each flagged point to a list; the last CTA to finish
// (a completion counter, after a fence) takes the lowest flagged index whose
// FP64 value equals the maximum and writes radius and argmax, as
// recheck_arg_kernel and finalize_kernel do.  Only this call's flagged points
// are visited, so m64 entries left by earlier calls are never read.
__global__ void __launch_bounds__(256) recheck_kernel(
    const float *__restrict__ pk, const float *__restrict__ rm, int64_t n, int d, const float *__restrict__ cen,
    const int32_t *kc_dev, int kc_max, const uint32_t *__restrict__ mind, const unsigned long long *key32,
    unsigned long long *max64, double *m64, DevStatus *st, const float *eblk, const float *ecmax,
    const float *lpscale, const uint32_t *__restrict__ list, const unsigned long long *lcount, uint32_t *flagged,
    unsigned *flagged_n, unsigned *done, double *radius_out, int64_t *argmax_out) {
    __shared__ int s_last;
    __shared__ unsigned long long s_arg[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool run = ld_volatile_i32(&st->code) == 0 && key_val(*key32) != 0;
    if (run) {
        const double sc = lpscale ? (double)*lpscale : 1.0;
        const int kc = (int)dev_count(kc_dev, kc_max);
        const double thr = flag_threshold(key32, d);
        const float opg = __fadd_ru(1.f, lp_slack(d));
        const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
        const int64_t cnt = list ? (int64_t)*lcount : n;
        for (int64_t base = (blockIdx.x * (int64_t)(blockDim.x >> 5) + warp) * 32; base < cnt; base += warps * 32) {
            const int64_t i = base + lane;
            int64_t x = i < cnt ? (list ? (int64_t)list[i] : i) : 0;
            if (i < cnt && !KC_IN_RANGE(st, x, n, KC_AT_RADIUS_LIST)) x = -1;
            const bool flag = i < cnt && x >= 0 && can_reach(mind, x, thr, eblk, ecmax, opg, sc);
            unsigned todo = __ballot_sync(0xFFFFFFFFu, flag);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const int64_t xs = __shfl_sync(0xFFFFFFFFu, x, src);
                const double v = min64_warp(pk, rm, xs, d, cen, kc, lane, eblk ? 0xFFFFFFFFu : mind[xs]);
                if (lane == src) {
                    m64[xs] = v;
                    atomicMax(max64, (unsigned long long)__double_as_longlong(v));
                    const unsigned slot = atomicAdd(flagged_n, 1u);
                    if (KC_IN_RANGE(st, slot, n, KC_AT_RADIUS_LIST)) flagged[slot] = (uint32_t)xs;
                }
            }
        }
    }
    // the last CTA to finish sees every other CTA's writes (fence, counter)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (ld_volatile_i32(&st->code) != 0) return;
    const uint64_t K = __ldcg(key32);
    if (key_val(K) == 0) {
        // every minimum is exactly 0
        if (threadIdx.x == 0) {
            *radius_out = 0.0;
            if (argmax_out) *argmax_out = key_idx(K);
        }
        return;
    }
    const unsigned long long mb = __ldcg(max64);
    const unsigned nf = __ldcg(flagged_n);
    unsigned long long best = 0;
    for (unsigned f = threadIdx.x; f < nf && f < (unsigned)n; f += blockDim.x) {
        const uint32_t x = __ldcg(flagged + f);
        if ((unsigned long long)__double_as_longlong(__ldcg(m64 + x)) == mb)
            best = umax64(best, 0xFFFFFFFFFFFFFFFFull - (unsigned long long)x);
    }
    best = warp_max_u64(best);
    if (lane == 0) s_arg[warp] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = umax64(best, s_arg[w]);
        *radius_out = __dsqrt_rn(__longlong_as_double((long long)mb));
        if (argmax_out) *argmax_out = (int64_t)(0xFFFFFFFFFFFFFFFFull - best);
    }
}

// One thread: radius and argmax from the FP64 recheck (float) or directly
// from the exact key (int32).
__global__ void finalize_kernel(int dtype, const unsigned long long *key32,
                                const unsigned long long *max64, const unsigned long long *arg64,
                                double *radius_out, int64_t *argmax_out, const DevStatus *st) {
    if (ld_volatile_i32(&st->code) != 0) return;
    const uint64_t K = *key32;
    double r2;
    int64_t am;
    if (dtype == KC_I32 || key_val(K) == 0) {
        r2 = dtype == KC_I32 ? (double)key_val(K) : 0.0;
        am = key_idx(K);
    } else {
        r2 = __longlong_as_double((long long)*max64);
        am = (int64_t)(0xFFFFFFFFFFFFFFFFull - *arg64);
    }
    *radius_out = __dsqrt_rn(r2);
    if (argmax_out) *argmax_out = am;
}

template <typename T, int DR>
cudaError_t run_min(RadiusArgs &a, cudaStream_t s, int grid) {
    const int tile = RAD_TILE_BYTES / (DR * (int)sizeof(T));
    const size_t smem = (size_t)tile * DR * sizeof(T);
    radius_min_kernel<T, DR><<<grid, RAD_NT, smem, s>>>(
        (const T *)a.pk, (const T *)a.rm, a.n, a.d, (const T *)a.cen, a.kc_dev, a.kc_max, a.mind, a.key32, a.st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_min(RadiusArgs &a, cudaStream_t s, int sms) {
    const int64_t groups = (nblocks(a.n) + RAD_W - 1) / RAD_W;
    const int64_t cap = (int64_t)sms * 8;
    const int grid = (int)(groups < cap ? groups : cap);
    // the row stride DR is the smallest specialisation >= d: padded
    // coordinates cost a subtract and a multiply-add each for every center
    if (a.d <= 2) return run_min<T, 2>(a, s, grid);
    if (a.d <= 3) return run_min<T, 3>(a, s, grid);
    if (a.d <= 4) return run_min<T, 4>(a, s, grid);
    if (a.d <= 8) return run_min<T, 8>(a, s, grid);
    if (a.d <= 10) return run_min<T, 10>(a, s, grid);
    if (a.d <= 16) return run_min<T, 16>(a, s, grid);
    const int64_t g2 = (a.n + RAD_NT - 1) / RAD_NT;
    const int grid2 = (int)(g2 < cap ? g2 : cap);
    radius_min_generic_kernel<T><<<grid2, RAD_NT, 0, s>>>((const T *)a.pk, a.n, a.d,
                                                          (const T *)a.cen, a.kc_dev, a.kc_max,
                                                          a.mind, a.key32, a.st);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_radius(RadiusArgs &a, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e;
    {
        const int64_t total = (int64_t)a.kc_max * a.d;
        const int64_t g = (total + 255) / 256;
        const int grid = (int)(g < 1 ? 1 : (g > sms * 4 ? sms * 4 : g));
        if (a.dtype == KC_F32)
            gather_kernel<float><<<grid, 256, 0, s>>>((const float *)a.pk, a.rm, a.n, a.d, a.centers,
                                                      a.kc_dev, a.kc_max, (float *)a.cen, a.st);
        else
            gather_kernel<int32_t><<<grid, 256, 0, s>>>((const int32_t *)a.pk, (const int32_t *)a.rm, a.n, a.d,
                                                        a.centers, a.kc_dev, a.kc_max, (int32_t *)a.cen, a.st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // row-major points (pk null) are read by the tensor-core path, by the
    // CUDA-core minimum for float points with d <= 16, and by the rechecks
    // after a Gonzalez kernel that held the minima (have_mind)
    if (a.rm && (a.pk || (!a.have_mind && (a.dtype != KC_F32 || (!(a.tc_at && tc_supported(a.d)) && a.d > 16)))))
        return cudaErrorInvalidValue;
    if (!a.rm && !a.pk) return cudaErrorInvalidValue;
    if (!a.have_mind) {
        if (a.dtype == KC_F32 && a.tc_at && tc_supported(a.d)) {
            // tensor-core filter: fp16 dot products bound every point's
            // canonical minimum; only points that can reach the maximum get
            // their exact canonical FP32 minimum (the rest get 0)
            e = launch_tc_radius((const float *)a.pk, a.rm, a.n, a.d, (const float *)a.cen, a.kc_dev, a.kc_max,
                                 tc_bufs(a), a.mind, a.key32, a.st, s);
        } else {
            e = a.dtype == KC_F32 ? dispatch_min<float>(a, s, sms) : dispatch_min<int32_t>(a, s, sms);
        }
        if (e != cudaSuccess) return e;
    }
    if (a.dtype == KC_F32 && a.flagged) {
        const bool tcl = !a.have_mind && a.tc_at && tc_supported(a.d);
        const int64_t g = (a.n + 255) / 256;
        const int grid = (int)(g > sms * 8 ? sms * 8 : g);
        recheck_kernel<<<grid, 256, 0, s>>>((const float *)a.pk, a.rm, a.n, a.d, (const float *)a.cen, a.kc_dev,
                                            a.kc_max, a.mind, a.key32, a.max64, a.m64, a.st, a.eblk, a.ecmax,
                                            a.lpscale, tcl ? a.tc_flist : nullptr, tcl ? a.tc_fcount : nullptr,
                                            a.flagged, a.flagged_n, a.done, a.radius_out, a.argmax_out);
        const bool tc = tcl;
        note_launches(2 + (a.have_mind || tc ? 0 : 1));
        return cudaGetLastError();
    }
    if (a.dtype == KC_F32) {
        // after the tensor-core filter only its listed points have a non-zero minimum
        const bool tcl = !a.have_mind && a.tc_at && tc_supported(a.d);
        const uint32_t *list = tcl ? a.tc_flist : nullptr;
        const unsigned long long *lcount = tcl ? a.tc_fcount : nullptr;
        const int64_t g = (a.n + 255) / 256;
        const int grid = (int)(g > sms * 8 ? sms * 8 : g);
        recheck_max_kernel<<<grid, 256, 0, s>>>((const float *)a.pk, a.rm, a.n, a.d, (const float *)a.cen,
                                                a.kc_dev, a.kc_max, a.mind, a.key32, a.max64, a.m64,
                                                a.st, a.eblk, a.ecmax, a.lpscale, list, lcount);
        recheck_arg_kernel<<<grid, 256, 0, s>>>(a.n, a.d, a.mind, a.key32, a.max64, a.m64, a.arg64,
                                                a.st, a.eblk, a.ecmax, a.lpscale, list, lcount);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    finalize_kernel<<<1, 1, 0, s>>>(a.dtype, a.key32, a.max64, a.arg64, a.radius_out, a.argmax_out,
                                    a.st);
    const bool tc = a.dtype == KC_F32 && a.tc_at && tc_supported(a.d);
    note_launches(2 + (a.have_mind || tc ? 0 : 1) + (a.dtype == KC_F32 ? 2 : 0));
    return cudaGetLastError();
}

}  // namespace kc
