// kc_pack.cu -- repack row-major points into the blocked coordinate-major
// layout every sweep kernel reads (one pass, before the k sweeps).
#include <type_traits>

#include "kc_internal.cuh"

namespace kc {

namespace {

constexpr int PACK_NT = 256;   // threads per CTA
constexpr int PACK_DC = 64;    // coordinates staged per pass through shared memory

__device__ __forceinline__ uint32_t bias_i32(int32_t v) { return (uint32_t)v ^ 0x80000000u; }

// Checks of one source value: floats for NaN/Inf and magnitude, int32 into
// the running biased range.
template <typename T>
__device__ __forceinline__ void pack_check(T v, bool &bad, bool &nonfin, uint32_t &lo, uint32_t &hi) {
    if constexpr (std::is_same<T, float>::value) {
        // NaN fails the comparison; |v| <= 2^54 keeps every squared distance
        // far below FLT_MAX (see the header).
        if (!(fabsf(v) <= 0x1p54f)) bad = true;
        if (!isfinite(v)) nonfin = true;
    } else {
        const uint32_t bv = bias_i32(v);
        lo = max(lo, 0xFFFFFFFFu - bv);
        hi = max(hi, bv);
    }
}

// One CTA handles one block of BLK points at a time.  The block's rows are
// one contiguous span of the source; a pass stages up to PACK_DC coordinates
// of every row in shared memory (row stride dc + 1, so both phases are free
// of bank conflicts) and writes them out coordinate-major, coalesced.  When
// the pass covers whole rows the span is read with 16-byte loads (vec).
// Rows past n are zero.  Floats are checked for NaN/Inf; int32 coordinates
// feed the global range [min, max] kept as two order-preserving unsigned
// maxima: range2[0] = max of ~bias(v) (so min v), range2[1] = max of bias(v).
template <typename T>
__global__ void __launch_bounds__(PACK_NT) pack_kernel(const T *__restrict__ src, int64_t n, int d, bool vec,
                                                       T *__restrict__ dst, uint32_t *range2, DevStatus *st) {
    using V4 = typename std::conditional<std::is_same<T, float>::value, float4, int4>::type;
    __shared__ T tile[BLK * (PACK_DC + 1)];
    const int64_t nb = nblocks(n);
    bool bad = false, nonfin = false;
    uint32_t lo = 0, hi = 0;   // as biased maxima (0 = identity)
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int64_t p0 = b * BLK;
        const int rows = (int)((n - p0) < BLK ? (n - p0) : BLK);
        for (int j0 = 0; j0 < d; j0 += PACK_DC) {
            const int dc = (d - j0) < PACK_DC ? (d - j0) : PACK_DC;
            const int stride = dc + 1;
            __syncthreads();
            if (dc == d) {
                // whole rows: elements f = r d + j of the span [p0 d, (p0 + rows) d)
                const T *base = src + p0 * (int64_t)d;
                const int total = rows * d;
                const int nv = vec ? total / 4 : 0;
                for (int q = threadIdx.x; q < nv; q += PACK_NT) {
                    const V4 w = reinterpret_cast<const V4 *>(base)[q];
                    const T vv[4] = {w.x, w.y, w.z, w.w};
                    int f = 4 * q, r = f / d, j = f - r * d;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        pack_check(vv[u], bad, nonfin, lo, hi);
                        tile[r * stride + j] = vv[u];
                        if (++j == d) {
                            j = 0;
                            ++r;
                        }
                    }
                }
                for (int f = 4 * nv + threadIdx.x; f < total; f += PACK_NT) {
                    const int r = f / d, j = f - r * d;
                    const T v = base[f];
                    pack_check(v, bad, nonfin, lo, hi);
                    tile[r * stride + j] = v;
                }
                for (int f = total + threadIdx.x; f < BLK * d; f += PACK_NT) {
                    const int r = f / d, j = f - r * d;
                    tile[r * stride + j] = T(0);
                }
            } else {
                for (int e = threadIdx.x; e < BLK * dc; e += PACK_NT) {
                    const int r = e / dc, j = e - r * dc;
                    T v = T(0);
                    if (r < rows) {
                        v = src[(p0 + r) * (int64_t)d + j0 + j];
                        pack_check(v, bad, nonfin, lo, hi);
                    }
                    tile[r * stride + j] = v;
                }
            }
            __syncthreads();
            for (int e = threadIdx.x; e < BLK * dc; e += PACK_NT) {
                const int j = e / BLK, r = e - j * BLK;
                dst[(b * d + j0 + j) * BLK + r] = tile[r * stride + j];
            }
        }
    }
    if constexpr (std::is_same<T, float>::value) {
        if (nonfin) set_status(st, KC_ERR_NONFINITE, 1, 0);
        else if (bad) set_status(st, KC_ERR_RANGE, 1, 0);
    } else {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            lo = max(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMax(&range2[0], lo);
            atomicMax(&range2[1], hi);
        }
    }
}

__global__ void range_check_kernel(const int32_t *range2, int d, DevStatus *st) {
    if (ld_volatile_i32(&st->code) == 0 && !int_range_ok(range2, d)) set_status(st, KC_ERR_RANGE, 2, 0);
}

}  // namespace

cudaError_t launch_range_check(const int32_t *range2, int d, DevStatus *st, cudaStream_t s) {
    range_check_kernel<<<1, 1, 0, s>>>(range2, d, st);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pack(const void *src, int dtype, int64_t n, int d, void *dst, int32_t *range2,
                        DevStatus *st, cudaStream_t s) {
    const int64_t nb = nblocks(n);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t cap = (int64_t)sms * 8;
    const int grid = (int)(nb < cap ? nb : cap);
    const bool vec = ((uintptr_t)src & 15) == 0;   // a block's span starts at p0 d, a multiple of 128 elements
    if (dtype == KC_F32)
        pack_kernel<float><<<grid, PACK_NT, 0, s>>>((const float *)src, n, d, vec, (float *)dst,
                                                    (uint32_t *)range2, st);
    else
        pack_kernel<int32_t><<<grid, PACK_NT, 0, s>>>((const int32_t *)src, n, d, vec, (int32_t *)dst,
                                                      (uint32_t *)range2, st);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace kc
