// kc_pack.cu -- repack row-major points into the blocked coordinate-major
// layout every sweep kernel reads (one pass, before the k sweeps).
#include <type_traits>

#include "kc_internal.cuh"

namespace kc {

namespace {

constexpr int PACK_DC = 32;   // coordinates staged per pass through shared memory

__device__ __forceinline__ uint32_t bias_i32(int32_t v) { return (uint32_t)v ^ 0x80000000u; }

// One CTA of BLK threads handles one block of BLK points at a time: the
// block's rows (contiguous in the source) are read coalesced into shared
// memory, then written out coordinate-major, also coalesced.  Rows past n are
// zero.  Floats are checked for NaN/Inf; int32 coordinates feed the global
// range [min, max] kept as two order-preserving unsigned maxima:
// range2[0] = max of ~bias(v) (so min v), range2[1] = max of bias(v).
template <typename T>
__global__ void __launch_bounds__(BLK) pack_kernel(const T *__restrict__ src, int64_t n, int d,
                                                   T *__restrict__ dst, uint32_t *range2,
                                                   DevStatus *st) {
    __shared__ T tile[BLK][PACK_DC + 1];
    const int64_t nb = nblocks(n);
    bool bad = false, nonfin = false;
    uint32_t lo = 0, hi = 0;   // as biased maxima (0 = identity)
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int64_t p0 = b * BLK;
        const int rows = (int)((n - p0) < BLK ? (n - p0) : BLK);
        for (int j0 = 0; j0 < d; j0 += PACK_DC) {
            const int dc = (d - j0) < PACK_DC ? (d - j0) : PACK_DC;
            __syncthreads();
            for (int e = threadIdx.x; e < BLK * dc; e += BLK) {
                const int r = e / dc, jj = e - r * dc;
                T v = T(0);
                if (r < rows) {
                    v = src[(p0 + r) * (int64_t)d + j0 + jj];
                    if constexpr (std::is_same<T, float>::value) {
                        // NaN fails the comparison; |v| <= 2^54 keeps every
                        // squared distance far below FLT_MAX (see the header).
                        if (!(fabsf(v) <= 0x1p54f)) bad = true;
                        if (!isfinite(v)) nonfin = true;
                    } else {
                        uint32_t bv = bias_i32(v);
                        lo = max(lo, 0xFFFFFFFFu - bv);
                        hi = max(hi, bv);
                    }
                }
                tile[r][jj] = v;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < BLK * dc; e += BLK) {
                const int jj = e / BLK, r = e - jj * BLK;
                dst[(b * d + j0 + jj) * BLK + r] = tile[r][jj];
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
    const int64_t cap = (int64_t)sms * 16;
    const int grid = (int)(nb < cap ? nb : cap);
    if (dtype == KC_F32)
        pack_kernel<float><<<grid, BLK, 0, s>>>((const float *)src, n, d, (float *)dst,
                                                (uint32_t *)range2, st);
    else
        pack_kernel<int32_t><<<grid, BLK, 0, s>>>((const int32_t *)src, n, d, (int32_t *)dst,
                                                  (uint32_t *)range2, st);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace kc
