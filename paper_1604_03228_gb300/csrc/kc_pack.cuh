// kc_pack.cuh -- the block packer shared by the single-array and the
// batched pack kernels: row-major points -> blocks of BLK points,
// coordinate-major inside a block (the layout every sweep kernel reads).
#pragma once
#include <type_traits>

#include "kc_internal.cuh"

namespace kc {

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

// Pack block b of an array of n points of dimension d (src row-major, dst
// the blocked layout) with the CTA's PACK_NT threads.  The block's rows are
// one contiguous span of the source; a pass stages up to PACK_DC coordinates
// of every row in tile (BLK * (PACK_DC + 1) elements, row stride dc + 1, so
// both phases are free of bank conflicts) and writes them out
// coordinate-major, coalesced.  When the pass covers whole rows the span is
// read with 16-byte loads (vec: src is 16-byte aligned).  Rows past n are
// zero.  Checks go to the thread's flags (floats) or running biased range
// (int32).
template <typename T>
__device__ __forceinline__ void pack_block(const T *__restrict__ src, int64_t n, int d, bool vec, T *__restrict__ dst,
                                           int64_t b, T *tile, bool &bad, bool &nonfin, uint32_t &lo, uint32_t &hi) {
    using V4 = typename std::conditional<std::is_same<T, float>::value, float4, int4>::type;
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

}  // namespace kc
