// kc_lp.cu -- low-precision copies of the packed FP32 points for the
// mixed-precision sweep, with a rigorous per-point error bound.
//
// Layout: blocks of BLK points as in the FP32 pack; inside a block, 32-bit
// words hold LP_G consecutive coordinates of one point (bf16, fp16: 2;
// fp8: 4):
//   word (i, jg) at ((i / BLK) * ng + jg) * BLK + i % BLK,  ng = ceil(d / LP_G),
// so a lane's 16-byte load carries 4 points x LP_G coordinates.  Coordinates
// past d are zero.
//
// decoded(x)_j is exactly what the sweep kernel computes from the stored code
// (bf16: the bf16 value; fp8 e4m3: the fp8 value times the column scale
// s_j = max_x |x_j| / 448, one FP32 multiply).  The bound
//   e_x >= || decoded(x) - x ||_2
// sums the exact squared differences with upward rounding.  e_pt holds it
// per point (used for the centers), e_blk the maximum over each block (used in
// the sweep).  The pack also zeroes the per-point stamp of the recheck memo.
//
// fp16 works in scaled units: one power of two S = 2^s for all coordinates,
// s chosen from the largest magnitude M so that M / S < 2^14 (no overflow,
// and 28 binades below it before fp16 runs out of normal numbers).  The code
// is fp16(x / S), decoded(x) its fp16 value, and every quantity the sweep
// uses (distances, e_x, the center bounds) is in units of S; S itself is
// stored in scale[0] for the final radius test.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "kc_internal.cuh"

namespace kc {

namespace {

// Largest |x_j| per column j: one warp covers 32 points of one (block, j);
// the CTA gathers its warps' maxima per column in shared memory (up to
// CM_SMEM columns, else straight in global memory) and adds them to the
// global maxima once, so the global words see one atomic per CTA and column
// instead of one per 32 values.
constexpr int CM_SMEM = 1024;
__global__ void colmax_kernel(const float *__restrict__ pk, int64_t n, int d, unsigned *__restrict__ colmax) {
    __shared__ unsigned cm[CM_SMEM];
    const bool local = d <= CM_SMEM;
    if (local)
        for (int j = threadIdx.x; j < d; j += blockDim.x) cm[j] = 0u;
    __syncthreads();
    const int64_t total = nblocks(n) * (int64_t)d * BLK;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / ((int64_t)d * BLK);
        const int j = (int)((e / BLK) % d);
        const int i = (int)(e % BLK);
        float v = (b * BLK + i < n) ? fabsf(pk[e]) : 0.f;
#pragma unroll
        for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
        if ((threadIdx.x & 31) == 0) atomicMax(local ? &cm[j] : &colmax[j], __float_as_uint(v));
    }
    __syncthreads();
    if (local)
        for (int j = threadIdx.x; j < d; j += blockDim.x)
            if (cm[j]) atomicMax(&colmax[j], cm[j]);
}

__device__ __forceinline__ float fp8_scale(const unsigned *colmax, int j) {
    const float m = __uint_as_float(colmax[j]);
    return m > 0.f ? m / 448.f : 1.f;
}

// fp16 exponent s (S = 2^s) from the column maxima: M / 2^s < 2^14 with M the
// largest magnitude, kept within [-100, 100] (finite coordinates below 2^54
// keep every scaled value and bound finite).
__device__ __forceinline__ int fp16_exponent(const unsigned *colmax, int d) {
    float m = 0.f;
    for (int j = 0; j < d; ++j) m = fmaxf(m, __uint_as_float(colmax[j]));
    if (!(m > 0.f)) return 0;
    int e;
    frexpf(m, &e);   // m = f 2^e, f in [0.5, 1)
    const int s = e - 14;
    return s < -100 ? -100 : (s > 100 ? 100 : s);
}

// One block b of BLK points (one thread per point).
template <int KIND>
__device__ void lp_pack_block(const float *__restrict__ pk, int64_t n, int d, const unsigned *__restrict__ colmax,
                              uint32_t *__restrict__ lp, float *__restrict__ ept, float *__restrict__ eblk,
                              uint32_t *__restrict__ stamp, int64_t b, float fp16_s = 1.f, float fp16_inv = 1.f) {
    constexpr int G = lp_group(KIND);
    const int ng = (d + G - 1) / G;
    {
        const int i = threadIdx.x;
        stamp[b * BLK + i] = 0u;
        const bool valid = b * BLK + i < n;
        float e2 = 0.f;
        for (int jg = 0; jg < ng; ++jg) {
            uint32_t word = 0;
#pragma unroll
            for (int t = 0; t < G; ++t) {
                const int j = jg * G + t;
                const float x = (valid && j < d) ? pk[(b * d + j) * BLK + i] : 0.f;
                float dec;
                uint32_t code;
                if (KIND == KC_SWEEP_BF16) {
                    const __nv_bfloat16 q = __float2bfloat16_rn(x);
                    code = (uint32_t)__bfloat16_as_ushort(q);
                    dec = __uint_as_float(code << 16);
                    word |= code << (16 * t);
                } else if (KIND == KC_SWEEP_FP16) {
                    // fp16(x / S); the unscaled value dec = fp16 * S is exact
                    // (a power-of-two multiple of an 11-bit value, in range)
                    const __half q = __float2half_rn(__fmul_rn(x, fp16_inv));
                    code = (uint32_t)__half_as_ushort(q);
                    dec = __fmul_rn(__half2float(q), fp16_s);
                    word |= code << (16 * t);
                } else {
                    const float s = j < d ? fp8_scale(colmax, j) : 1.f;
                    const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(__fdiv_rn(x, s), __NV_SATFINITE, __NV_E4M3);
                    const __half_raw h = __nv_cvt_fp8_to_halfraw(q, __NV_E4M3);
                    dec = __fmul_rn(__half2float(__half(h)), s);
                    code = (uint32_t)q;
                    word |= code << (8 * t);
                }
                // decoded(x) is within a factor 2 of x (or 0), so the FP32
                // difference is exact (Sterbenz); the sum rounds upward.
                const float diff = fabsf(__fsub_rn(x, dec));
                e2 = __fmaf_ru(diff, diff, e2);
            }
            lp[(b * ng + jg) * BLK + i] = word;
        }
        float e = valid ? __fsqrt_ru(e2) : 0.f;
        if (KIND == KC_SWEEP_FP16) e = __fmul_ru(e, fp16_inv);   // in units of S
        ept[b * BLK + i] = e;
        float m = e;
#pragma unroll
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        __shared__ float wm[BLK / 32];
        if ((i & 31) == 0) wm[i >> 5] = m;
        __syncthreads();
        if (i == 0) {
            float mm = 0.f;
            for (int w = 0; w < BLK / 32; ++w) mm = fmaxf(mm, wm[w]);
            eblk[b] = mm;
        }
        __syncthreads();
    }
}

template <int KIND>
__global__ void __launch_bounds__(BLK) lp_pack_kernel(const float *__restrict__ pk, int64_t n, int d,
                                                      const unsigned *__restrict__ colmax, float *__restrict__ scale,
                                                      uint32_t *__restrict__ lp, float *__restrict__ ept,
                                                      float *__restrict__ eblk, uint32_t *__restrict__ stamp) {
    constexpr int G = lp_group(KIND);
    const int ng = (d + G - 1) / G;
    if (KIND == KC_SWEEP_FP8 && blockIdx.x == 0)
        for (int j = threadIdx.x; j < ng * G; j += blockDim.x) scale[j] = j < d ? fp8_scale(colmax, j) : 1.f;
    float fs = 1.f, fi = 1.f;
    if (KIND == KC_SWEEP_FP16) {
        const int e = fp16_exponent(colmax, d);
        fs = ldexpf(1.f, e);
        fi = ldexpf(1.f, -e);
        if (blockIdx.x == 0 && threadIdx.x == 0) scale[0] = fs;
    }
    for (int64_t b = blockIdx.x; b < nblocks(n); b += gridDim.x)
        lp_pack_block<KIND>(pk, n, d, colmax, lp, ept, eblk, stamp, b, fs, fi);
}

// bf16 copies of many packed arrays in one launch (segment s owns blocks
// [blk0, blk0 + nblocks(n)) of the launch).
__global__ void __launch_bounds__(BLK) lp_pack_many_kernel(const LpSeg *__restrict__ segs, int nseg,
                                                           int64_t total_blocks) {
    __shared__ LpSeg S;
    for (int64_t gb = blockIdx.x; gb < total_blocks; gb += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int lo = 0, hi = nseg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (segs[mid].blk0 <= gb) lo = mid;
                else hi = mid - 1;
            }
            S = segs[lo];
        }
        __syncthreads();
        lp_pack_block<KC_SWEEP_BF16>(S.pk, S.n, S.d, nullptr, S.lp, S.ept, S.eblk, S.stamp, gb - S.blk0);
    }
}

}  // namespace

cudaError_t launch_lp_pack_many(const LpSeg *segs, int nseg, int64_t total_blocks, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)(total_blocks < (int64_t)sms * 16 ? total_blocks : (int64_t)sms * 16);
    lp_pack_many_kernel<<<grid, BLK, 0, s>>>(segs, nseg, total_blocks);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lp_pack(int kind, const float *pk, int64_t n, int d, unsigned *colmax, float *scale, uint32_t *lp,
                           float *ept, float *eblk, uint32_t *stamp, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t nb = nblocks(n);
    const int grid = (int)(nb < (int64_t)sms * 16 ? nb : (int64_t)sms * 16);
    int kernels = 1;
    if (kind == KC_SWEEP_FP8 || kind == KC_SWEEP_FP16) {
        cudaMemsetAsync(colmax, 0, (size_t)d * sizeof(unsigned), s);
        const int64_t total = nb * (int64_t)d * BLK;
        const int g2 = (int)((total + 255) / 256 < (int64_t)sms * 8 ? (total + 255) / 256 : (int64_t)sms * 8);
        colmax_kernel<<<g2, 256, 0, s>>>(pk, n, d, colmax);
        if (kind == KC_SWEEP_FP8)
            lp_pack_kernel<KC_SWEEP_FP8><<<grid, BLK, 0, s>>>(pk, n, d, colmax, scale, lp, ept, eblk, stamp);
        else
            lp_pack_kernel<KC_SWEEP_FP16><<<grid, BLK, 0, s>>>(pk, n, d, colmax, scale, lp, ept, eblk, stamp);
        kernels = 2;
    } else {
        lp_pack_kernel<KC_SWEEP_BF16><<<grid, BLK, 0, s>>>(pk, n, d, colmax, scale, lp, ept, eblk, stamp);
    }
    note_launches(kernels);
    return cudaGetLastError();
}

}  // namespace kc
