// kc_pack.cu -- repack row-major points into the blocked coordinate-major
// layout every sweep kernel reads (one pass, before the k sweeps).
#include <type_traits>

#include "kc_pack.cuh"

namespace kc {

namespace {

// Floats are checked for NaN/Inf; int32 coordinates feed the global range
// [min, max] kept as two order-preserving unsigned maxima: range2[0] = max of
// ~bias(v) (so min v), range2[1] = max of bias(v).
template <typename T>
__global__ void __launch_bounds__(PACK_NT) pack_kernel(const T *__restrict__ src, int64_t n, int d, bool vec,
                                                       T *__restrict__ dst, uint32_t *range2, DevStatus *st) {
    __shared__ T tile[BLK * (PACK_DC + 1)];
    bool bad = false, nonfin = false;
    uint32_t lo = 0, hi = 0;   // as biased maxima (0 = identity)
    for (int64_t b = blockIdx.x; b < nblocks(n); b += gridDim.x) pack_block<T>(src, n, d, vec, dst, b, tile, bad, nonfin, lo, hi);
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
