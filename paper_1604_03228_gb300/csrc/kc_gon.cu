// kc_gon.cu -- persistent Gonzalez kernel: all k farthest-point steps of GON
// (Section 3.1; O(k n) distance evaluations, Section 5.1) in one cooperative
// launch, without relaunching between steps.
//
// Each step, every CTA
//   1. reads the newest center's d coordinates into shared memory,
//   2. sweeps its points (a warp streams one 128-point block at a time, lane
//      l owning 4 points with one 16-byte load per coordinate): squared
//      distance to the center, running minimum update (the minimum is only
//      written back where it fell), and the running (value, lowest index)
//      maximum as a 64-bit key,
//   3. reduces the key over the CTA (warp shuffles, then shared memory) and
//      publishes it with a release store into its own slot for this step,
//   4. polls all CTAs' slots of this step (acquire loads, bounded by a cycle
//      budget) and reduces them to the same global key in every CTA.
// The winner of step it is center it+1.  The slot exchange is the only grid
// synchronisation: it carries the data, so no separate barrier or atomic is
// needed.  Slots are per step and zeroed before the launch, so a non-zero
// slot always belongs to the current step.
#include <type_traits>

#include "kc_internal.cuh"

namespace kc {

namespace {

constexpr int GON_NT = 512;
constexpr int GON_W = GON_NT / 32;

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<int32_t> { using type = int4; };

template <typename T, int DC>
__device__ __forceinline__ void dist4(const T *__restrict__ blk, int d, const T *cs, int lane,
                                      typename AccOf<T>::type acc[4]) {
    using V4 = typename Vec4<T>::type;
    const V4 *src = reinterpret_cast<const V4 *>(blk) + lane;
    using A = typename AccOf<T>::type;
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

template <typename T, int DC>
__global__ void __launch_bounds__(GON_NT) gon_kernel(GonArgs a) {
    using A = typename AccOf<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *cs = reinterpret_cast<T *>(smem_raw);
    __shared__ uint64_t red[GON_W];
    __shared__ uint64_t s_key;
    __shared__ int s_abort;

    const int G = gridDim.x, cta = blockIdx.x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int d = DC > 0 ? DC : a.d;
    const int64_t n = a.n;
    const int64_t nb = nblocks(n);
    const T *pk = (const T *)a.pk;

    // Errors from the pack kernel (or an earlier call in async mode) stop
    // every CTA before the first exchange; all CTAs read the same word.
    if (ld_volatile_i32(&a.st->code) != 0) return;
    if constexpr (std::is_same<T, int32_t>::value) {
        if (!int_range_ok(a.range2, d)) {
            if (cta == 0 && tid == 0) set_status(a.st, KC_ERR_RANGE, 2, 0);
            return;
        }
    }
    if (tid == 0) s_abort = 0;
    int64_t c = a.first;
    if (cta == 0 && tid == 0) a.centers[0] = c;

    int it = 0;
    uint64_t K = 0;
    for (it = 0; it < a.k; ++it) {
        for (int j = tid; j < d; j += GON_NT) cs[j] = pk[pk_index(c, j, d)];
        __syncthreads();

        uint64_t best = 0;
        for (int64_t b = (int64_t)cta * GON_W + warp; b < nb; b += (int64_t)G * GON_W) {
            A acc[4];
            dist4<T, DC>(pk + b * d * BLK, d, cs, lane, acc);
            uint4 *mp = reinterpret_cast<uint4 *>(a.mind + b * BLK) + lane;
            uint4 m = make_uint4(acc_bits(acc[0]), acc_bits(acc[1]), acc_bits(acc[2]),
                                 acc_bits(acc[3]));
            if (it == 0) {
                *mp = m;
            } else {
                const uint4 o = *mp;
                const uint4 nm = make_uint4(min(o.x, m.x), min(o.y, m.y), min(o.z, m.z),
                                            min(o.w, m.w));
                if (nm.x != o.x || nm.y != o.y || nm.z != o.z || nm.w != o.w) *mp = nm;
                m = nm;
            }
            const int64_t i0 = b * BLK + lane * 4;
            if (i0 < n) best = umax64(best, make_key(m.x, (uint32_t)i0));
            if (i0 + 1 < n) best = umax64(best, make_key(m.y, (uint32_t)(i0 + 1)));
            if (i0 + 2 < n) best = umax64(best, make_key(m.z, (uint32_t)(i0 + 2)));
            if (i0 + 3 < n) best = umax64(best, make_key(m.w, (uint32_t)(i0 + 3)));
        }

        // CTA reduction, then publish this CTA's key for step `it`.
        best = warp_max_u64(best);
        if (lane == 0) red[warp] = best;
        __syncthreads();
        if (warp == 0) {
            uint64_t v = lane < GON_W ? red[lane] : 0;
            v = warp_max_u64(v);
            if (lane == 0) {
                if (v == 0) v = 1;   // CTA without points: present, never wins
                st_release_u64(&a.slots[(int64_t)it * G + cta], v);
            }
        }

        // Gather every CTA's key of this step.
        uint64_t g = 0;
        for (int s = tid; s < G; s += GON_NT) {
            const uint64_t *p = &a.slots[(int64_t)it * G + s];
            uint64_t v = ld_acquire_u64(p);
            if (v == 0) {
                const long long t0 = clock64();
                while ((v = ld_acquire_u64(p)) == 0) {
                    if (ld_volatile_i32(&a.st->code) != 0 || clock64() - t0 > a.timeout_cycles) {
                        set_status(a.st, KC_ERR_TIMEOUT, 3, it);
                        s_abort = 1;
                        break;
                    }
                }
            }
            g = umax64(g, v);
        }
        g = warp_max_u64(g);
        __syncthreads();   // warp 0 has finished reading red[]
        if (lane == 0) red[warp] = g;
        __syncthreads();
        if (s_abort) return;
        if (warp == 0) {
            uint64_t v = lane < GON_W ? red[lane] : 0;
            v = warp_max_u64(v);
            if (lane == 0) s_key = v;
        }
        __syncthreads();
        K = s_key;
        if (key_val(K) == 0) {   // every point is a center already: stop early
            ++it;
            break;
        }
        if (it + 1 < a.k) {
            c = key_idx(K);
            if (cta == 0 && tid == 0) a.centers[it + 1] = c;
        }
    }
    if (cta == 0 && tid == 0) {
        *a.k_out = it;
        *a.final_key = K;
    }
}

template <typename T, int DC>
void *gon_fn() {
    return (void *)gon_kernel<T, DC>;
}

void *pick_gon(int dtype, int d) {
    if (dtype == KC_F32) {
        switch (d) {
            case 2: return gon_fn<float, 2>();
            case 3: return gon_fn<float, 3>();
            case 8: return gon_fn<float, 8>();
            case 10: return gon_fn<float, 10>();
            case 16: return gon_fn<float, 16>();
            case 32: return gon_fn<float, 32>();
            case 64: return gon_fn<float, 64>();
            default: return gon_fn<float, 0>();
        }
    }
    switch (d) {
        case 2: return gon_fn<int32_t, 2>();
        case 10: return gon_fn<int32_t, 10>();
        default: return gon_fn<int32_t, 0>();
    }
}

}  // namespace

int gon_max_grid(int dtype, int d) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pick_gon(dtype, d), GON_NT,
                                                  (size_t)d * 4);
    return occ * sms;
}

int gon_warps_per_cta() { return GON_W; }

cudaError_t launch_gon(GonArgs &a, cudaStream_t s) {
    void *fn = pick_gon(a.dtype, a.d);
    const size_t smem = (size_t)a.d * 4;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    void *args[] = {&a};
    note_launches(1);
    return cudaLaunchCooperativeKernel(fn, dim3(a.grid), dim3(GON_NT), args, smem, s);
}

}  // namespace kc
