// kc_batch.cu -- device helpers for MRG (Algorithm 1) and for many
// independent instances: packing many arrays in one launch, the round-2
// union of MRG, gathering the union's points, and the per-instance FP64
// radius recheck.
#include <type_traits>

#include "kc_pack.cuh"

namespace kc {

namespace {

// Pack many row-major arrays: segment s covers blocks [blk0[s], blk0[s+1]).
template <typename T>
__global__ void __launch_bounds__(PACK_NT) pack_many_kernel(const PackSeg *__restrict__ segs, int nseg,
                                                            int64_t total_blocks, DevStatus *st) {
    __shared__ T tile[BLK * (PACK_DC + 1)];
    __shared__ PackSeg S;
    __shared__ int s_seg;
    for (int64_t gb = blockIdx.x; gb < total_blocks; gb += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int lo = 0, hi = nseg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (segs[mid].blk0 <= gb) lo = mid;
                else hi = mid - 1;
            }
            s_seg = lo;
            S = segs[lo];
        }
        __syncthreads();
        bool bad = false, nonfin = false;
        uint32_t lo_b = 0, hi_b = 0;
        pack_block<T>((const T *)S.src, S.n, S.d, ((uintptr_t)S.src & 15) == 0, (T *)S.dst, gb - S.blk0, tile, bad,
                      nonfin, lo_b, hi_b);
        if constexpr (std::is_same<T, float>::value) {
            if (nonfin) set_status(st, KC_ERR_NONFINITE, 1, s_seg);
            else if (bad) set_status(st, KC_ERR_RANGE, 1, s_seg);
        } else {
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                lo_b = max(lo_b, __shfl_xor_sync(0xFFFFFFFFu, lo_b, o));
                hi_b = max(hi_b, __shfl_xor_sync(0xFFFFFFFFu, hi_b, o));
            }
            if ((threadIdx.x & 31) == 0 && S.range2) {
                atomicMax((uint32_t *)&S.range2[0], lo_b);
                atomicMax((uint32_t *)&S.range2[1], hi_b);
            }
        }
    }
}

// MRG round 2 input: S = union of the round-1 center sets in ascending global
// index.  The parts are contiguous index ranges in order, so sorting each
// part's centers and concatenating the parts in order sorts the union.  One
// CTA per part; the part's output offset is the sum of the earlier k_out.
__global__ void mrg_union_kernel(const int64_t *__restrict__ c1, const int32_t *__restrict__ k1, int m,
                                 int k, int64_t *__restrict__ U, int64_t *nU) {
    const int i = blockIdx.x;
    __shared__ int64_t s_off;
    if (threadIdx.x == 0) {
        int64_t off = 0;
        for (int j = 0; j < i; ++j) off += k1[j];
        s_off = off;
        if (i == m - 1) *nU = off + k1[i];
    }
    __syncthreads();
    const int ki = k1[i];
    const int64_t *ci = c1 + (int64_t)i * k;
    for (int t = threadIdx.x; t < ki; t += blockDim.x) {
        const int64_t v = ci[t];
        int rank = 0;
        for (int u = 0; u < ki; ++u) rank += ci[u] < v;
        U[s_off + rank] = v;
    }
}

// Pack the points U[0..nU) (global indices into the packed source) into a
// new packed array in U order.
template <typename T>
__global__ void gather_pack_kernel(const T *__restrict__ pk, int d, const int64_t *__restrict__ U,
                                   const int64_t *nU, int64_t cap, T *__restrict__ out) {
    const int64_t nu = *nU;
    const int64_t total = nblocks(cap) * BLK * (int64_t)d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / ((int64_t)d * BLK);
        const int64_t rem = e - b * d * BLK;
        const int j = (int)(rem / BLK), r = (int)(rem - (int64_t)j * BLK);
        const int64_t p = b * BLK + r;
        out[e] = p < nu ? pk[pk_index(U[p], j, d)] : T(0);
    }
}

// Round-2 instance descriptor, finished on the device (its size is known
// only there).
__global__ void mrg_round2_prep_kernel(GonInst *inst, GonInst proto, const int64_t *nU, int kmax) {
    GonInst I = proto;
    I.n = *nU;
    I.k = (int)(I.n < kmax ? I.n : kmax);
    *inst = I;
}

// Per-instance covering radius for the batched form: the FP32 minima and the
// final key are the Gonzalez kernel's; points whose FP32 minimum can reach the
// FP64 maximum (see kc_radius.cu for the bound) get their FP64 minimum over the
// instance's centers, one warp per flagged point.  One CTA per instance.
template <typename T>
__global__ void batch_radius_kernel(const GonInst *__restrict__ insts, int ninst, const DevStatus *st) {
    const int i = blockIdx.x;
    if (i >= ninst || ld_volatile_i32(&st->code) != 0) return;
    const GonInst I = insts[i];
    const uint64_t K = *I.final_key;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    if constexpr (std::is_same<T, int32_t>::value) {
        if (threadIdx.x == 0) *I.radius_out = __dsqrt_rn((double)key_val(K));
        return;
    } else {
        if (key_val(K) == 0) {
            if (threadIdx.x == 0) *I.radius_out = 0.0;
            return;
        }
        __shared__ unsigned long long s_max;
        if (threadIdx.x == 0) s_max = 0;
        __syncthreads();
        const int d = I.d;
        const int kc = *I.k_out;
        const T *pk = (const T *)I.pk;
        const double thr = (double)__uint_as_float(key_val(K)) * (1.0 - 3.0 * f32_gamma(d));
        const float opg = __fadd_ru(1.f, lp_slack(d));
        const float ecmax = I.lp_kind ? *I.ecmax_out : 0.f;
        double best = -1.0;
        for (int64_t base = (int64_t)warp * 32; base < I.n; base += (int64_t)W * 32) {
            const int64_t x = base + lane;
            bool flag = false;
            if (x < I.n) {
                if (I.lp_kind) {
                    const uint32_t hi = ((uint32_t)reinterpret_cast<const uint16_t *>(I.mind)[I.lo + x] + 1u) << 16;
                    const float U = lp_upper(hi, __fadd_ru(I.eblk[(I.lo + x) / BLK], ecmax), opg);
                    flag = (double)U * (double)U >= thr;
                } else {
                    flag = (double)__uint_as_float(I.mind[I.lo + x]) >= thr;
                }
            }
            unsigned todo = __ballot_sync(0xFFFFFFFFu, flag);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const int64_t xs = base + src;
                double mm = INFINITY;
                for (int ci = lane; ci < kc; ci += 32) {
                    const int64_t c = I.centers[ci] - I.base;
                    double s = 0.0;
                    for (int j = 0; j < d; ++j)
                        s = sq_step64(s, pk[pk_index(I.lo + xs, j, d)], pk[pk_index(I.lo + c, j, d)]);
                    mm = fmin(mm, s);
                }
#pragma unroll
                for (int o = 16; o; o >>= 1) mm = fmin(mm, __shfl_xor_sync(0xFFFFFFFFu, mm, o));
                best = fmax(best, mm);
            }
        }
        if (lane == 0 && best >= 0.0) atomicMax(&s_max, (unsigned long long)__double_as_longlong(best));
        __syncthreads();
        if (threadIdx.x == 0) *I.radius_out = __dsqrt_rn(__longlong_as_double((long long)s_max));
    }
}

}  // namespace

cudaError_t launch_pack_many(const PackSeg *segs, int nseg, int64_t total_blocks, int dtype, DevStatus *st,
                             cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t cap = (int64_t)sms * 8;
    const int grid = (int)(total_blocks < cap ? total_blocks : cap);
    if (dtype == KC_F32) pack_many_kernel<float><<<grid, PACK_NT, 0, s>>>(segs, nseg, total_blocks, st);
    else pack_many_kernel<int32_t><<<grid, PACK_NT, 0, s>>>(segs, nseg, total_blocks, st);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mrg_union(const int64_t *c1, const int32_t *k1, int m, int k, int64_t *U, int64_t *nU,
                             cudaStream_t s) {
    mrg_union_kernel<<<m, 256, 0, s>>>(c1, k1, m, k, U, nU);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_pack(const void *pk, int dtype, int d, const int64_t *U, const int64_t *nU,
                               int64_t cap, void *out, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t total = nblocks(cap) * BLK * (int64_t)d;
    const int64_t g = (total + 255) / 256;
    const int grid = (int)(g < (int64_t)sms * 8 ? g : (int64_t)sms * 8);
    if (dtype == KC_F32)
        gather_pack_kernel<float><<<grid, 256, 0, s>>>((const float *)pk, d, U, nU, cap, (float *)out);
    else
        gather_pack_kernel<int32_t><<<grid, 256, 0, s>>>((const int32_t *)pk, d, U, nU, cap, (int32_t *)out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mrg_round2_prep(GonInst *inst, const GonInst &proto, const int64_t *nU, int kmax,
                                   cudaStream_t s) {
    mrg_round2_prep_kernel<<<1, 1, 0, s>>>(inst, proto, nU, kmax);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_batch_radius(const GonInst *insts, int ninst, int dtype, const DevStatus *st,
                                cudaStream_t s) {
    if (dtype == KC_F32) batch_radius_kernel<float><<<ninst, 256, 0, s>>>(insts, ninst, st);
    else batch_radius_kernel<int32_t><<<ninst, 256, 0, s>>>(insts, ninst, st);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace kc
