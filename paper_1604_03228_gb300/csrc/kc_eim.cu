// kc_eim.cu -- kernels of EIM: EIM-MapReduce-Sample (Algorithm 2) with
// Select and the parameter phi (Algorithm 3, Section 4.2), followed by GON on
// the returned sample.  The host loop that drives them is kc_eim in
// kc_api.cu; one loop iteration is
//   sample    every x in R joins S with probability pS and H with pH, drawn
//             from a counter-based splitmix64 uniform U(seed, it, x, stream)
//   d(H, S)   exact distance of every H point to S (canonical FP32 for float
//             points, exact int32 otherwise)
//   select    the point at 1-based position p of H ordered by distance to S
//             descending, lower index first on ties; its distance is thr
//   prune     x stays in R only if d(x, S) > thr (equal is removed, Section
//             4.1); the scan over S stops at the first center within thr
// and at the end C = S u R is compacted in ascending index order.
#include <type_traits>

#include "kc_internal.cuh"

namespace kc {

namespace {

constexpr int EIM_NT = 256;
constexpr int PRUNE_TILE_BYTES = 32 * 1024;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// U(seed, it, x, stream) in [0, 1): splitmix64 output number (counter + 1) of
// the stream with state `seed`, counter = it << 33 | x << 1 | stream, top 53
// bits scaled by 2^-53 (exact in double).
__device__ __forceinline__ double eim_uniform(uint64_t seed, uint64_t it, uint64_t x, uint64_t stream) {
    const uint64_t ctr = (it << 33) | (x << 1) | stream;
    const uint64_t h = mix64(seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull);
    return (double)(h >> 11) * 0x1p-53;
}

__global__ void iota_kernel(uint32_t *R, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        R[i] = (uint32_t)i;
}

__global__ void sample_kernel(const uint32_t *__restrict__ R, int64_t rn, uint64_t seed, int it, double pS,
                              double pH, uint8_t *__restrict__ inS, uint32_t *__restrict__ S,
                              unsigned long long *sn, uint32_t *__restrict__ H, unsigned long long *hn,
                              int64_t hcap, DevStatus *st) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rn; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = R[i];
        if (eim_uniform(seed, (uint64_t)it, x, 0) < pS) {
            inS[x] = 1;
            S[atomicAdd(sn, 1ull)] = x;
        }
        if (eim_uniform(seed, (uint64_t)it, x, 1) < pH) {
            const unsigned long long pos = atomicAdd(hn, 1ull);
            if ((int64_t)pos < hcap) H[pos] = x;
            else set_status(st, KC_ERR_OOM, 5, (int64_t)pos);
        }
    }
}

// Rows of the row-major source for idx[from..to) into out[(i - from) * d ..].
template <typename T>
__global__ void gather_rows_kernel(const T *__restrict__ src, int d, const uint32_t *__restrict__ idx,
                                   int64_t from, int64_t to, T *__restrict__ out) {
    const int64_t total = (to - from) * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / d;
        const int j = (int)(e - i * d);
        out[(from + i) * d + j] = src[(int64_t)idx[from + i] * d + j];
    }
}

template <typename T>
__device__ __forceinline__ typename AccOf<T>::type dist_rows(const T *a, const T *b, int d) {
    typename AccOf<T>::type acc = 0;
    for (int j = 0; j < d; ++j) acc = sq_step(acc, a[j], b[j]);
    return acc;
}

// d(h, S) for every h in H: thread t of a CTA holds center s (its row in
// registers when d <= DR), loops over the H rows staged in shared memory, and
// the warp minimum per h goes to an atomicMin on dH[h] (value bits; float
// bits of non-negative values order as unsigned integers).
template <typename T, int DR>
__global__ void __launch_bounds__(EIM_NT) dist_hs_kernel(const T *__restrict__ Hc, int64_t hn,
                                                         const T *__restrict__ Sc, int64_t sn, int d,
                                                         uint32_t *__restrict__ dH) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *hs = reinterpret_cast<T *>(smem_raw);
    const int hchunk = PRUNE_TILE_BYTES / (DR * (int)sizeof(T));
    const int lane = threadIdx.x & 31;
    for (int64_t s0 = (int64_t)blockIdx.x * EIM_NT; s0 < sn; s0 += (int64_t)gridDim.x * EIM_NT) {
        const int64_t s = s0 + threadIdx.x;
        const bool valid = s < sn;
        T c[DR];
#pragma unroll
        for (int j = 0; j < DR; ++j) c[j] = (valid && j < d) ? Sc[s * d + j] : T(0);
        for (int64_t h0 = 0; h0 < hn; h0 += hchunk) {
            const int hc = (int)((hn - h0) < hchunk ? (hn - h0) : hchunk);
            __syncthreads();
            for (int e = threadIdx.x; e < hc * DR; e += EIM_NT) {
                const int i = e / DR, j = e - i * DR;
                hs[e] = j < d ? Hc[(h0 + i) * d + j] : T(0);
            }
            __syncthreads();
            for (int i = 0; i < hc; ++i) {
                typename AccOf<T>::type acc = 0;
#pragma unroll
                for (int j = 0; j < DR; ++j) acc = sq_step(acc, hs[i * DR + j], c[j]);
                uint32_t v = valid ? acc_bits(acc) : 0xFFFFFFFFu;
#pragma unroll
                for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
                if (lane == 0) atomicMin(&dH[h0 + i], v);
            }
        }
    }
}

// Generic d > 64 version: one thread per (h, s-chunk) pair is too little
// work, so this one simply loops rows from global memory.
template <typename T>
__global__ void dist_hs_generic_kernel(const T *__restrict__ Hc, int64_t hn, const T *__restrict__ Sc,
                                       int64_t sn, int d, uint32_t *__restrict__ dH) {
    const int lane = threadIdx.x & 31;
    for (int64_t s0 = (int64_t)blockIdx.x * blockDim.x; s0 < sn; s0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = s0 + threadIdx.x;
        for (int64_t i = 0; i < hn; ++i) {
            uint32_t v = s < sn ? acc_bits(dist_rows<T>(Hc + i * d, Sc + s * d, d)) : 0xFFFFFFFFu;
#pragma unroll
            for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
            if (lane == 0) atomicMin(&dH[i], v);
        }
    }
}

// Select (Algorithm 3): rank of every H point in (distance desc, index asc)
// order; the one at rank p-1 gives thr.
__global__ void select_kernel(const uint32_t *__restrict__ H, const uint32_t *__restrict__ dH, int64_t hn,
                              int64_t p, uint32_t *thr, uint32_t *v) {
    for (int64_t i = threadIdx.x; i < hn; i += blockDim.x) {
        const uint32_t di = dH[i], xi = H[i];
        int64_t rank = 0;
        for (int64_t j = 0; j < hn; ++j) {
            const uint32_t dj = dH[j];
            rank += (dj > di) || (dj == di && H[j] < xi);
        }
        if (rank == p - 1) {
            *thr = di;
            *v = xi;
        }
    }
}

// Prune: x in R stays iff d(x, S) > thr.  A CTA takes EIM_NT points of R
// (one per thread, coordinates in registers) and walks S in shared-memory
// tiles; a thread stops at its first center within thr, and the CTA stops
// when all of its points are decided.
template <typename T, int DR>
__global__ void __launch_bounds__(EIM_NT) prune_kernel(const T *__restrict__ src, int d,
                                                       const uint32_t *__restrict__ R, int64_t rn,
                                                       const uint8_t *__restrict__ inS,
                                                       const T *__restrict__ Sc, int64_t sn,
                                                       const uint32_t *thr_p, uint32_t *__restrict__ Rn,
                                                       unsigned long long *rnn) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *cs = reinterpret_cast<T *>(smem_raw);
    const int tile = PRUNE_TILE_BYTES / (DR * (int)sizeof(T));
    const uint32_t thr = *thr_p;
    for (int64_t r0 = (int64_t)blockIdx.x * EIM_NT; r0 < rn; r0 += (int64_t)gridDim.x * EIM_NT) {
        const int64_t i = r0 + threadIdx.x;
        const bool valid = i < rn;
        const uint32_t x = valid ? R[i] : 0u;
        bool removed = !valid || inS[x];      // d(x, S) = 0 for sampled points
        T xc[DR];
#pragma unroll
        for (int j = 0; j < DR; ++j) xc[j] = (!removed && j < d) ? src[(int64_t)x * d + j] : T(0);
        for (int64_t t0 = 0; t0 < sn; t0 += tile) {
            if (__syncthreads_and(removed)) break;
            const int tc = (int)((sn - t0) < tile ? (sn - t0) : tile);
            for (int e = threadIdx.x; e < tc * DR; e += EIM_NT) {
                const int ci = e / DR, j = e - ci * DR;
                cs[e] = j < d ? Sc[(t0 + ci) * d + j] : T(0);
            }
            __syncthreads();
            if (!removed) {
                for (int ci = 0; ci < tc; ++ci) {
                    typename AccOf<T>::type acc = 0;
#pragma unroll
                    for (int j = 0; j < DR; ++j) acc = sq_step(acc, xc[j], cs[ci * DR + j]);
                    if (acc_bits(acc) <= thr) {
                        removed = true;
                        break;
                    }
                }
            }
        }
        if (!removed) Rn[atomicAdd(rnn, 1ull)] = x;
        __syncthreads();
    }
}

template <typename T>
__global__ void prune_generic_kernel(const T *__restrict__ src, int d, const uint32_t *__restrict__ R,
                                     int64_t rn, const uint8_t *__restrict__ inS, const T *__restrict__ Sc,
                                     int64_t sn, const uint32_t *thr_p, uint32_t *__restrict__ Rn,
                                     unsigned long long *rnn) {
    const uint32_t thr = *thr_p;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rn; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = R[i];
        bool removed = inS[x];
        for (int64_t s = 0; s < sn && !removed; ++s)
            removed = acc_bits(dist_rows<T>(src + (int64_t)x * d, Sc + s * d, d)) <= thr;
        if (!removed) Rn[atomicAdd(rnn, 1ull)] = x;
    }
}

// R without the points just sampled into S (no pivot this iteration).
__global__ void drop_sampled_kernel(const uint32_t *__restrict__ R, int64_t rn, const uint8_t *__restrict__ inS,
                                    uint32_t *__restrict__ Rn, unsigned long long *rnn) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rn; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = R[i];
        if (!inS[x]) Rn[atomicAdd(rnn, 1ull)] = x;
    }
}

__global__ void mark_kernel(const uint32_t *__restrict__ R, int64_t rn, uint8_t *__restrict__ mask) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rn; i += (int64_t)gridDim.x * blockDim.x)
        mask[R[i]] = 1;
}

// Ordered compaction of a byte mask into ascending int64 indices:
// per-chunk counts, one-CTA exclusive scan, then per-chunk ordered writes.
constexpr int CMP_NT = 1024;

__global__ void compact_count_kernel(const uint8_t *__restrict__ mask, int64_t n, int *__restrict__ counts) {
    for (int64_t c = blockIdx.x; c * CMP_NT < n; c += gridDim.x) {
        const int64_t i = c * CMP_NT + threadIdx.x;
        const int cnt = __syncthreads_count(i < n && mask[i]);
        if (threadIdx.x == 0) counts[c] = cnt;
    }
}

__global__ void compact_scan_kernel(const int *__restrict__ counts, int64_t nchunks, int64_t *__restrict__ offs,
                                    int64_t *total) {
    __shared__ int64_t part[CMP_NT];
    const int64_t per = (nchunks + CMP_NT - 1) / CMP_NT;
    const int64_t a = threadIdx.x * per, b = (a + per) < nchunks ? (a + per) : nchunks;
    int64_t s = 0;
    for (int64_t i = a; i < b; ++i) s += counts[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int t = 0; t < CMP_NT; ++t) {
            const int64_t v = part[t];
            part[t] = run;
            run += v;
        }
        *total = run;
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int64_t i = a; i < b; ++i) {
        offs[i] = run;
        run += counts[i];
    }
}

__global__ void compact_write_kernel(const uint8_t *__restrict__ mask, int64_t n, const int64_t *__restrict__ offs,
                                     int64_t *__restrict__ out) {
    __shared__ int wsum[CMP_NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c = blockIdx.x; c * CMP_NT < n; c += gridDim.x) {
        const int64_t i = c * CMP_NT + threadIdx.x;
        const bool f = i < n && mask[i];
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, f);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        if (f) out[offs[c] + before + __popc(bal & ((1u << lane) - 1u))] = i;
        __syncthreads();
    }
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

int grid_for(int64_t work, int nt, int per_sm = 8) {
    const int64_t g = (work + nt - 1) / nt;
    const int64_t cap = (int64_t)sm_count() * per_sm;
    return (int)(g < 1 ? 1 : (g < cap ? g : cap));
}

}  // namespace

cudaError_t launch_eim_iota(uint32_t *R, int64_t n, cudaStream_t s) {
    iota_kernel<<<grid_for(n, 256), 256, 0, s>>>(R, n);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_eim_sample(const uint32_t *R, int64_t rn, uint64_t seed, int it, double pS, double pH,
                              uint8_t *inS, uint32_t *S, unsigned long long *sn, uint32_t *H, unsigned long long *hn,
                              int64_t hcap, DevStatus *st, cudaStream_t s) {
    sample_kernel<<<grid_for(rn, 256), 256, 0, s>>>(R, rn, seed, it, pS, pH, inS, S, sn, H, hn, hcap, st);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_eim_gather_rows(const void *src, int dtype, int d, const uint32_t *idx, int64_t from, int64_t to,
                                   void *out, cudaStream_t s) {
    if (to <= from) return cudaSuccess;
    const int g = grid_for((to - from) * d, 256);
    if (dtype == KC_F32)
        gather_rows_kernel<float><<<g, 256, 0, s>>>((const float *)src, d, idx, from, to, (float *)out);
    else
        gather_rows_kernel<int32_t><<<g, 256, 0, s>>>((const int32_t *)src, d, idx, from, to, (int32_t *)out);
    note_launches(1);
    return cudaGetLastError();
}

template <typename T, int DR>
static void run_dist_hs(const void *Hc, int64_t hn, const void *Sc, int64_t sn, int d, uint32_t *dH, cudaStream_t s) {
    const int hchunk = PRUNE_TILE_BYTES / (DR * (int)sizeof(T));
    const size_t smem = (size_t)hchunk * DR * sizeof(T);
    dist_hs_kernel<T, DR><<<grid_for(sn, EIM_NT, 4), EIM_NT, smem, s>>>((const T *)Hc, hn, (const T *)Sc, sn, d, dH);
}

cudaError_t launch_eim_dist_hs(int dtype, const void *Hc, int64_t hn, const void *Sc, int64_t sn, int d, uint32_t *dH,
                               cudaStream_t s) {
    cudaMemsetAsync(dH, 0xFF, (size_t)hn * sizeof(uint32_t), s);
    if (dtype == KC_F32) {
        if (d <= 16) run_dist_hs<float, 16>(Hc, hn, Sc, sn, d, dH, s);
        else if (d <= 64) run_dist_hs<float, 64>(Hc, hn, Sc, sn, d, dH, s);
        else dist_hs_generic_kernel<float><<<grid_for(sn, 256, 4), 256, 0, s>>>((const float *)Hc, hn, (const float *)Sc, sn, d, dH);
    } else {
        if (d <= 16) run_dist_hs<int32_t, 16>(Hc, hn, Sc, sn, d, dH, s);
        else if (d <= 64) run_dist_hs<int32_t, 64>(Hc, hn, Sc, sn, d, dH, s);
        else dist_hs_generic_kernel<int32_t><<<grid_for(sn, 256, 4), 256, 0, s>>>((const int32_t *)Hc, hn, (const int32_t *)Sc, sn, d, dH);
    }
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_eim_select(const uint32_t *H, const uint32_t *dH, int64_t hn, int64_t p, uint32_t *thr, uint32_t *v,
                              cudaStream_t s) {
    select_kernel<<<1, 1024, 0, s>>>(H, dH, hn, p, thr, v);
    note_launches(1);
    return cudaGetLastError();
}

template <typename T, int DR>
static void run_prune(const void *src, int d, const uint32_t *R, int64_t rn, const uint8_t *inS, const void *Sc,
                      int64_t sn, const uint32_t *thr, uint32_t *Rn, unsigned long long *rnn, cudaStream_t s) {
    const int tile = PRUNE_TILE_BYTES / (DR * (int)sizeof(T));
    const size_t smem = (size_t)tile * DR * sizeof(T);
    prune_kernel<T, DR><<<grid_for(rn, EIM_NT, 8), EIM_NT, smem, s>>>((const T *)src, d, R, rn, inS, (const T *)Sc, sn,
                                                                      thr, Rn, rnn);
}

cudaError_t launch_eim_prune(int dtype, const void *src, int d, const uint32_t *R, int64_t rn, const uint8_t *inS,
                             const void *Sc, int64_t sn, const uint32_t *thr, uint32_t *Rn, unsigned long long *rnn,
                             cudaStream_t s) {
    if (dtype == KC_F32) {
        // the coordinate count rounded up to a power of two (zero terms are
        // still evaluated, so a tight bound matters most at small d)
        if (d <= 2) run_prune<float, 2>(src, d, R, rn, inS, Sc, sn, thr, Rn, rnn, s);
        else if (d <= 4) run_prune<float, 4>(src, d, R, rn, inS, Sc, sn, thr, Rn, rnn, s);
        else if (d <= 8) run_prune<float, 8>(src, d, R, rn, inS, Sc, sn, thr, Rn, rnn, s);
        else if (d <= 16) run_prune<float, 16>(src, d, R, rn, inS, Sc, sn, thr, Rn, rnn, s);
        else if (d <= 64) run_prune<float, 64>(src, d, R, rn, inS, Sc, sn, thr, Rn, rnn, s);
        else prune_generic_kernel<float><<<grid_for(rn, 256), 256, 0, s>>>((const float *)src, d, R, rn, inS, (const float *)Sc, sn, thr, Rn, rnn);
    } else {
        if (d <= 2) run_prune<int32_t, 2>(src, d, R, rn, inS, Sc, sn, thr, Rn, rnn, s);
        else if (d <= 4) run_prune<int32_t, 4>(src, d, R, rn, inS, Sc, sn, thr, Rn, rnn, s);
        else if (d <= 8) run_prune<int32_t, 8>(src, d, R, rn, inS, Sc, sn, thr, Rn, rnn, s);
        else if (d <= 16) run_prune<int32_t, 16>(src, d, R, rn, inS, Sc, sn, thr, Rn, rnn, s);
        else if (d <= 64) run_prune<int32_t, 64>(src, d, R, rn, inS, Sc, sn, thr, Rn, rnn, s);
        else prune_generic_kernel<int32_t><<<grid_for(rn, 256), 256, 0, s>>>((const int32_t *)src, d, R, rn, inS, (const int32_t *)Sc, sn, thr, Rn, rnn);
    }
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_eim_drop_sampled(const uint32_t *R, int64_t rn, const uint8_t *inS, uint32_t *Rn,
                                    unsigned long long *rnn, cudaStream_t s) {
    drop_sampled_kernel<<<grid_for(rn, 256), 256, 0, s>>>(R, rn, inS, Rn, rnn);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_eim_mark(const uint32_t *R, int64_t rn, uint8_t *mask, cudaStream_t s) {
    if (rn <= 0) return cudaSuccess;
    mark_kernel<<<grid_for(rn, 256), 256, 0, s>>>(R, rn, mask);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_compact(const uint8_t *mask, int64_t n, int *counts, int64_t *offs, int64_t *out, int64_t *total,
                           cudaStream_t s) {
    const int64_t nchunks = (n + CMP_NT - 1) / CMP_NT;
    const int g = (int)(nchunks < (int64_t)sm_count() * 2 ? nchunks : (int64_t)sm_count() * 2);
    compact_count_kernel<<<g, CMP_NT, 0, s>>>(mask, n, counts);
    compact_scan_kernel<<<1, CMP_NT, 0, s>>>(counts, nchunks, offs, total);
    compact_write_kernel<<<g, CMP_NT, 0, s>>>(mask, n, offs, out);
    note_launches(3);
    return cudaGetLastError();
}

}  // namespace kc
