// kc_probe.cu -- kc_read_sweep: a plain read of a device buffer, repeated in
// one launch, for the bandwidth roofline of a sweep whose points stay in L2
// (the paper has no counterpart; Section 5.1's k passes over the points are
// what it bounds).  Every thread streams 16-byte words grid-stride and folds
// them with XOR into one word per CTA, so no load can be dropped and the
// only stores are one per CTA.
#include "kc_internal.cuh"

namespace kc {
namespace {

constexpr int PROBE_NT = 512;

__global__ void __launch_bounds__(PROBE_NT) read_sweep_kernel(const uint4 *__restrict__ buf, int64_t words, int reps,
                                                              unsigned long long *sink) {
    uint32_t acc = 0;
    const int64_t stride = (int64_t)gridDim.x * PROBE_NT;
    for (int r = 0; r < reps; ++r) {
        // four independent loads in flight per thread
        int64_t i = blockIdx.x * (int64_t)PROBE_NT + threadIdx.x;
        for (; i + 3 * stride < words; i += 4 * stride) {
            const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride), c = __ldcg(buf + i + 2 * stride),
                        d = __ldcg(buf + i + 3 * stride);
            acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
        }
        for (; i < words; i += stride) {
            const uint4 a = __ldcg(buf + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
        acc = acc * 0x9E3779B9u + (uint32_t)r;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc ^= __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicXor(sink, (unsigned long long)acc);
}

}  // namespace
}  // namespace kc

using namespace kc;

extern "C" kc_status kc_read_sweep(const void *buf, size_t bytes, int32_t reps, unsigned long long *sink,
                                   void *stream) {
    if (!buf || !sink || reps < 1 || bytes < 16 || (bytes & 15) || ((uintptr_t)buf & 15)) return KC_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return KC_ERR_CUDA;
    note_launches(1);
    read_sweep_kernel<<<sms * 4, PROBE_NT, 0, (cudaStream_t)stream>>>((const uint4 *)buf, (int64_t)(bytes / 16), reps,
                                                                       sink);
    return cudaGetLastError() == cudaSuccess ? KC_OK : KC_ERR_CUDA;
}
