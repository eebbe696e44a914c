// kc_noalloc.cu -- kc_gonzalez_noalloc: Gonzalez with every byte of device
// scratch taken from one fixed, statically allocated device array, so the
// call itself never allocates memory.
//
// Who needs this: callers that must not allocate device memory during a
// call.  cudaMalloc and cudaFree can synchronise the whole device and stall
// every other stream, which latency-critical loops (a serving loop answering
// requests) cannot afford; and a process whose device memory is already
// reserved by another allocator (a framework's caching allocator that holds
// nearly all HBM) may see a fresh cudaMalloc fail even though the memory is
// idle.  The regular entry points cache their scratch but still allocate it
// on first use and grow it for larger inputs; this one uses the array below
// and nothing else.
//
// Limits and sharing:
//  - The array holds KC_NOALLOC_MAX_BYTES (64 MiB).  Each GPU that loads this
//    library keeps it for the life of the process.  Inputs needing more
//    scratch (roughly n * (4 d + 12) bytes for float points, n * (4 d + 4)
//    for int32) are rejected with KC_ERR_ARG before any work is enqueued.
//  - The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress, with that device current; make that first call
//    before any stream capture.
//  - Every call, from any thread or stream, uses the same array, which keeps
//    the previous call's contents; each call clears the parts that must start
//    at zero.  Calls whose GPU work overlaps in time race on the array and
//    corrupt each other's results: serialise them.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "kc_internal.cuh"

namespace kc {
int gon_warps_per_cta();
void set_last_error(const char *text);   // the text kc_last_error() returns
}

using namespace kc;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[KC_NOALLOC_MAX_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_na_mu;
void *g_na_addr[MAX_DEVICES] = {nullptr};

kc_status na_fail(kc_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return s;
}

#define NA_CUDA(call, what)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return na_fail(KC_ERR_CUDA, "%s: %s", (what), cudaGetErrorString(e_)); \
    } while (0)

// Device address of the static array for the current device (looked up once
// per device, with that device current).
kc_status scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= MAX_DEVICES) return na_fail(KC_ERR_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return na_fail(KC_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                           cudaGetErrorString(e));
        g_na_addr[dev] = p;
    }
    *out = g_na_addr[dev];
    return KC_OK;
}

bool on_device(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice && at.device == dev) || at.type == cudaMemoryTypeManaged;
}

struct Bump {
    size_t off = 0;
    size_t take(size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        size_t at = off;
        off += bytes;
        return at;
    }
};

const char *na_status_text(const DevStatus &d) {
    switch (d.code) {
        case KC_ERR_NONFINITE: return "a float coordinate is NaN or infinite";
        case KC_ERR_RANGE:
            return d.where == 1 ? "a float coordinate exceeds 2^54 in magnitude"
                                : "int32 coordinates too far apart: d*(max-min)^2 must be < 2^32";
        case KC_ERR_TIMEOUT: return "device wait timed out";
        case KC_ERR_ARG: return "invalid device-side argument";
        default: return "device error";
    }
}

}  // namespace

extern "C" kc_status kc_gonzalez_noalloc(const void *pts, int64_t n, int32_t d, int32_t k, int64_t first,
                                         int64_t *centers, int32_t *k_out, double *radius,
                                         const kc_opts *opts) {
    set_last_error("");
    if (!pts || !centers || !k_out || !radius) return na_fail(KC_ERR_ARG, "null pointer argument");
    if (n < 1 || n > (int64_t)N_MAX) return na_fail(KC_ERR_ARG, "n=%lld outside [1, 2^32-2]", (long long)n);
    if (d < 1) return na_fail(KC_ERR_ARG, "d=%d must be >= 1", d);
    if (k < 1) return na_fail(KC_ERR_ARG, "k=%d must be >= 1", k);
    if (first < 0 || first >= n) return na_fail(KC_ERR_ARG, "first=%lld outside [0, n)", (long long)first);
    kc_opts o;
    memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    if (o.dtype != KC_F32 && o.dtype != KC_I32) return na_fail(KC_ERR_ARG, "dtype must be KC_F32 or KC_I32");
    if (o.flags != 0) return na_fail(KC_ERR_ARG, "kc_gonzalez_noalloc takes no flags (it always waits)");
    if (o.sweep != KC_SWEEP_F32)
        return na_fail(KC_ERR_ARG, "kc_gonzalez_noalloc sweeps in FP32 only (sweep must be KC_SWEEP_F32)");
    if (o.reserved != 0) return na_fail(KC_ERR_ARG, "kc_opts.reserved must be 0");
    cudaStream_t s = (cudaStream_t)o.stream;
    int dev = 0;
    NA_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (!on_device(pts, dev) || !on_device(centers, dev) || !on_device(k_out, dev) || !on_device(radius, dev))
        return na_fail(KC_ERR_ARG, "kc_gonzalez_noalloc needs device pointers for all arguments");

    // Scratch plan inside the static array (zero-initialised part first).
    int sms = 0;
    NA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
    const int keff = (int)(k < n ? k : n);
    const int64_t nb = nblocks(n);
    int grid;
    {
        const int maxg = gon_max_grid(o.dtype, d);
        const int W = gon_warps_per_cta();
        int64_t want = (nb + 2 * W - 1) / (2 * W);
        grid = want >= sms ? (int)(((want + sms - 1) / sms) * sms) : (int)(want < 1 ? 1 : want);
        if (grid > maxg) grid = maxg;
        if (grid < 1) return na_fail(KC_ERR_CUDA, "no co-resident grid for the Gonzalez kernel");
    }
    Bump b;
    const size_t o_status = b.take(sizeof(DevStatus));
    const size_t o_range = b.take(2 * sizeof(int32_t));
    const size_t o_key32 = b.take(8), o_max64 = b.take(8), o_arg64 = b.take(8);
    const size_t o_slots = b.take((size_t)slot_words(keff, grid, false) * 8);
    const size_t zero_bytes = b.off;
    const size_t o_pk = b.take((size_t)nb * BLK * d * 4);
    const size_t o_mind = b.take((size_t)nb * BLK * 4);
    const size_t o_cen = b.take((size_t)keff * d * 4);
    const size_t o_m64 = b.take(o.dtype == KC_F32 ? (size_t)n * 8 : 8);
    if (b.off > (size_t)KC_NOALLOC_MAX_BYTES)
        return na_fail(KC_ERR_ARG,
                       "kc_gonzalez_noalloc: n=%lld d=%d k=%d needs %zu bytes of scratch, more than the "
                       "fixed %d-byte static array; use kc_gonzalez",
                       (long long)n, d, k, b.off, (int)KC_NOALLOC_MAX_BYTES);

    void *base = nullptr;
    kc_status r = scratch_address(dev, &base);
    if (r != KC_OK) return r;
    char *p = (char *)base;
    DevStatus *st = (DevStatus *)(p + o_status);

    GonArgs g{};
    gon_single(g, p + o_pk, o.dtype, n, d, keff, first, (uint32_t *)(p + o_mind), (uint64_t *)(p + o_slots),
               centers, k_out, (uint64_t *)(p + o_key32), (const int32_t *)(p + o_range), grid);
    g.st = st;
    {
        int khz = device_clock_khz(dev);
        if (khz <= 0) khz = 2100000;
        g.timeout_cycles = (o.timeout_ms > 0 ? o.timeout_ms : 2000) * (long long)khz;
    }

    RadiusArgs ra{};
    ra.pk = g.single.pk;
    ra.dtype = o.dtype;
    ra.n = n;
    ra.d = d;
    ra.centers = centers;
    ra.kc_dev = k_out;
    ra.kc_max = keff;
    ra.cen = p + o_cen;
    ra.mind = g.single.mind;
    ra.key32 = (unsigned long long *)(p + o_key32);
    ra.max64 = (unsigned long long *)(p + o_max64);
    ra.arg64 = (unsigned long long *)(p + o_arg64);
    ra.m64 = (double *)(p + o_m64);
    ra.radius_out = radius;
    ra.argmax_out = nullptr;
    ra.st = st;
    ra.have_mind = true;

    NA_CUDA(cudaMemsetAsync(p, 0, zero_bytes, s), "scratch clear");
    NA_CUDA(launch_pack(pts, o.dtype, n, d, (void *)g.single.pk, (int32_t *)g.single.range2, st, s),
            "pack launch");
    NA_CUDA(launch_gon(g, s), "gonzalez launch");
    NA_CUDA(launch_radius(ra, s), "radius launch");
    DevStatus hs;
    NA_CUDA(cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s), "status read-back");
    NA_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (hs.code != 0) return na_fail((kc_status)hs.code, "%s", na_status_text(hs));
    return KC_OK;
}
