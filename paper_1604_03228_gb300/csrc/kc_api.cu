// kc_api.cu -- the C ABI (include/kcenter.h): argument checks, host/device
// pointer handling, cached device scratch, and the launch sequence of each
// entry point.  All arithmetic of the method runs in the kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "kc_internal.cuh"

namespace kc {
int gon_warps_per_cta();
}

using namespace kc;

namespace {

thread_local std::string g_err;

// ------------------------------------------------------------ tracing
std::atomic<int64_t> g_launches{0};
std::atomic<unsigned long long> g_prune_pairs{0};   // sum of |R| x |S| over EIM prunes
std::atomic<int> g_trace_on{0};
thread_local int t_kernels = 0;

struct TraceRec {
    char name[24];
    int kernels;
    cudaEvent_t a, b;
};
std::mutex g_tmu;
std::vector<TraceRec> g_trace;
std::vector<cudaEvent_t> g_evpool;

cudaEvent_t ev_get() {
    std::lock_guard<std::mutex> lk(g_tmu);
    if (!g_evpool.empty()) {
        cudaEvent_t e = g_evpool.back();
        g_evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one launch step with events on the call's stream while tracing.
struct TraceStep {
    bool on;
    TraceRec r{};
    cudaStream_t s;
    int k0 = 0;
    TraceStep(const char *name, cudaStream_t s_) : on(name != nullptr && g_trace_on.load() != 0), s(s_) {
        if (!on) return;
        strncpy(r.name, name, sizeof r.name - 1);
        r.a = ev_get();
        r.b = ev_get();
        cudaEventRecord(r.a, s);
        k0 = t_kernels;
    }
    ~TraceStep() {
        if (!on) return;
        cudaEventRecord(r.b, s);
        r.kernels = t_kernels - k0;
        std::lock_guard<std::mutex> lk(g_tmu);
        g_trace.push_back(r);
    }
};

kc_status fail(kc_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

kc_status cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(KC_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(KC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define KC_CUDA(call, what)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, (what));  \
    } while (0)

// ------------------------------------------------------------ scratch
// Device scratch is cached per (device, stream): a grow-only arena plus a
// small persistent status word and a pinned host mirror for read-back.
struct Arena {
    char *dev = nullptr;
    size_t bytes = 0;
    DevStatus *status = nullptr;   // persistent across calls on this stream
    DevStatus *host_status = nullptr;
    char *pinned = nullptr;        // staging for descriptor uploads
    size_t pinned_bytes = 0;
    cudaEvent_t pinned_ev = nullptr;
    bool pinned_busy = false;
    // the argmax key (value bits: the largest canonical FP32 minimum) of the
    // last solve or radius on this stream, for kc_last_fp32_radius
    const unsigned long long *last_key32 = nullptr;
    int last_dtype = KC_F32;
};

// Copy `bytes` of host data to device memory `dst` in stream order through
// the arena's pinned staging buffer (waiting first for the previous upload
// from that buffer to finish).
kc_status upload(Arena *a, cudaStream_t s, const void *src, size_t bytes, void *dst) {
    if (bytes == 0) return KC_OK;
    if (a->pinned_busy) {
        KC_CUDA(cudaEventSynchronize(a->pinned_ev), "cudaEventSynchronize");
        a->pinned_busy = false;
    }
    if (bytes > a->pinned_bytes) {
        if (a->pinned) cudaFreeHost(a->pinned);
        a->pinned = nullptr;
        a->pinned_bytes = 0;
        const size_t want = bytes + bytes / 4 + 4096;
        KC_CUDA(cudaMallocHost(&a->pinned, want), "pinned staging allocation");
        a->pinned_bytes = want;
    }
    if (!a->pinned_ev) KC_CUDA(cudaEventCreateWithFlags(&a->pinned_ev, cudaEventDisableTiming), "cudaEventCreate");
    memcpy(a->pinned, src, bytes);
    KC_CUDA(cudaMemcpyAsync(dst, a->pinned, bytes, cudaMemcpyHostToDevice, s), "descriptor upload");
    KC_CUDA(cudaEventRecord(a->pinned_ev, s), "cudaEventRecord");
    a->pinned_busy = true;
    return KC_OK;
}

std::mutex g_mu;
std::map<std::pair<int, uintptr_t>, Arena *> g_arenas;

kc_status arena_for(cudaStream_t s, Arena **out) {
    int dev = 0;
    KC_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_pair(dev, (uintptr_t)s);
    auto it = g_arenas.find(key);
    if (it != g_arenas.end()) {
        *out = it->second;
        return KC_OK;
    }
    Arena *a = new Arena();
    cudaError_t e = cudaMalloc(&a->status, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMemset(a->status, 0, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMallocHost(&a->host_status, sizeof(DevStatus));
    if (e != cudaSuccess) {
        if (a->status) cudaFree(a->status);
        delete a;
        return cuda_fail(e, "scratch status allocation");
    }
    g_arenas[key] = a;
    *out = a;
    return KC_OK;
}

kc_status arena_reserve(Arena *a, size_t bytes, cudaStream_t s) {
    if (bytes <= a->bytes) return KC_OK;
    KC_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (a->dev) cudaFree(a->dev);
    a->dev = nullptr;
    a->bytes = 0;
    const size_t want = bytes + bytes / 8 + (1u << 20);
    cudaError_t e = cudaMalloc(&a->dev, want);
    if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
    a->bytes = want;
    return KC_OK;
}

// Bump allocator over the arena (run once with base == nullptr to size it).
struct Carve {
    char *base;
    size_t off = 0;
    explicit Carve(char *b) : base(b) {}
    template <typename T> T *take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

bool is_device_ptr(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeDevice) return at.device == dev;
    if (at.type == cudaMemoryTypeManaged) return true;
    return false;
}

// The address at which the device reads a pinned (page-locked, mapped) host
// buffer, or null for pageable or device memory.
const void *pinned_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost) return nullptr;
    return at.devicePointer;
}

kc_opts default_opts() {
    kc_opts o;
    memset(&o, 0, sizeof o);
    o.dtype = KC_F32;
    o.phi = 6.0;
    return o;
}

long long timeout_cycles(const kc_opts &o) {
    int dev = 0;
    cudaGetDevice(&dev);
    int khz = device_clock_khz(dev);
    if (khz <= 0) khz = 2100000;
    const long long ms = o.timeout_ms > 0 ? o.timeout_ms : 2000;
    return ms * (long long)khz;
}

const char *where_name(int w) {
    switch (w) {
        case 1: return "point check";
        case 2: return "int32 range check";
        case 3: return "GON step exchange";
        case 4: return "center index check";
        case KC_AT_CENTER_LOAD: return "GON winner index (checked build)";
        case KC_AT_RESIDENT_SMEM: return "resident shared-memory column (checked build)";
        case KC_AT_CANDIDATE: return "candidate buffer (checked build)";
        case KC_AT_RECHECK: return "exact recheck index (checked build)";
        case KC_AT_CENTER_COPY: return "center copy slot (checked build)";
        case KC_AT_EIM_INDEX: return "EIM point index (checked build)";
        case KC_AT_RADIUS_LIST: return "radius recheck list (checked build)";
        case KC_AT_SLOT: return "exchange slot (checked build)";
        default: return "device";
    }
}

kc_status status_text(const DevStatus &d) {
    switch (d.code) {
        case KC_OK: return KC_OK;
        case KC_ERR_NONFINITE:
            return fail(KC_ERR_NONFINITE, "a float coordinate is NaN or infinite");
        case KC_ERR_RANGE:
            return fail(KC_ERR_RANGE,
                        d.where == 1 ? "a float coordinate exceeds 2^54 in magnitude"
                                     : "int32 coordinates too far apart: d*(max-min)^2 must be < 2^32");
        case KC_ERR_TIMEOUT:
            return fail(KC_ERR_TIMEOUT, "device wait timed out in %s (step %lld)", where_name(d.where),
                        (long long)d.info);
        case KC_ERR_ARG:
            return fail(KC_ERR_ARG, "%s failed (item %lld)", where_name(d.where), (long long)d.info);
        case KC_ERR_BOUNDS:
            return fail(KC_ERR_BOUNDS, "index %lld outside its buffer at %s", (long long)d.info, where_name(d.where));
        default:
            return fail((kc_status)d.code, "device error %d in %s", d.code, where_name(d.where));
    }
}

// Wait for the stream, read and clear the status word.
kc_status finish(Arena *a, cudaStream_t s) {
    KC_CUDA(cudaMemcpyAsync(a->host_status, a->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s),
            "status read-back");
    KC_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    DevStatus d = *a->host_status;
    if (d.code != 0) {
        KC_CUDA(cudaMemset(a->status, 0, sizeof(DevStatus)), "status reset");
        return status_text(d);
    }
    return KC_OK;
}

struct CallCtx {
    kc_opts o;
    cudaStream_t s;
    int dev;
    bool async;
    Arena *arena;
};

kc_status begin(const kc_opts *opts, CallCtx &c, uint32_t allowed = KC_ASYNC) {
    c.o = opts ? *opts : default_opts();
    if (c.o.dtype != KC_F32 && c.o.dtype != KC_I32) return fail(KC_ERR_ARG, "dtype must be KC_F32 or KC_I32");
    if (c.o.flags & ~allowed) return fail(KC_ERR_ARG, "flags 0x%x not accepted by this call", c.o.flags);
    if (c.o.sweep < KC_SWEEP_F32 || c.o.sweep > KC_SWEEP_FP16) return fail(KC_ERR_ARG, "unknown sweep %d", c.o.sweep);
    c.s = (cudaStream_t)c.o.stream;
    c.async = (c.o.flags & KC_ASYNC) != 0;
    KC_CUDA(cudaGetDevice(&c.dev), "cudaGetDevice");
    return arena_for(c.s, &c.arena);
}

// Input points: device pointer as is, else copied into `staging`.
// The points as the pack kernel reads them: device memory as is; pinned host
// memory in place (pin: its device address; the kernel reads it once over
// the host link); pageable memory through the staging copy.
kc_status stage_points(const CallCtx &c, const void *pts, size_t bytes, bool dev_in, void *staging,
                       const void **out, const void *pin = nullptr) {
    if (dev_in) {
        *out = pts;
        return KC_OK;
    }
    if (pin) {
        *out = pin;
        return KC_OK;
    }
    KC_CUDA(cudaMemcpyAsync(staging, pts, bytes, cudaMemcpyHostToDevice, c.s), "copy points to device");
    *out = staging;
    return KC_OK;
}

// Low-precision sweep kind for a call: only float points use it.
int lp_of(const kc_opts &o) { return o.dtype == KC_F32 ? o.sweep : 0; }

// CTA groups of the mixed-precision sweep filter their exact rechecks against
// their own largest lower bound (1) or the group's (0, the default);
// KC_LP_LOCAL_T=0|1 overrides.  Measured on 8M x 64, k = 1024: the CTA's own
// bound skips one exchange per step but leaves a different CTA rechecking
// the most points at every step (bf16 180 -> 365 ms, fp16 183 -> 239 ms).
int lp_local_t(int lp) {
    (void)lp;
    if (const char *env = getenv("KC_LP_LOCAL_T")) return atoi(env) != 0;
    return 0;
}

// Scratch of the mixed-precision sweep over one packed array of n points.
struct LPBufs {
    uint32_t *lp = nullptr;
    float *eblk = nullptr, *ept = nullptr, *scale = nullptr;
    unsigned *colmax = nullptr;
    uint32_t *m32 = nullptr, *stamp = nullptr;   // recheck memo
};

void take_lp(Carve &cv, LPBufs &L, int lp, int64_t n, int d) {
    if (!lp) {
        L = LPBufs{};
        return;
    }
    const int64_t nb = nblocks(n);
    const int ng = lp_ngroups(lp, d);
    L.lp = cv.take<uint32_t>((size_t)nb * ng * BLK);
    L.eblk = cv.take<float>((size_t)nb);
    L.ept = cv.take<float>((size_t)nb * BLK);
    L.scale = cv.take<float>((size_t)ng * 4);
    L.colmax = cv.take<unsigned>((size_t)d);
    L.m32 = cv.take<uint32_t>((size_t)nb * BLK);
    L.stamp = cv.take<uint32_t>((size_t)nb * BLK);
}

// Tensor-core radius filter scratch for kc centers over n float points
// (left null, i.e. CUDA cores, for int32 points, d > 128, little work per
// point, or KC_RADIUS_TC=0 in the environment).  The CUDA cores' time grows
// with k d per point, the tensor-core path's with ceil(k / 256) (Kp = d + 3
// rounded up to 16) plus a dozen launches; measured on uniform points
// (ms per call, CUDA cores against tensor cores): 10M x 16, k = 200: 2.35
// against 1.00; 10M x 8, k = 200: 1.28 against 0.86; 2M x 32, k = 100: 1.92
// against 0.39; 1M x 16, k = 200: 0.37 against 0.27; but 1M x 10, k = 100:
// 0.22 against 0.26; 10M x 16, k = 64: 0.94 against 1.00; 10M x 4, k = 200:
// 0.75 against 0.88.  So: k d >= 1536 from 256k points, k d >= 8192 below.
bool tc_radius_wanted(int dtype, int64_t n, int d, int kc) {
    const int64_t kd = (int64_t)kc * d;
    bool use = dtype == KC_F32 && tc_supported(d) && (kd >= 8192 || (kd >= 1536 && n >= 262144));
    if (const char *env = getenv("KC_RADIUS_TC")) use = dtype == KC_F32 && tc_supported(d) && atoi(env) != 0;
    return use;
}

void take_tc(Carve &cv, RadiusArgs &ra, int dtype, int64_t n, int d, int kc) {
    if (!tc_radius_wanted(dtype, n, d, kc)) {
        ra.tc_at = nullptr;
        return;
    }
    ra.tc_at = cv.take<char>(tc_point_bytes(n, d));
    ra.tc_an = cv.take<float>((size_t)tc_point_rows(n));
    ra.tc_ae = cv.take<float>((size_t)tc_point_rows(n));
    ra.tc_bt = cv.take<char>(tc_center_bytes(kc, d));
    ra.tc_cn = cv.take<float>((size_t)tc_center_tiles(kc) * 256);
    ra.tc_ce = cv.take<float>((size_t)tc_center_tiles(kc) * 256);
    ra.tc_maxes = cv.take<unsigned>(3);
    ra.tc_absmax = cv.take<unsigned>(3);   // scale words (the row-major path uses all three)
    ra.tc_mlo = cv.take<float>((size_t)n);
    ra.tc_mhi = cv.take<float>((size_t)n);
    ra.tc_mlomax = cv.take<unsigned>(1);
    ra.tc_flist = cv.take<uint32_t>((size_t)n);
    ra.tc_fcount = cv.take<unsigned long long>(1);
}

void copy_tc(RadiusArgs &dst, const RadiusArgs &src) {
    dst.tc_at = src.tc_at;
    dst.tc_bt = src.tc_bt;
    dst.tc_an = src.tc_an;
    dst.tc_ae = src.tc_ae;
    dst.tc_cn = src.tc_cn;
    dst.tc_ce = src.tc_ce;
    dst.tc_maxes = src.tc_maxes;
    dst.tc_absmax = src.tc_absmax;
    dst.tc_mlo = src.tc_mlo;
    dst.tc_mhi = src.tc_mhi;
    dst.tc_mlomax = src.tc_mlomax;
    dst.tc_flist = src.tc_flist;
    dst.tc_fcount = src.tc_fcount;
}

// Point an instance at the low-precision data (its own cenT [d][kcap] and
// ecmax slot).
void attach_lp(GonInst &I, const LPBufs &L, int lp, float *cenT, int kcap, float *ecmax) {
    I.lp = L.lp;
    I.eblk = L.eblk;
    I.ept = L.ept;
    I.scale = L.scale;
    I.cenT = cenT;
    I.kcap = kcap;
    I.ecmax_out = ecmax;
    I.m32 = L.m32;
    I.stamp = L.stamp;
    I.lp_kind = lp;
}

int choose_gon_grid(int dtype, int d, int64_t n, int lp = 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int maxg = gon_max_grid(dtype, d, lp);
    const int W = gon_warps_per_cta();
    const int64_t nb = nblocks(n);
    // Aim for about two 128-point blocks per warp; whole waves of SMs.
    int64_t want = (nb + 2 * W - 1) / (2 * W);
    int g;
    if (want >= sms) {
        int64_t per = (want + sms - 1) / sms;
        g = (int)(per * sms);
    } else {
        g = (int)(want < 1 ? 1 : want);
    }
    if (const char *env = getenv("KC_GON_GRID")) {
        int v = atoi(env);
        if (v > 0) g = v;
    }
    if (g > maxg) g = maxg;
    return g < 1 ? 1 : g;
}

}  // namespace

namespace kc {
void note_launches(int kernels) {
    g_launches += kernels;
    t_kernels += kernels;
}
void set_last_error(const char *text) { g_err = text ? text : ""; }

int device_clock_khz(int dev) {
    static std::atomic<int> cache[64];
    int khz = 0;
    if (dev < 0 || dev >= 64) {
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
        return khz;
    }
    khz = cache[dev].load(std::memory_order_relaxed);
    if (khz == 0) {
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
        if (khz <= 0) khz = -1;
        cache[dev].store(khz, std::memory_order_relaxed);
    }
    return khz;
}
}  // namespace kc

extern "C" {

const char *kc_version(void) { return "kcenter-gb300 0.1 (sm_103a)"; }

void kc_trace_enable(int32_t on) { g_trace_on = on ? 1 : 0; }

int32_t kc_counters(int64_t *out, int32_t cap) {
    unsigned long long v[15] = {0}, g[8] = {0, 0, 0, 0, 0, 0, 0, 0}, tc[6] = {0, 0, 0, 0, 0, 0};
    if (cudaDeviceSynchronize() != cudaSuccess || read_counters(g, true) != cudaSuccess ||
        read_tc_counters(tc, true) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    v[2] = tc[0];
    v[3] = tc[1];
    for (int i = 0; i < 4; ++i) v[11 + i] = tc[2 + i];
    v[0] = g[0];
    v[1] = g[1];
    v[4] = g_prune_pairs.exchange(0);
    v[5] = g[2];
    v[6] = g[3];
    v[7] = g[4];
    v[8] = g[5];
    v[9] = g[6];
    v[10] = g[7];
    for (int i = 0; i < cap && i < 15; ++i) out[i] = (int64_t)v[i];
    return 15;
}

int64_t kc_launch_count(void) { return g_launches.load(); }

int32_t kc_trace_read(kc_trace_rec *out, int32_t cap) {
    std::vector<TraceRec> recs;
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        recs.swap(g_trace);
    }
    int32_t i = 0;
    for (auto &r : recs) {
        float ms = 0.f;
        cudaEventSynchronize(r.b);
        cudaEventElapsedTime(&ms, r.a, r.b);
        if (out && i < cap) {
            memset(&out[i], 0, sizeof(kc_trace_rec));
            memcpy(out[i].name, r.name, sizeof out[i].name);
            out[i].kernels = r.kernels;
            out[i].ms = ms;
        }
        ++i;
    }
    std::lock_guard<std::mutex> lk(g_tmu);
    for (auto &r : recs) {
        g_evpool.push_back(r.a);
        g_evpool.push_back(r.b);
    }
    return (int32_t)recs.size();
}

const char *kc_last_error(void) { return g_err.c_str(); }

void kc_release(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : g_arenas) {
        cudaSetDevice(kv.first.first);
        Arena *a = kv.second;
        a->last_key32 = nullptr;
        if (a->dev) cudaFree(a->dev);
        if (a->status) cudaFree(a->status);
        if (a->host_status) cudaFreeHost(a->host_status);
        if (a->pinned_busy) cudaEventSynchronize(a->pinned_ev);
        if (a->pinned) cudaFreeHost(a->pinned);
        if (a->pinned_ev) cudaEventDestroy(a->pinned_ev);
        delete a;
    }
    g_arenas.clear();
    cudaSetDevice(cur);
}

kc_status kc_last_fp32_radius(void *stream, double *radius32) {
    g_err.clear();
    if (!radius32) return fail(KC_ERR_ARG, "null pointer argument");
    Arena *a = nullptr;
    kc_status r = arena_for((cudaStream_t)stream, &a);
    if (r != KC_OK) return r;
    if (!a->last_key32) return fail(KC_ERR_ARG, "no solve or radius has run on this stream");
    unsigned long long key = 0;
    KC_CUDA(cudaMemcpyAsync(&key, a->last_key32, sizeof key, cudaMemcpyDeviceToHost, (cudaStream_t)stream),
            "key read-back");
    KC_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize");
    const uint32_t v = (uint32_t)(key >> 32);
    if (a->last_dtype == KC_I32) {
        *radius32 = std::sqrt((double)v);
    } else {
        float f;
        memcpy(&f, &v, sizeof f);
        *radius32 = std::sqrt((double)f);
    }
    return KC_OK;
}

kc_status kc_sync(void *stream) {
    Arena *a = nullptr;
    kc_status r = arena_for((cudaStream_t)stream, &a);
    if (r != KC_OK) return r;
    return finish(a, (cudaStream_t)stream);
}

kc_status kc_gonzalez(const void *pts, int64_t n, int32_t d, int32_t k, int64_t first,
                      int64_t *centers, int32_t *k_out, double *radius, const kc_opts *opts) {
    g_err.clear();
    if (!pts || !centers || !k_out || !radius) return fail(KC_ERR_ARG, "null pointer argument");
    if (n < 1 || n > (int64_t)N_MAX) return fail(KC_ERR_ARG, "n=%lld outside [1, 2^32-2]", (long long)n);
    if (d < 1) return fail(KC_ERR_ARG, "d=%d must be >= 1", d);
    if (k < 1) return fail(KC_ERR_ARG, "k=%d must be >= 1", k);
    if (first < 0 || first >= n) return fail(KC_ERR_ARG, "first=%lld outside [0, n)", (long long)first);
    CallCtx c;
#ifdef KC_CHECKS
    kc_status r = begin(opts, c, KC_ASYNC | KC_TEST_WITHHOLD | KC_TEST_BAD_INDEX);
#else
    kc_status r = begin(opts, c, KC_ASYNC | KC_TEST_WITHHOLD);
#endif
    if (r != KC_OK) return r;
    const bool bad_index = (c.o.flags & KC_TEST_BAD_INDEX) != 0;

    const bool dev_pts = is_device_ptr(pts, c.dev);
    const void *pin_pts = dev_pts ? nullptr : pinned_device_ptr(pts);   // read in place by the pack
    const bool dev_cen = is_device_ptr(centers, c.dev);
    const bool dev_kout = is_device_ptr(k_out, c.dev);
    const bool dev_rad = is_device_ptr(radius, c.dev);
    if (c.async && !(dev_pts && dev_cen && dev_kout && dev_rad))
        return fail(KC_ERR_ARG, "KC_ASYNC needs device pointers for all arguments");

    const int keff = (int)(k < n ? k : n);
    const int lp = lp_of(c.o);
    // points that fit on chip: the resident kernel reads the rows in place
    // (device memory or the staging copy) and keeps them for all k steps
    int res_cap = 0, res_sw = 0;
    const int res_grid = (!lp && !pin_pts && !bad_index) ? gon_resident_plan(c.o.dtype, d, n, &res_cap, &res_sw) : 0;
    const int grid = res_grid ? res_grid : choose_gon_grid(c.o.dtype, d, n, lp);
    // the FP32 streaming group shares the last blocks of every step between its
    // CTAs when every warp has at least two whole rounds of its own before the
    // tail (tail_start; KC_GON_TAIL=0 keeps every block with its CTA)
    const bool dyn = !lp && !res_grid && c.o.dtype == KC_F32 &&
                     nblocks(n) >= 4 * (int64_t)grid * gon_warps_per_cta();   // claimed blocks pay off
    bool use_tail = dyn && grid > 1 && nblocks(n) * 7 / 8 / ((int64_t)grid * gon_warps_per_cta()) >= 2;
    if (const char *env = getenv("KC_GON_TAIL")) use_tail = use_tail && atoi(env) != 0;
    const int64_t nb = nblocks(n);
    const size_t esz = 4;
    LPBufs LB;
    float *cenT = nullptr, *ecmax = nullptr;

    auto layout = [&](Carve &cv, GonArgs &g, RadiusArgs &ra, void **staging, int64_t **cen_dev,
                      int32_t **kout_dev, double **rad_dev, size_t *zero_bytes) {
        // zero-initialised region first
        int32_t *range2 = cv.take<int32_t>(2);
        unsigned long long *key32 = cv.take<unsigned long long>(1);
        unsigned long long *max64 = cv.take<unsigned long long>(1);
        unsigned long long *arg64 = cv.take<unsigned long long>(1);
        // per (step, CTA): argmax keys, and for the mixed-precision sweep the
        // CTAs' lower bounds too
        uint64_t *slots = cv.take<uint64_t>(res_grid ? (size_t)keff * grid * res_sw
                                                      : (size_t)slot_words(keff, grid, lp != 0));
        int *tail = use_tail ? cv.take<int>((size_t)keff) : nullptr;
        unsigned *flag_words = c.o.dtype == KC_F32 ? cv.take<unsigned>(2) : nullptr;   // flagged count, done
        *zero_bytes = cv.off;
        *staging = (dev_pts || pin_pts) ? nullptr : cv.take<char>((size_t)n * d * esz);
        void *pk = res_grid ? nullptr : cv.take<char>((size_t)nb * BLK * d * esz);
        uint32_t *mind = cv.take<uint32_t>((size_t)nb * BLK);
        void *cen = cv.take<char>((size_t)keff * d * esz);
        double *m64 = cv.take<double>(c.o.dtype == KC_F32 ? (size_t)n : 1);
        *cen_dev = dev_cen ? centers : cv.take<int64_t>(keff);
        *kout_dev = dev_kout ? k_out : cv.take<int32_t>(1);
        *rad_dev = dev_rad ? radius : cv.take<double>(1);
        take_lp(cv, LB, lp, n, d);
        cenT = lp ? cv.take<float>((size_t)keff * d) : nullptr;
        ecmax = lp ? cv.take<float>(1) : nullptr;
        gon_single(g, pk, c.o.dtype, n, d, keff, first, mind, slots, *cen_dev, *kout_dev,
                   (uint64_t *)key32, range2, grid);
        g.single.tail = tail;
        if (lp) {
            attach_lp(g.single, LB, lp, cenT, keff, ecmax);
            g.lp_kind = lp;
            g.lp_local_t = lp_local_t(lp);
            ra.eblk = LB.eblk;
            ra.ecmax = ecmax;
            ra.lpscale = lp == KC_SWEEP_FP16 ? LB.scale : nullptr;
        }
        ra.pk = pk;
        ra.dtype = c.o.dtype;
        ra.n = n;
        ra.d = d;
        ra.centers = *cen_dev;
        ra.kc_dev = *kout_dev;
        ra.kc_max = keff;
        ra.cen = cen;
        ra.mind = mind;
        ra.key32 = key32;
        ra.max64 = max64;
        ra.arg64 = arg64;
        ra.m64 = m64;
        ra.radius_out = *rad_dev;
        ra.argmax_out = nullptr;
        ra.have_mind = true;
        if (flag_words) {
            ra.flagged = cv.take<uint32_t>((size_t)n);
            ra.flagged_n = flag_words;
            ra.done = flag_words + 1;
        }
    };

    GonArgs g{};
    RadiusArgs ra{};
    void *staging;
    int64_t *cen_dev;
    int32_t *kout_dev;
    double *rad_dev;
    size_t zero_bytes;
    {
        Carve sizing(nullptr);
        layout(sizing, g, ra, &staging, &cen_dev, &kout_dev, &rad_dev, &zero_bytes);
        r = arena_reserve(c.arena, sizing.off, c.s);
        if (r != KC_OK) return r;
    }
    Carve cv(c.arena->dev);
    layout(cv, g, ra, &staging, &cen_dev, &kout_dev, &rad_dev, &zero_bytes);
    g.st = c.arena->status;
    ra.st = c.arena->status;
    g.timeout_cycles = timeout_cycles(c.o);
    g.withhold = (c.o.flags & KC_TEST_WITHHOLD) ? 1 : 0;
    g.bad_index = bad_index ? 1 : 0;
    g.dyn = dyn ? 1 : 0;
    c.arena->last_key32 = ra.key32;
    c.arena->last_dtype = c.o.dtype;

    KC_CUDA(cudaMemsetAsync(c.arena->dev, 0, zero_bytes, c.s), "scratch clear");
    const void *src;
    r = stage_points(c, pts, (size_t)n * d * esz, dev_pts, staging, &src, pin_pts);
    if (r != KC_OK) return r;
    // exact rechecks read the FP32 rows where they are in device memory
    if (lp && !pin_pts) g.single.rm = (const float *)src;
    if (res_grid) {
        // the resident kernel reads (and checks) the rows itself: no pack
        g.single.pk = src;
        g.res_cap = res_cap;
        ra.pk = nullptr;
        ra.rm = (const float *)src;
    } else {
        TraceStep t("pack", c.s);
        KC_CUDA(launch_pack(src, c.o.dtype, n, d, (void *)g.single.pk, (int32_t *)g.single.range2,
                            c.arena->status, c.s),
                "pack launch");
        if (lp)
            KC_CUDA(launch_lp_pack(lp, (const float *)g.single.pk, n, d, LB.colmax, LB.scale, LB.lp, LB.ept,
                                   LB.eblk, LB.stamp, c.s),
                    "low-precision pack");
    }
    {
        TraceStep t("gonzalez", c.s);
        KC_CUDA(launch_gon(g, c.s), "gonzalez launch");
        if (res_grid && c.o.dtype == KC_I32)
            KC_CUDA(launch_range_check(g.single.range2, d, c.arena->status, c.s), "range check");
    }
    {
        TraceStep t("radius_recheck", c.s);
        KC_CUDA(launch_radius(ra, c.s), "radius launch");
    }

    if (!dev_cen)
        KC_CUDA(cudaMemcpyAsync(centers, cen_dev, (size_t)keff * sizeof(int64_t), cudaMemcpyDeviceToHost, c.s),
                "copy centers out");
    if (!dev_kout)
        KC_CUDA(cudaMemcpyAsync(k_out, kout_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, c.s), "copy k_out");
    if (!dev_rad)
        KC_CUDA(cudaMemcpyAsync(radius, rad_dev, sizeof(double), cudaMemcpyDeviceToHost, c.s), "copy radius");
    if (c.async) return KC_OK;
    return finish(c.arena, c.s);
}

kc_status kc_radius(const void *pts, int64_t n, int32_t d, const int64_t *centers, int32_t kc,
                    double *radius, int64_t *argmax_point, const kc_opts *opts) {
    g_err.clear();
    if (!pts || !centers || !radius) return fail(KC_ERR_ARG, "null pointer argument");
    if (n < 1 || n > (int64_t)N_MAX) return fail(KC_ERR_ARG, "n=%lld outside [1, 2^32-2]", (long long)n);
    if (d < 1) return fail(KC_ERR_ARG, "d=%d must be >= 1", d);
    if (kc < 1) return fail(KC_ERR_ARG, "kc=%d must be >= 1", kc);
    CallCtx c;
    kc_status r = begin(opts, c);
    if (r != KC_OK) return r;

    // On the tensor-core path, and for float points with d <= 16 on the CUDA
    // cores, the row-major points are read where they are (device memory,
    // else a device copy): no pack.  Otherwise the pack reads pinned host
    // memory in place.
    const bool rowmajor = tc_radius_wanted(c.o.dtype, n, d, kc) || (c.o.dtype == KC_F32 && d <= 16);
    const bool dev_pts = is_device_ptr(pts, c.dev);
    const void *pin_pts = (dev_pts || rowmajor) ? nullptr : pinned_device_ptr(pts);
    const bool dev_cin = is_device_ptr(centers, c.dev);
    const bool dev_rad = is_device_ptr(radius, c.dev);
    const bool dev_arg = argmax_point ? is_device_ptr(argmax_point, c.dev) : true;
    if (c.async && !(dev_pts && dev_cin && dev_rad && dev_arg))
        return fail(KC_ERR_ARG, "KC_ASYNC needs device pointers for all arguments");
    if (!dev_cin) {
        for (int32_t i = 0; i < kc; ++i)
            if (centers[i] < 0 || centers[i] >= n)
                return fail(KC_ERR_ARG, "center %d index %lld outside [0, n)", i, (long long)centers[i]);
    }
    const int64_t nb = nblocks(n);
    const size_t esz = 4;

    RadiusArgs ra{};
    void *staging = nullptr;
    const int64_t *cin_dev = nullptr;
    double *rad_dev = nullptr;
    int64_t *arg_dev = nullptr;
    size_t zero_bytes = 0;
    auto layout = [&](Carve &cv) {
        int32_t *range2 = cv.take<int32_t>(2);
        (void)range2;
        ra.key32 = cv.take<unsigned long long>(1);
        ra.max64 = cv.take<unsigned long long>(1);
        ra.arg64 = cv.take<unsigned long long>(1);
        unsigned *flag_words = c.o.dtype == KC_F32 ? cv.take<unsigned>(2) : nullptr;   // flagged count, done
        zero_bytes = cv.off;
        if (flag_words) {
            ra.flagged_n = flag_words;
            ra.done = flag_words + 1;
            ra.flagged = cv.take<uint32_t>((size_t)n);
        }
        staging = (dev_pts || pin_pts) ? nullptr : cv.take<char>((size_t)n * d * esz);
        ra.pk = rowmajor ? nullptr : cv.take<char>((size_t)nb * BLK * d * esz);
        ra.mind = cv.take<uint32_t>((size_t)nb * BLK);
        ra.cen = cv.take<char>((size_t)kc * d * esz);
        ra.m64 = cv.take<double>(c.o.dtype == KC_F32 ? (size_t)n : 1);
        cin_dev = dev_cin ? centers : cv.take<int64_t>(kc);
        rad_dev = dev_rad ? radius : cv.take<double>(1);
        arg_dev = (argmax_point && dev_arg) ? argmax_point : cv.take<int64_t>(1);
        take_tc(cv, ra, c.o.dtype, n, d, kc);
    };
    {
        Carve sizing(nullptr);
        layout(sizing);
        r = arena_reserve(c.arena, sizing.off, c.s);
        if (r != KC_OK) return r;
    }
    Carve cv(c.arena->dev);
    layout(cv);
    int32_t *range2 = reinterpret_cast<int32_t *>(c.arena->dev);
    ra.dtype = c.o.dtype;
    ra.n = n;
    ra.d = d;
    ra.centers = cin_dev;
    ra.kc_dev = nullptr;
    ra.kc_max = kc;
    ra.radius_out = rad_dev;
    ra.argmax_out = arg_dev;
    ra.st = c.arena->status;
    ra.have_mind = false;
    c.arena->last_key32 = ra.key32;
    c.arena->last_dtype = c.o.dtype;

    KC_CUDA(cudaMemsetAsync(c.arena->dev, 0, zero_bytes, c.s), "scratch clear");
    const void *src;
    r = stage_points(c, pts, (size_t)n * d * esz, dev_pts, staging, &src, pin_pts);
    if (r != KC_OK) return r;
    if (!dev_cin)
        KC_CUDA(cudaMemcpyAsync((void *)cin_dev, centers, (size_t)kc * sizeof(int64_t), cudaMemcpyHostToDevice, c.s),
                "copy centers in");
    if (rowmajor) {
        ra.rm = (const float *)src;   // checked by the tensor-core prep or the minimum kernel
    } else {
        TraceStep t("pack", c.s);
        KC_CUDA(launch_pack(src, c.o.dtype, n, d, (void *)ra.pk, range2, c.arena->status, c.s), "pack launch");
        if (c.o.dtype == KC_I32) KC_CUDA(launch_range_check(range2, d, c.arena->status, c.s), "range check");
    }
    {
        TraceStep t("radius", c.s);
        KC_CUDA(launch_radius(ra, c.s), "radius launch");
    }
    if (!dev_rad)
        KC_CUDA(cudaMemcpyAsync(radius, rad_dev, sizeof(double), cudaMemcpyDeviceToHost, c.s), "copy radius");
    if (argmax_point && !dev_arg)
        KC_CUDA(cudaMemcpyAsync(argmax_point, arg_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, c.s),
                "copy argmax");
    if (c.async) return KC_OK;
    return finish(c.arena, c.s);
}

}  // extern "C"

namespace {

// CTA groups for parts of sizes sz (k centers each, at most sz):
// proportional to each part's work n_i k_i, at least one CTA, at most one
// per W blocks (one block per warp), within maxg co-resident CTAs.  queue:
// more parts than CTAs, one CTA per part from a queue.  The parts run on the
// queue kernel's 256-thread CTAs (four per SM) with every part a group
// ("heavy"): the finer CTA granularity balances uneven parts (Zipf round 1
// on 10M x 16: 0.83 -> 1.00 of HBM against one 1024-thread CTA per SM).
void mrg_groups(const std::vector<int64_t> &sz, int k, int maxg, int W, std::vector<int> &G, bool &queue) {
    const int m = (int)sz.size();
    G.assign((size_t)m, 1);
    queue = m > maxg;
    if (queue) return;
    double tot = 0;
    std::vector<double> work((size_t)m);
    for (int i = 0; i < m; ++i) {
        work[i] = (double)sz[i] * (double)std::min<int64_t>(k, sz[i]);
        tot += work[i];
    }
    std::vector<int> cap((size_t)m);
    int sum = 0;
    for (int i = 0; i < m; ++i) {
        const int64_t nbi = nblocks(sz[i]) + 1;
        cap[i] = (int)std::max<int64_t>(1, (nbi + W - 1) / W);
        G[i] = (int)std::max(1.0, std::floor(maxg * work[i] / tot));
        G[i] = std::min(G[i], cap[i]);
        sum += G[i];
    }
    while (sum > maxg) {   // trim the largest groups
        int j = 0;
        for (int i = 1; i < m; ++i) if (G[i] > G[j]) j = i;
        if (G[j] <= 1) break;
        --G[j];
        --sum;
    }
    while (sum < maxg) {   // hand out the rest to the most loaded CTAs
        int j = -1;
        double best = 0;
        for (int i = 0; i < m; ++i)
            if (G[i] < cap[i] && work[i] / G[i] > best) {
                best = work[i] / G[i];
                j = i;
            }
        if (j < 0) break;
        ++G[j];
        ++sum;
    }
}

// MRG, Algorithm 1: round 1 on the m parts; while the union holds more than
// capacity points (capacity < m k), further rounds on ceil(|S| / capacity)
// contiguous parts of the ascending union (host loop); then GON on the
// union.  rounds_out (host, may be null) gets the number of rounds.
kc_status mrg_run(const void *pts, int64_t n, int32_t d, int32_t k, int32_t m, const int64_t *offsets,
                  int64_t capacity, int64_t *centers, int32_t *k_out, double *radius, int32_t *rounds_out,
                  const kc_opts *opts) {
    g_err.clear();
    if (!pts || !centers || !k_out || !radius) return fail(KC_ERR_ARG, "null pointer argument");
    if (n < 1 || n > (int64_t)N_MAX) return fail(KC_ERR_ARG, "n=%lld outside [1, 2^32-2]", (long long)n);
    if (d < 1) return fail(KC_ERR_ARG, "d=%d must be >= 1", d);
    if (k < 1) return fail(KC_ERR_ARG, "k=%d must be >= 1", k);
    if (m < 1 || m > n) return fail(KC_ERR_ARG, "m=%d must be in [1, n]", m);
    if (capacity < 2 * (int64_t)k)
        return fail(KC_ERR_ARG, "capacity=%lld must be at least 2k=%lld", (long long)capacity, 2 * (long long)k);
    const bool multi = capacity < (int64_t)m * k;
    CallCtx c;
    kc_status r = begin(opts, c);
    if (r != KC_OK) return r;
    if (multi && c.async) return fail(KC_ERR_ARG, "more than two rounds run a host loop and do not take KC_ASYNC");
    const bool dev_pts = is_device_ptr(pts, c.dev);
    const void *pin_pts = dev_pts ? nullptr : pinned_device_ptr(pts);   // read in place by the pack
    const bool dev_cen = is_device_ptr(centers, c.dev);
    const bool dev_kout = is_device_ptr(k_out, c.dev);
    const bool dev_rad = is_device_ptr(radius, c.dev);
    if (c.async && !(dev_pts && dev_cen && dev_kout && dev_rad && (!offsets || is_device_ptr(offsets, c.dev))))
        return fail(KC_ERR_ARG, "KC_ASYNC needs device pointers for all arguments");

    // Parts: the given offsets, else the balanced split off[i] = floor(i n / m)
    // (every part has at most ceil(n/m) points, Algorithm 1).
    std::vector<int64_t> off((size_t)m + 1);
    if (offsets) {
        if (is_device_ptr(offsets, c.dev)) {
            KC_CUDA(cudaMemcpyAsync(off.data(), offsets, off.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, c.s),
                    "copy offsets");
            KC_CUDA(cudaStreamSynchronize(c.s), "cudaStreamSynchronize");
        } else {
            memcpy(off.data(), offsets, off.size() * sizeof(int64_t));
        }
    } else {
        for (int i = 0; i <= m; ++i) off[i] = (int64_t)((__int128)i * n / m);
    }
    if (off[0] != 0 || off[m] != n) return fail(KC_ERR_ARG, "offsets must start at 0 and end at n");
    for (int i = 0; i < m; ++i)
        if (off[i + 1] <= off[i]) return fail(KC_ERR_ARG, "part %d is empty or offsets decrease", i);

    // Round-1 CTA groups on the queue kernel's CTAs (mrg_groups).
    const int lp = lp_of(c.o);
    const int maxg = gon_max_grid(c.o.dtype, d, lp);
    const int qslots0 = gon_queue_grid(c.o.dtype, d, 0);   // later rounds sweep in FP32
    const int W = gon_warps_per_cta();
    std::vector<int> G, ki((size_t)m);
    std::vector<int64_t> slot_off((size_t)m + 1, 0), sz1((size_t)m);
    bool queue1 = false;
    for (int i = 0; i < m; ++i) {
        sz1[i] = off[i + 1] - off[i];
        ki[i] = (int)std::min<int64_t>(k, sz1[i]);
    }
    const int qslots = gon_queue_grid(c.o.dtype, d, lp), Wq = gon_queue_warps();
    mrg_groups(sz1, k, qslots, Wq, G, queue1);
    for (int i = 0; i < m; ++i)
        slot_off[i + 1] = slot_off[i] + (queue1 ? 0 : slot_words(ki[i], G[i], lp != 0));
    int grid1 = 0;
    for (int i = 0; i < m; ++i) grid1 += G[i];
    if (queue1) grid1 = qslots;
    std::vector<int64_t> cen_off((size_t)m + 1, 0);
    for (int i = 0; i < m; ++i) cen_off[i + 1] = cen_off[i] + ki[i];
    LPBufs LB;
    float *cenT1 = nullptr, *ecmax1 = nullptr;
    RadiusArgs Rtc{};
    const int64_t ucap = (int64_t)m * k;
    const int G2 = (int)std::min<int64_t>(std::max<int64_t>(1, (nblocks(ucap) + W - 1) / W), std::min(maxg, 16));
    const int64_t nb = nblocks(n);
    const size_t esz = 4;

    struct L {
        int32_t *range2;
        unsigned long long *key32, *max64, *arg64;
        uint64_t *slots1, *slots2, *fk2;
        int64_t *nU;
        int *counter;
        void *staging, *pk, *pkU, *cen;
        uint32_t *mind, *mindU;
        int64_t *c1, *U, *U2;
        void *pkU2;
        uint64_t *slotsR;
        int32_t *k1;
        uint64_t *fk1;
        GonInst *insts1, *inst2;
        double *m64;
        int64_t *cen_dev;
        int32_t *kout_dev;
        double *rad_dev;
        size_t zero_bytes;
    } Lo{};
    auto layout = [&](Carve &cv) {
        Lo.range2 = cv.take<int32_t>(2);
        Lo.key32 = cv.take<unsigned long long>(1);
        Lo.max64 = cv.take<unsigned long long>(1);
        Lo.arg64 = cv.take<unsigned long long>(1);
        Lo.fk2 = cv.take<uint64_t>(1);
        Lo.nU = cv.take<int64_t>(1);
        Lo.counter = cv.take<int>(1);
        Lo.slots1 = cv.take<uint64_t>((size_t)std::max<int64_t>(1, slot_off[m]));
        Lo.slots2 = cv.take<uint64_t>((size_t)slot_words(k, G2, false));
        Lo.zero_bytes = cv.off;
        Lo.staging = (dev_pts || pin_pts) ? nullptr : cv.take<char>((size_t)n * d * esz);
        Lo.pk = cv.take<char>((size_t)nb * BLK * d * esz);
        Lo.mind = cv.take<uint32_t>((size_t)nb * BLK);
        Lo.c1 = cv.take<int64_t>((size_t)ucap);
        Lo.k1 = cv.take<int32_t>((size_t)m);
        Lo.fk1 = cv.take<uint64_t>((size_t)m);
        Lo.U = cv.take<int64_t>((size_t)ucap);
        Lo.pkU = cv.take<char>((size_t)nblocks(ucap) * BLK * d * esz);
        Lo.mindU = cv.take<uint32_t>((size_t)nblocks(ucap) * BLK);
        Lo.insts1 = cv.take<GonInst>((size_t)m);
        take_lp(cv, LB, lp, n, d);
        cenT1 = lp ? cv.take<float>((size_t)cen_off[m] * d) : nullptr;
        ecmax1 = lp ? cv.take<float>((size_t)m) : nullptr;
        take_tc(cv, Rtc, c.o.dtype, n, d, k);
        Lo.inst2 = cv.take<GonInst>(1);
        if (multi) {   // later rounds: the other union buffers and per-round slots
            Lo.U2 = cv.take<int64_t>((size_t)ucap);
            Lo.pkU2 = cv.take<char>((size_t)nblocks(ucap) * BLK * d * esz);
            Lo.slotsR = cv.take<uint64_t>((size_t)k * std::max(1, qslots0));
        }
        Lo.cen = cv.take<char>((size_t)k * d * esz);
        Lo.m64 = cv.take<double>(c.o.dtype == KC_F32 ? (size_t)n : 1);
        Lo.cen_dev = dev_cen ? centers : cv.take<int64_t>((size_t)k);
        Lo.kout_dev = dev_kout ? k_out : cv.take<int32_t>(1);
        Lo.rad_dev = dev_rad ? radius : cv.take<double>(1);
    };
    {
        Carve sizing(nullptr);
        layout(sizing);
        r = arena_reserve(c.arena, sizing.off, c.s);
        if (r != KC_OK) return r;
    }
    Carve cv(c.arena->dev);
    layout(cv);
    DevStatus *st = c.arena->status;
    c.arena->last_key32 = Lo.key32;
    c.arena->last_dtype = c.o.dtype;

    // Round-1 descriptors (host-built, uploaded once).
    std::vector<GonInst> h1((size_t)m);
    {
        int cta = 0;
        for (int i = 0; i < m; ++i) {
            GonInst &I = h1[i];
            memset(&I, 0, sizeof I);
            I.pk = Lo.pk;
            I.mind = Lo.mind;
            I.slots = Lo.slots1 + slot_off[i];
            I.centers = Lo.c1 + (int64_t)i * k;
            I.k_out = Lo.k1 + i;
            I.final_key = Lo.fk1 + i;
            I.map = nullptr;
            I.range2 = Lo.range2;
            I.radius_out = nullptr;
            I.lo = off[i];
            I.n = off[i + 1] - off[i];
            I.base = off[i];
            I.first = 0;
            I.d = d;
            I.k = ki[i];
            I.cta0 = queue1 ? 0 : cta;
            I.G = queue1 ? 1 : G[i];
            I.kcap = ki[i];
            if (lp) attach_lp(I, LB, lp, cenT1 + cen_off[i] * d, ki[i], ecmax1 + i);
            cta += I.G;
        }
    }
    GonInst proto;
    memset(&proto, 0, sizeof proto);
    proto.pk = Lo.pkU;
    proto.mind = Lo.mindU;
    proto.slots = Lo.slots2;
    proto.centers = Lo.cen_dev;
    proto.k_out = Lo.kout_dev;
    proto.final_key = Lo.fk2;
    proto.map = Lo.U;
    proto.range2 = Lo.range2;
    proto.d = d;
    proto.cta0 = 0;
    proto.G = G2;

    KC_CUDA(cudaMemsetAsync(c.arena->dev, 0, Lo.zero_bytes, c.s), "scratch clear");
    const void *src;
    r = stage_points(c, pts, (size_t)n * d * esz, dev_pts, Lo.staging, &src, pin_pts);
    if (r != KC_OK) return r;
    if (lp && !pin_pts)
        for (int i = 0; i < m; ++i) h1[i].rm = (const float *)src + off[i] * d;
    r = upload(c.arena, c.s, h1.data(), h1.size() * sizeof(GonInst), Lo.insts1);
    if (r != KC_OK) return r;
    const long long tmo = timeout_cycles(c.o);
    {
        TraceStep t("pack", c.s);
        KC_CUDA(launch_pack(src, c.o.dtype, n, d, Lo.pk, Lo.range2, st, c.s), "pack launch");
        if (lp)
            KC_CUDA(launch_lp_pack(lp, (const float *)Lo.pk, n, d, LB.colmax, LB.scale, LB.lp, LB.ept, LB.eblk,
                                   LB.stamp, c.s),
                    "low-precision pack");
    }
    {
        TraceStep t("mrg_round1", c.s);
        GonArgs g{};
        g.insts = Lo.insts1;
        g.ninst = m;
        g.dtype = c.o.dtype;
        g.dc = d;
        g.dmax = d;
        g.st = st;
        g.timeout_cycles = tmo;
        g.grid = grid1;
        g.counter = Lo.counter;
        g.lp_kind = lp;
        g.lp_local_t = lp_local_t(lp);
        g.queue = 1;   // queue kernel: every part a CTA group, or one CTA per part from the queue
        if (!queue1) {
            g.nheavy = m;
            g.gheavy = grid1;
        }
        KC_CUDA(launch_gon(g, c.s), "mrg round 1 launch");
    }
    {
        TraceStep t("mrg_union", c.s);
        KC_CUDA(launch_mrg_union(Lo.c1, Lo.k1, m, k, Lo.U, Lo.nU, c.s), "union launch");
        KC_CUDA(launch_gather_pack(Lo.pk, c.o.dtype, d, Lo.U, Lo.nU, ucap, Lo.pkU, c.s), "gather launch");
    }
    int rounds = 1;
    if (multi) {
        // Further rounds while the union exceeds the capacity: parts are
        // contiguous ranges of the ascending union (part i: positions
        // [floor(i |S| / m'), floor((i + 1) |S| / m'))), solved with the FP32
        // sweep on the gathered copy, their centers mapped back to global
        // indices, united and gathered again.
        int64_t *Ucur = Lo.U, *Unext = Lo.U2;
        void *pkcur = Lo.pkU, *pknext = Lo.pkU2;
        for (;;) {
            int64_t nU = 0;
            KC_CUDA(cudaMemcpyAsync(&nU, Lo.nU, sizeof nU, cudaMemcpyDeviceToHost, c.s), "count read-back");
            KC_CUDA(cudaStreamSynchronize(c.s), "cudaStreamSynchronize");
            {
                DevStatus h;
                KC_CUDA(cudaMemcpy(&h, st, sizeof h, cudaMemcpyDeviceToHost), "status read-back");
                if (h.code != 0) return finish(c.arena, c.s);
            }
            if (nU <= capacity) break;
            if (rounds >= 64) return fail(KC_ERR_ARG, "MRG did not fit the capacity within 64 rounds");
            const int mp = (int)((nU + capacity - 1) / capacity);
            std::vector<int64_t> offr((size_t)mp + 1), szr((size_t)mp);
            for (int i = 0; i <= mp; ++i) offr[i] = (int64_t)((__int128)i * nU / mp);
            for (int i = 0; i < mp; ++i) szr[i] = offr[i + 1] - offr[i];
            std::vector<int> Gr;
            bool queuer = false;
            mrg_groups(szr, k, qslots0, Wq, Gr, queuer);
            std::vector<GonInst> hr((size_t)mp);
            int64_t soff = 0;
            int cta = 0;
            for (int i = 0; i < mp; ++i) {
                GonInst &I = hr[i];
                memset(&I, 0, sizeof I);
                const int kr = (int)std::min<int64_t>(k, szr[i]);
                I.pk = pkcur;
                I.mind = Lo.mindU;
                I.slots = queuer ? nullptr : Lo.slotsR + soff;
                I.centers = Lo.c1 + (int64_t)i * k;
                I.k_out = Lo.k1 + i;
                I.final_key = Lo.fk1 + i;
                I.map = Ucur + offr[i];
                I.range2 = Lo.range2;
                I.lo = offr[i];
                I.n = szr[i];
                I.first = 0;
                I.d = d;
                I.k = kr;
                I.cta0 = queuer ? 0 : cta;
                I.G = queuer ? 1 : Gr[i];
                I.kcap = kr;
                cta += I.G;
                soff += queuer ? 0 : slot_words(kr, Gr[i], false);
            }
            KC_CUDA(cudaMemsetAsync(Lo.slotsR, 0, (size_t)std::max<int64_t>(1, soff) * sizeof(uint64_t), c.s),
                    "slot clear");
            KC_CUDA(cudaMemsetAsync(Lo.counter, 0, sizeof(int), c.s), "counter clear");
            if ((r = upload(c.arena, c.s, hr.data(), hr.size() * sizeof(GonInst), Lo.insts1)) != KC_OK) return r;
            {
                TraceStep t("mrg_roundk", c.s);
                GonArgs g{};
                g.insts = Lo.insts1;
                g.ninst = mp;
                g.dtype = c.o.dtype;
                g.dc = d;
                g.dmax = d;
                g.st = st;
                g.timeout_cycles = tmo;
                g.grid = queuer ? qslots0 : cta;
                g.queue = 1;
                if (!queuer) {
                    g.nheavy = mp;
                    g.gheavy = cta;
                }
                g.counter = Lo.counter;
                KC_CUDA(launch_gon(g, c.s), "mrg round launch");
                KC_CUDA(launch_mrg_union(Lo.c1, Lo.k1, mp, k, Unext, Lo.nU, c.s), "union launch");
                KC_CUDA(launch_gather_pack(Lo.pk, c.o.dtype, d, Unext, Lo.nU, ucap, pknext, c.s), "gather launch");
            }
            std::swap(Ucur, Unext);
            std::swap(pkcur, pknext);
            ++rounds;
        }
        proto.pk = pkcur;
        proto.map = Ucur;
    }
    KC_CUDA(launch_mrg_round2_prep(Lo.inst2, proto, Lo.nU, k, c.s), "final round prep");
    {
        TraceStep t("mrg_round2", c.s);
        GonArgs g{};
        g.insts = Lo.inst2;
        g.ninst = 1;
        g.dtype = c.o.dtype;
        g.dc = d;
        g.dmax = d;
        g.st = st;
        g.timeout_cycles = tmo;
        g.grid = G2;
        KC_CUDA(launch_gon(g, c.s), "mrg round 2 launch");
    }
    ++rounds;
    if (rounds_out) *rounds_out = rounds;
    {
        TraceStep t("radius", c.s);
        RadiusArgs ra{};
        ra.pk = Lo.pk;
        ra.dtype = c.o.dtype;
        ra.n = n;
        ra.d = d;
        ra.centers = Lo.cen_dev;
        ra.kc_dev = Lo.kout_dev;
        ra.kc_max = k;
        ra.cen = Lo.cen;
        ra.mind = Lo.mind;
        ra.key32 = Lo.key32;
        ra.max64 = Lo.max64;
        ra.arg64 = Lo.arg64;
        ra.m64 = Lo.m64;
        ra.radius_out = Lo.rad_dev;
        ra.argmax_out = nullptr;
        ra.st = st;
        ra.have_mind = false;
        copy_tc(ra, Rtc);
        KC_CUDA(launch_radius(ra, c.s), "radius launch");
    }
    if (!dev_cen)
        KC_CUDA(cudaMemcpyAsync(centers, Lo.cen_dev, (size_t)k * sizeof(int64_t), cudaMemcpyDeviceToHost, c.s),
                "copy centers out");
    if (!dev_kout)
        KC_CUDA(cudaMemcpyAsync(k_out, Lo.kout_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, c.s), "copy k_out");
    if (!dev_rad)
        KC_CUDA(cudaMemcpyAsync(radius, Lo.rad_dev, sizeof(double), cudaMemcpyDeviceToHost, c.s), "copy radius");
    if (c.async) return KC_OK;
    return finish(c.arena, c.s);
}

}  // namespace

extern "C" {

kc_status kc_mrg(const void *pts, int64_t n, int32_t d, int32_t k, int32_t m, const int64_t *offsets,
                 int64_t *centers, int32_t *k_out, double *radius, const kc_opts *opts) {
    return mrg_run(pts, n, d, k, m, offsets, INT64_MAX, centers, k_out, radius, nullptr, opts);
}

kc_status kc_mrg_rounds(const void *pts, int64_t n, int32_t d, int32_t k, int32_t m, const int64_t *offsets,
                        int64_t capacity, int64_t *centers, int32_t *k_out, double *radius, int32_t *rounds,
                        const kc_opts *opts) {
    return mrg_run(pts, n, d, k, m, offsets, capacity, centers, k_out, radius, rounds, opts);
}

kc_status kc_eim(const void *pts, int64_t n, int32_t d, int32_t k, double eps, int64_t *centers, int32_t *k_out,
                 double *radius, const kc_opts *opts) {
    g_err.clear();
    if (!pts || !centers || !k_out || !radius) return fail(KC_ERR_ARG, "null pointer argument");
    if (n < 1 || n > (int64_t)N_MAX) return fail(KC_ERR_ARG, "n=%lld outside [1, 2^32-2]", (long long)n);
    if (d < 1) return fail(KC_ERR_ARG, "d=%d must be >= 1", d);
    if (k < 1) return fail(KC_ERR_ARG, "k=%d must be >= 1", k);
    if (!(eps > 0.0 && eps < 1.0)) return fail(KC_ERR_ARG, "eps=%g must be in (0, 1)", eps);
    CallCtx c;
    kc_status r = begin(opts, c);
    if (r != KC_OK) return r;
    if (c.async) return fail(KC_ERR_ARG, "kc_eim runs a host loop over sampling rounds and does not take KC_ASYNC");
    const double phi = c.o.phi > 0 ? c.o.phi : 6.0;
    const uint64_t seed = c.o.seed;
    const bool dev_pts = is_device_ptr(pts, c.dev);
    const bool dev_cen = is_device_ptr(centers, c.dev);
    const bool dev_kout = is_device_ptr(k_out, c.dev);
    const bool dev_rad = is_device_ptr(radius, c.dev);

    // Loop constants of Algorithm 2 (natural logarithm, n fixed).
    const double ne = pow((double)n, eps);
    const double ln = log((double)n);
    const double base = ne * ln;
    const double limit = (4.0 / eps) * (double)k * base;
    const int64_t pos = (int64_t)ceil(phi * ln);
    const int64_t hcap = std::max<int64_t>(4096, (int64_t)ceil(64.0 * base) + 1024);
    const int64_t nb = nblocks(n);
    const int64_t nchunks = (n + 1023) / 1024;
    const size_t esz = 4;
    const int keff_max = (int)std::min<int64_t>(k, n);
    const int lp = lp_of(c.o);
    const int grid = choose_gon_grid(c.o.dtype, d, n, lp);
    LPBufs LB;
    float *cenT = nullptr, *ecmax = nullptr;
    RadiusArgs Rtc{}, Ptc{};

    struct L {
        unsigned long long *sn, *hn, *rnn;
        int64_t *total;
        int32_t *range2;
        unsigned long long *key32, *max64, *arg64;
        uint32_t *thr, *v;
        uint64_t *fk, *slots;
        uint8_t *mask;
        PruneBufs pb;
        void *staging, *pk, *Sc, *Hc, *pkC, *cen;
        uint32_t *mind, *mindC, *R0, *R1, *S, *H, *dH;
        int *counts;
        int64_t *offs, *C;
        double *m64;
        int64_t *cen_dev;
        int32_t *kout_dev;
        double *rad_dev;
        size_t zero_bytes;
    } Lo{};
    auto layout = [&](Carve &cv) {
        Lo.sn = cv.take<unsigned long long>(1);
        Lo.hn = cv.take<unsigned long long>(1);
        Lo.rnn = cv.take<unsigned long long>(1);
        Lo.total = cv.take<int64_t>(1);
        Lo.range2 = cv.take<int32_t>(2);
        Lo.key32 = cv.take<unsigned long long>(1);
        Lo.max64 = cv.take<unsigned long long>(1);
        Lo.arg64 = cv.take<unsigned long long>(1);
        Lo.thr = cv.take<uint32_t>(1);
        Lo.v = cv.take<uint32_t>(1);
        Lo.fk = cv.take<uint64_t>(1);
        Lo.slots = cv.take<uint64_t>((size_t)slot_words(keff_max, grid, lp != 0));
        Lo.mask = cv.take<uint8_t>((size_t)n);
        Lo.zero_bytes = cv.off;
        Lo.staging = dev_pts ? nullptr : cv.take<char>((size_t)n * d * esz);
        Lo.pk = cv.take<char>((size_t)nb * BLK * d * esz);
        Lo.mind = cv.take<uint32_t>((size_t)nb * BLK);
        Lo.R0 = cv.take<uint32_t>((size_t)n);
        Lo.R1 = cv.take<uint32_t>((size_t)n);
        Lo.S = cv.take<uint32_t>((size_t)n);
        Lo.Sc = cv.take<char>((size_t)n * d * esz);
        Lo.H = cv.take<uint32_t>((size_t)hcap);
        Lo.Hc = cv.take<char>((size_t)hcap * d * esz);
        Lo.dH = cv.take<uint32_t>((size_t)hcap);
        Lo.counts = cv.take<int>((size_t)nchunks);
        Lo.offs = cv.take<int64_t>((size_t)nchunks);
        Lo.C = cv.take<int64_t>((size_t)n);
        Lo.pkC = cv.take<char>((size_t)nb * BLK * d * esz);
        Lo.mindC = cv.take<uint32_t>((size_t)nb * BLK);
        Lo.cen = cv.take<char>((size_t)keff_max * d * esz);
        Lo.m64 = cv.take<double>(c.o.dtype == KC_F32 ? (size_t)n : 1);
        Lo.cen_dev = dev_cen ? centers : cv.take<int64_t>((size_t)keff_max);
        Lo.kout_dev = dev_kout ? k_out : cv.take<int32_t>(1);
        Lo.rad_dev = dev_rad ? radius : cv.take<double>(1);
        take_lp(cv, LB, lp, n, d);
        cenT = lp ? cv.take<float>((size_t)keff_max * d) : nullptr;
        ecmax = lp ? cv.take<float>(1) : nullptr;
        take_tc(cv, Rtc, c.o.dtype, n, d, keff_max);
        // Tensor-core prune from d = 16 on: below, the fp16 bounds (about 1%
        // relative) leave too many pairs near the threshold undecided (2-D,
        // 1M points: 338 ms against 112 ms on CUDA cores), and a pair costs
        // the CUDA cores little.  KC_PRUNE_TC=0/1 forces either path.
        const char *ptc = getenv("KC_PRUNE_TC");
        const bool tcp = c.o.dtype == KC_F32 && tc_supported(d) && (ptc ? atoi(ptc) != 0 : d >= 16);
        Ptc.tc_at = nullptr;
        if (tcp) {   // tiles for up to n points of R and n centers of S
            Ptc.tc_at = cv.take<char>(tc_point_bytes(n, d));
            Ptc.tc_an = cv.take<float>((size_t)tc_point_rows(n));
            Ptc.tc_ae = cv.take<float>((size_t)tc_point_rows(n));
            Ptc.tc_rin = cv.take<uint8_t>((size_t)tc_point_rows(n));
            Ptc.tc_bt = cv.take<char>(tc_center_bytes(n, d));
            Ptc.tc_cn = cv.take<float>((size_t)tc_center_tiles(n) * 256);
            Ptc.tc_ce = cv.take<float>((size_t)tc_center_tiles(n) * 256);
            Ptc.tc_maxes = cv.take<unsigned>(3);
            Ptc.tc_absmax = cv.take<unsigned>(3);
        }
        Lo.pb = PruneBufs{};
        if (tcp) {   // deferred exact checks: up to 2 pairs per point before full rescans
            Lo.pb.pcap = std::max<int64_t>(2 * n, 1 << 16);
            if (const char *e = getenv("KC_PRUNE_PAIR_CAP")) Lo.pb.pcap = std::max<int64_t>(1, atoll(e));
            Lo.pb.pairs = cv.take<uint2>((size_t)Lo.pb.pcap);
            Lo.pb.flag = cv.take<uint8_t>((size_t)n);
            Lo.pb.hit = cv.take<uint8_t>((size_t)n);
            Lo.pb.pend = cv.take<uint32_t>((size_t)n);
            Lo.pb.npairs = cv.take<unsigned long long>(1);
            Lo.pb.npend = cv.take<unsigned long long>(1);
        }
    };
    {
        Carve sizing(nullptr);
        layout(sizing);
        r = arena_reserve(c.arena, sizing.off, c.s);
        if (r != KC_OK) return r;
    }
    Carve cv(c.arena->dev);
    layout(cv);
    DevStatus *st = c.arena->status;
    c.arena->last_key32 = Lo.key32;
    c.arena->last_dtype = c.o.dtype;
    auto read_u64 = [&](const unsigned long long *p, unsigned long long *out) -> kc_status {
        KC_CUDA(cudaMemcpyAsync(out, p, sizeof *out, cudaMemcpyDeviceToHost, c.s), "count read-back");
        KC_CUDA(cudaStreamSynchronize(c.s), "cudaStreamSynchronize");
        return KC_OK;
    };
    auto device_error = [&]() -> bool {
        DevStatus h;
        if (cudaMemcpy(&h, st, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return true;
        return h.code != 0;
    };

    KC_CUDA(cudaMemsetAsync(c.arena->dev, 0, Lo.zero_bytes, c.s), "scratch clear");
    const void *src;
    r = stage_points(c, pts, (size_t)n * d * esz, dev_pts, Lo.staging, &src);
    if (r != KC_OK) return r;
    {
        TraceStep t("pack", c.s);
        KC_CUDA(launch_pack(src, c.o.dtype, n, d, Lo.pk, Lo.range2, st, c.s), "pack launch");
        if (c.o.dtype == KC_I32) KC_CUDA(launch_range_check(Lo.range2, d, st, c.s), "range check");
        KC_CUDA(launch_eim_iota(Lo.R0, n, c.s), "iota launch");
        if (Ptc.tc_at) KC_CUDA(launch_tc_absmax((const float *)Lo.pk, n, d, Ptc.tc_absmax, c.s), "absmax");
    }
    KC_CUDA(cudaStreamSynchronize(c.s), "cudaStreamSynchronize");
    if (device_error()) return finish(c.arena, c.s);

    int64_t rn = n, sn = 0;
    uint32_t *Rc = Lo.R0, *Rx = Lo.R1;
    int it = 0;
    while ((double)rn > limit) {
        const double pS = fmin(1.0, 9.0 * (double)k * base / (double)rn);
        const double pH = fmin(1.0, 4.0 * base / (double)rn);
        unsigned long long sn_new = 0, hn = 0, rnn = 0;
        {
            TraceStep t("eim_sample", c.s);
            KC_CUDA(cudaMemsetAsync(Lo.hn, 0, sizeof(unsigned long long), c.s), "clear");
            KC_CUDA(cudaMemsetAsync(Lo.rnn, 0, sizeof(unsigned long long), c.s), "clear");
            KC_CUDA(launch_eim_sample(Rc, rn, seed, it, pS, pH, Lo.mask, Lo.S, Lo.sn, Lo.H, Lo.hn, hcap, st, c.s),
                    "sample launch");
        }
        if ((r = read_u64(Lo.sn, &sn_new)) != KC_OK) return r;
        if ((r = read_u64(Lo.hn, &hn)) != KC_OK) return r;
        if ((int64_t)hn > hcap || device_error()) return finish(c.arena, c.s);
        KC_CUDA(launch_eim_gather_rows(src, c.o.dtype, d, Lo.S, sn, (int64_t)sn_new, Lo.Sc, c.s), "gather S");
        sn = (int64_t)sn_new;
        if (hn > 0 && sn > 0) {
            {
                TraceStep t("eim_select", c.s);
                KC_CUDA(launch_eim_gather_rows(src, c.o.dtype, d, Lo.H, 0, (int64_t)hn, Lo.Hc, c.s), "gather H");
                KC_CUDA(launch_eim_dist_hs(c.o.dtype, Lo.Hc, (int64_t)hn, Lo.Sc, sn, d, Lo.dH, c.s), "d(H,S)");
                const int64_t p = std::min<int64_t>((int64_t)hn, std::max<int64_t>(1, pos));
                KC_CUDA(launch_eim_select(Lo.H, Lo.dH, (int64_t)hn, p, Lo.thr, Lo.v, c.s), "select");
            }
            TraceStep t("eim_prune", c.s);
            g_prune_pairs += (unsigned long long)rn * (unsigned long long)sn;
            if (Ptc.tc_at && sn >= 256) {
                // tensor-core R x S block with exact rechecks of undecided pairs
                KC_CUDA(launch_tc_prune((const float *)src, d, Rc, rn, Lo.mask, (const float *)Lo.Sc, sn, tc_bufs(Ptc),
                                        Lo.pb, Lo.thr, Rx, Lo.rnn, st, c.s),
                        "prune");
            } else {
                KC_CUDA(launch_eim_prune(c.o.dtype, src, d, Rc, rn, Lo.mask, Lo.Sc, sn, Lo.thr, Rx, Lo.rnn, c.s),
                        "prune");
            }
        } else {
            KC_CUDA(launch_eim_drop_sampled(Rc, rn, Lo.mask, Rx, Lo.rnn, c.s), "drop sampled");
        }
        if ((r = read_u64(Lo.rnn, &rnn)) != KC_OK) return r;
        rn = (int64_t)rnn;
        std::swap(Rc, Rx);
        ++it;
    }

    // C = S u R in ascending index order, then GON on C and the radius on V.
    int64_t nC = 0;
    {
        TraceStep t("eim_compact", c.s);
        KC_CUDA(launch_eim_mark(Rc, rn, Lo.mask, c.s), "mark");
        KC_CUDA(launch_compact(Lo.mask, n, Lo.counts, Lo.offs, Lo.C, Lo.total, c.s), "compact");
        KC_CUDA(cudaMemcpyAsync(&nC, Lo.total, sizeof nC, cudaMemcpyDeviceToHost, c.s), "count read-back");
        KC_CUDA(cudaStreamSynchronize(c.s), "cudaStreamSynchronize");
        KC_CUDA(launch_gather_pack(Lo.pk, c.o.dtype, d, Lo.C, Lo.total, nC, Lo.pkC, c.s), "gather C");
        if (lp && nC > 0)
            KC_CUDA(launch_lp_pack(lp, (const float *)Lo.pkC, nC, d, LB.colmax, LB.scale, LB.lp, LB.ept, LB.eblk,
                                   LB.stamp,
                                   c.s),
                    "low-precision pack");
    }
    if (nC < 1) return fail(KC_ERR_CUDA, "EIM produced an empty sample");
    const int kC = (int)std::min<int64_t>(k, nC);
    {
        TraceStep t("gonzalez", c.s);
        GonArgs g{};
        gon_single(g, Lo.pkC, c.o.dtype, nC, d, kC, 0, Lo.mindC, Lo.slots, Lo.cen_dev, Lo.kout_dev, Lo.fk,
                   Lo.range2, std::min(grid, choose_gon_grid(c.o.dtype, d, nC, lp)));
        g.single.map = Lo.C;
        if (lp) {
            attach_lp(g.single, LB, lp, cenT, kC, ecmax);
            g.lp_kind = lp;
            g.lp_local_t = lp_local_t(lp);
        }
        g.st = st;
        g.timeout_cycles = timeout_cycles(c.o);
        KC_CUDA(launch_gon(g, c.s), "gonzalez launch");
    }
    {
        TraceStep t("radius", c.s);
        RadiusArgs ra{};
        ra.pk = Lo.pk;
        ra.dtype = c.o.dtype;
        ra.n = n;
        ra.d = d;
        ra.centers = Lo.cen_dev;
        ra.kc_dev = Lo.kout_dev;
        ra.kc_max = kC;
        ra.cen = Lo.cen;
        ra.mind = Lo.mind;
        ra.key32 = Lo.key32;
        ra.max64 = Lo.max64;
        ra.arg64 = Lo.arg64;
        ra.m64 = Lo.m64;
        ra.radius_out = Lo.rad_dev;
        ra.argmax_out = nullptr;
        ra.st = st;
        ra.have_mind = false;
        copy_tc(ra, Rtc);
        KC_CUDA(launch_radius(ra, c.s), "radius launch");
    }
    if (!dev_cen)
        KC_CUDA(cudaMemcpyAsync(centers, Lo.cen_dev, (size_t)kC * sizeof(int64_t), cudaMemcpyDeviceToHost, c.s),
                "copy centers out");
    if (!dev_kout)
        KC_CUDA(cudaMemcpyAsync(k_out, Lo.kout_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, c.s), "copy k_out");
    if (!dev_rad)
        KC_CUDA(cudaMemcpyAsync(radius, Lo.rad_dev, sizeof(double), cudaMemcpyDeviceToHost, c.s), "copy radius");
    return finish(c.arena, c.s);
}

}  // extern "C"

// ------------------------------------------------------------ batched GON
//
// Launch policy.  Instances are ordered longest-first by modelled work
// w = n k (d b + 8) bytes (b bytes per streamed coordinate, the running
// minimum read and written).  With S resident queue-mode CTAs and the fair
// share W / S of the total work W, an instance with w > theta W / S is heavy:
// it is solved by a CTA group of G = ceil(w / (W / S)) CTAs (at most one per
// warp's worth of 128-point blocks) at the front of a cooperative grid, while
// the groups take at most half of the CTAs.  The other instances go through
// the queue longest-first, and group CTAs join the queue when their instance
// is done.  theta = +inf is the plain queue.  KC_AUTOTUNE times every theta
// of kThetas on the batch itself and keeps the fastest per batch shape.
namespace {

constexpr double kThetaQueue = 1e300;
constexpr double kThetas[] = {kThetaQueue, 4.0, 2.0, 1.0, 0.5};
constexpr double kThetaDefault = 1.0;

struct BatchShape {
    int count = 0, dtype = 0, lp = 0, dc = 0, dmax = 0;
    std::vector<int> order;   // descriptor position -> instance
    std::vector<int> G;       // CTAs per descriptor position (1: queue)
    int nheavy = 0, gheavy = 0, grid = 0;
    double theta = kThetaQueue;
};

void batch_policy(BatchShape &b, const int64_t *n, const int32_t *d, const int32_t *k, double theta) {
    const int count = b.count;
    const double bpc = b.lp == KC_SWEEP_BF16 ? 2.0 : 4.0;
    std::vector<double> w((size_t)count);
    double W = 0;
    for (int i = 0; i < count; ++i) {
        w[i] = (double)n[i] * (double)std::min<int64_t>(k[i], n[i]) * (d[i] * bpc + 8.0);
        W += w[i];
    }
    std::vector<int> lpt((size_t)count);
    for (int i = 0; i < count; ++i) lpt[i] = i;
    std::stable_sort(lpt.begin(), lpt.end(), [&](int a, int c) { return w[a] > w[c]; });
    const int slots = gon_queue_grid(b.dtype, b.dc, b.lp);
    const double share = W / std::max(1, slots);
    b.order.clear();
    b.G.clear();
    b.nheavy = b.gheavy = 0;
    b.theta = theta;
    std::vector<char> heavy((size_t)count, 0);
    for (int q = 0; q < count && theta < kThetaQueue; ++q) {
        const int i = lpt[q];
        if (!(w[i] > theta * share)) break;
        const int64_t gmax = std::max<int64_t>(1, nblocks(n[i]) / gon_queue_warps());
        const int g = (int)std::min<double>(std::ceil(w[i] / share), (double)gmax);
        if (g < 2) continue;
        if (b.gheavy + g > slots / 2) break;
        heavy[i] = 1;
        b.order.push_back(i);
        b.G.push_back(g);
        b.gheavy += g;
        ++b.nheavy;
    }
    for (int q = 0; q < count; ++q)
        if (!heavy[lpt[q]]) {
            b.order.push_back(lpt[q]);
            b.G.push_back(1);
        }
    const int nlight = count - b.nheavy;
    b.grid = b.nheavy ? std::max(b.gheavy, std::min(slots, b.gheavy + nlight)) : std::min(slots, count);
}

uint64_t batch_signature(const BatchShape &b, const int64_t *n, const int32_t *d, const int32_t *k) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (v >> (8 * i)) & 0xFFu;
            h *= 1099511628211ull;
        }
    };
    mix((uint64_t)b.count);
    mix((uint64_t)b.dtype);
    mix((uint64_t)b.lp);
    int dev = 0;
    cudaGetDevice(&dev);
    mix((uint64_t)dev);
    for (int i = 0; i < b.count; ++i) {
        mix((uint64_t)n[i]);
        mix((uint64_t)d[i]);
        mix((uint64_t)k[i]);
    }
    return h;
}

std::mutex g_tune_mu;
std::map<uint64_t, double> g_tune;   // batch signature -> fastest theta


bool tuned_theta(uint64_t sig, double *theta) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(sig);
    if (it == g_tune.end()) return false;
    *theta = it->second;
    return true;
}

void remember_theta(uint64_t sig, double theta) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[sig] = theta;
}

// The theta for a batch: KC_BATCH_THETA if set ("inf": the plain queue;
// it also skips tuning), else the tuned one for this shape, else the
// default.  Returns whether the choice is settled (no tuning needed).
bool pick_theta(uint64_t sig, double *theta) {
    const char *e = getenv("KC_BATCH_THETA");
    if (e && *e) {
        const double v = strcmp(e, "inf") == 0 ? kThetaQueue : atof(e);
        *theta = v > 0 ? v : kThetaDefault;
        return true;
    }
    *theta = kThetaDefault;
    return tuned_theta(sig, theta);
}

// Device buffers of one batch, carved from one allocation.  The zero region
// (queue counter, per-instance range words, group slots) starts the layout.
struct BatchBufs {
    struct Per {
        void *staging, *pk;
        uint32_t *mind;
        int64_t *cen;
        int32_t *range2;
        uint32_t *lpw;
        float *ept, *eblk, *cenT, *ecmax;
        uint32_t *m32, *stamp;
        uint64_t *slots;
    };
    std::vector<Per> per;
    int *counter = nullptr;
    size_t zero_bytes = 0;
    int32_t *kout_dev = nullptr;
    double *rad_dev = nullptr;
    uint64_t *fkeys = nullptr;
    PackSeg *segs_dev = nullptr;
    GonInst *insts_dev = nullptr;
    LpSeg *lsegs_dev = nullptr;
    DevStatus *st = nullptr;   // set by the caller
    char *base = nullptr;
    int64_t blocks = 0;        // packed blocks of all instances
};

// Lay out the batch's buffers (sizing pass when cv's base is null).
// staging[i] / out pointers: used as given when the caller's memory is on
// the device (dev_* true), else carved.
void batch_layout(Carve &cv, const BatchShape &b, BatchBufs &B, const int64_t *n, const int32_t *d, const int32_t *k,
                  int64_t *const *centers, int32_t *k_out, double *radii, const char *dev_pts, const char *dev_cen,
                  bool dev_kout, bool dev_rad) {
    const int count = b.count;
    const size_t esz = 4;
    B.per.assign((size_t)count, BatchBufs::Per{});
    B.base = cv.base;
    B.counter = cv.take<int>(1);
    for (int i = 0; i < count; ++i) B.per[i].range2 = cv.take<int32_t>(2);
    for (int q = 0; q < b.nheavy; ++q) {
        const int i = b.order[q];
        B.per[i].slots = cv.take<uint64_t>((size_t)slot_words(std::min<int64_t>(k[i], n[i]), b.G[q], b.lp != 0));
    }
    B.zero_bytes = cv.off;
    B.kout_dev = dev_kout ? k_out : cv.take<int32_t>((size_t)count);
    B.rad_dev = dev_rad ? radii : cv.take<double>((size_t)count);
    B.fkeys = cv.take<uint64_t>((size_t)count);
    B.segs_dev = cv.take<PackSeg>((size_t)count);
    B.insts_dev = cv.take<GonInst>((size_t)count);
    B.lsegs_dev = cv.take<LpSeg>(b.lp ? (size_t)count : 0);
    for (int i = 0; i < count; ++i) {
        const int64_t nbi = nblocks(n[i]);
        const int ki = (int)std::min<int64_t>(k[i], n[i]);
        BatchBufs::Per &P = B.per[i];
        P.staging = dev_pts[i] ? nullptr : cv.take<char>((size_t)n[i] * d[i] * esz);
        P.pk = cv.take<char>((size_t)nbi * BLK * d[i] * esz);
        P.mind = cv.take<uint32_t>((size_t)nbi * BLK);
        P.cen = dev_cen[i] ? centers[i] : cv.take<int64_t>((size_t)ki);
        if (b.lp) {
            P.lpw = cv.take<uint32_t>((size_t)nbi * lp_ngroups(b.lp, d[i]) * BLK);
            P.ept = cv.take<float>((size_t)nbi * BLK);
            P.eblk = cv.take<float>((size_t)nbi);
            P.cenT = cv.take<float>((size_t)ki * d[i]);
            P.m32 = cv.take<uint32_t>((size_t)nbi * BLK);
            P.stamp = cv.take<uint32_t>((size_t)nbi * BLK);
            P.ecmax = cv.take<float>(1);
        }
    }
}

// Host image of the descriptors PackSeg[count], GonInst[count] and
// LpSeg[count] (descriptor order), contiguous from B.segs_dev.
std::vector<char> batch_descriptors(const BatchShape &b, BatchBufs &B, const void *const *pts, const int64_t *n,
                                    const int32_t *d, const int32_t *k, const char *dev_pts, size_t *bytes) {
    const int count = b.count;
    const size_t gi_off = (char *)B.insts_dev - (char *)B.segs_dev;
    const size_t ls_off = (char *)B.lsegs_dev - (char *)B.segs_dev;
    *bytes = b.lp ? ls_off + sizeof(LpSeg) * count : gi_off + sizeof(GonInst) * count;
    std::vector<char> host(*bytes + 256, 0);
    PackSeg *hs = reinterpret_cast<PackSeg *>(host.data());
    GonInst *hg = reinterpret_cast<GonInst *>(host.data() + gi_off);
    LpSeg *hl = reinterpret_cast<LpSeg *>(host.data() + ls_off);
    int64_t blk0 = 0;
    int cta0 = 0;
    for (int q = 0; q < count; ++q) {
        const int i = b.order[q];
        const BatchBufs::Per &P = B.per[i];
        PackSeg &S = hs[q];
        S.src = dev_pts[i] ? pts[i] : P.staging;
        S.dst = P.pk;
        S.range2 = P.range2;
        S.n = n[i];
        S.blk0 = blk0;
        S.d = d[i];
        if (b.lp) {
            LpSeg &Ls = hl[q];
            Ls.pk = (const float *)P.pk;
            Ls.lp = P.lpw;
            Ls.ept = P.ept;
            Ls.eblk = P.eblk;
            Ls.stamp = P.stamp;
            Ls.n = n[i];
            Ls.blk0 = blk0;
            Ls.d = d[i];
        }
        blk0 += nblocks(n[i]);
        GonInst &I = hg[q];
        I.pk = P.pk;
        I.mind = P.mind;
        I.slots = q < b.nheavy ? P.slots : nullptr;
        I.centers = P.cen;
        I.k_out = B.kout_dev + i;
        I.final_key = B.fkeys + i;
        I.map = nullptr;
        I.range2 = P.range2;
        I.radius_out = B.rad_dev + i;
        I.lo = 0;
        I.n = n[i];
        I.base = 0;
        I.first = 0;
        I.d = d[i];
        I.k = (int)std::min<int64_t>(k[i], n[i]);
        I.cta0 = q < b.nheavy ? cta0 : 0;
        I.G = q < b.nheavy ? b.G[q] : 1;
        if (q < b.nheavy) cta0 += b.G[q];
        I.kcap = I.k;
        if (b.lp) {
            I.lp = P.lpw;
            I.eblk = P.eblk;
            I.ept = P.ept;
            I.scale = nullptr;
            I.cenT = P.cenT;
            I.m32 = P.m32;
            I.stamp = P.stamp;
            I.ecmax_out = P.ecmax;
            I.lp_kind = b.lp;
            // the exact rechecks read the instance's FP32 rows (device memory
            // or its staging copy) rather than its packed copy
            I.rm = (const float *)(dev_pts[i] ? pts[i] : P.staging);
        }
    }
    B.blocks = blk0;
    return host;
}

// Enqueue one solve of the batch (descriptors already on the device):
// clear the zero region, pack, GON, radii.  Stream-capturable.
kc_status batch_enqueue(const BatchShape &b, const BatchBufs &B, long long timeout, bool trace, cudaStream_t s) {
    KC_CUDA(cudaMemsetAsync(B.base, 0, B.zero_bytes, s), "scratch clear");
    {
        TraceStep t(trace ? "pack" : nullptr, s);
        KC_CUDA(launch_pack_many(B.segs_dev, b.count, B.blocks, b.dtype, B.st, s), "pack launch");
        if (b.lp) KC_CUDA(launch_lp_pack_many(B.lsegs_dev, b.count, B.blocks, s), "low-precision pack");
    }
    {
        TraceStep t(trace ? "gonzalez_batch" : nullptr, s);
        GonArgs g{};
        g.insts = B.insts_dev;
        g.ninst = b.count;
        g.dtype = b.dtype;
        g.dc = b.dc;
        g.dmax = b.dmax;
        g.st = B.st;
        g.timeout_cycles = timeout;
        g.grid = b.grid;
        g.queue = 1;
        g.counter = B.counter;
        g.lp_kind = b.lp;
        g.nheavy = b.nheavy;
        g.gheavy = b.gheavy;
        KC_CUDA(launch_gon(g, s), "batch launch");
    }
    {
        TraceStep t(trace ? "radius_batch" : nullptr, s);
        KC_CUDA(launch_batch_radius(B.insts_dev, b.count, b.dtype, B.st, s), "batch radius launch");
    }
    return KC_OK;
}

// Shared argument checks and the shape of a batch (everything but the policy).
kc_status batch_check(int32_t count, const void *const *pts, const int64_t *n, const int32_t *d, const int32_t *k,
                      int64_t *const *centers, const int32_t *k_out, const double *radii, const kc_opts &o,
                      BatchShape &b) {
    if (count < 1) return fail(KC_ERR_ARG, "count=%d must be >= 1", count);
    if (!pts || !n || !d || !k || !centers || !k_out || !radii) return fail(KC_ERR_ARG, "null pointer argument");
    int dmax = 0, dcommon = d[0];
    for (int i = 0; i < count; ++i) {
        if (!pts[i] || !centers[i]) return fail(KC_ERR_ARG, "instance %d: null pointer", i);
        if (n[i] < 1 || n[i] > (int64_t)N_MAX) return fail(KC_ERR_ARG, "instance %d: n outside [1, 2^32-2]", i);
        if (d[i] < 1) return fail(KC_ERR_ARG, "instance %d: d must be >= 1", i);
        if (k[i] < 1) return fail(KC_ERR_ARG, "instance %d: k must be >= 1", i);
        dmax = std::max(dmax, (int)d[i]);
        if (d[i] != dcommon) dcommon = 0;
    }
    b.count = count;
    b.dtype = o.dtype;
    b.lp = lp_of(o);
    if (b.lp == KC_SWEEP_FP8 || b.lp == KC_SWEEP_FP16)
        return fail(KC_ERR_ARG,
                    "the batched form takes KC_SWEEP_F32 or KC_SWEEP_BF16 (fp8 and fp16 need per-instance scales)");
    b.dc = (dcommon == 3 || dcommon == 8 || dcommon == 32) && o.dtype == KC_F32 ? dcommon : 0;
    b.dmax = dmax;
    return KC_OK;
}

}  // namespace

extern "C" {

kc_status kc_gonzalez_batch(int32_t count, const void *const *pts, const int64_t *n, const int32_t *d,
                            const int32_t *k, int64_t *const *centers, int32_t *k_out, double *radii,
                            const kc_opts *opts) {
    g_err.clear();
    BatchShape b;
    kc_status r = batch_check(count, pts, n, d, k, centers, k_out, radii, opts ? *opts : default_opts(), b);
    if (r != KC_OK) return r;
    CallCtx c;
    if ((r = begin(opts, c, KC_ASYNC | KC_AUTOTUNE)) != KC_OK) return r;
    const bool dev_kout = is_device_ptr(k_out, c.dev);
    const bool dev_rad = is_device_ptr(radii, c.dev);
    std::vector<char> dev_pts((size_t)count), dev_cen((size_t)count);
    bool all_dev = dev_kout && dev_rad;
    for (int i = 0; i < count; ++i) {
        dev_pts[i] = is_device_ptr(pts[i], c.dev);
        dev_cen[i] = is_device_ptr(centers[i], c.dev);
        all_dev = all_dev && dev_pts[i] && dev_cen[i];
    }
    if (c.async && !all_dev) return fail(KC_ERR_ARG, "KC_ASYNC needs device pointers for all arguments");
    const bool tune = (c.o.flags & KC_AUTOTUNE) != 0;
    if (tune && c.async) return fail(KC_ERR_ARG, "KC_AUTOTUNE times the batch and does not take KC_ASYNC");
    const uint64_t sig = batch_signature(b, n, d, k);
    double theta = kThetaDefault;
    const bool known = pick_theta(sig, &theta);

    BatchBufs B;
    // One solve with the given theta: layout, inputs, descriptors, launches.
    auto solve = [&](double th, float *ms) -> kc_status {
        batch_policy(b, n, d, k, th);
        Carve sizing(nullptr);
        batch_layout(sizing, b, B, n, d, k, centers, k_out, radii, dev_pts.data(), dev_cen.data(), dev_kout, dev_rad);
        kc_status rr = arena_reserve(c.arena, sizing.off, c.s);
        if (rr != KC_OK) return rr;
        Carve cv(c.arena->dev);
        batch_layout(cv, b, B, n, d, k, centers, k_out, radii, dev_pts.data(), dev_cen.data(), dev_kout, dev_rad);
        B.st = c.arena->status;
        size_t up_bytes = 0;
        std::vector<char> host = batch_descriptors(b, B, pts, n, d, k, dev_pts.data(), &up_bytes);
        for (int i = 0; i < count; ++i)
            if (!dev_pts[i])
                KC_CUDA(cudaMemcpyAsync(B.per[i].staging, pts[i], (size_t)n[i] * d[i] * 4, cudaMemcpyHostToDevice,
                                        c.s),
                        "copy points to device");
        if ((rr = upload(c.arena, c.s, host.data(), up_bytes, B.segs_dev)) != KC_OK) return rr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (ms) {
            KC_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
            KC_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
            KC_CUDA(cudaEventRecord(e0, c.s), "cudaEventRecord");
        }
        rr = batch_enqueue(b, B, timeout_cycles(c.o), true, c.s);
        if (ms) {
            if (rr == KC_OK) {
                KC_CUDA(cudaEventRecord(e1, c.s), "cudaEventRecord");
                KC_CUDA(cudaEventSynchronize(e1), "cudaEventSynchronize");
                KC_CUDA(cudaEventElapsedTime(ms, e0, e1), "cudaEventElapsedTime");
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
        return rr;
    };

    if (tune && !known) {
        // Every candidate solves the batch exactly (selection does not depend
        // on the launch shape); the fastest theta is remembered.
        float best_ms = 0.f;
        for (double th : kThetas) {
            float ms = 0.f;
            if ((r = solve(th, &ms)) != KC_OK) return r;
            if ((r = finish(c.arena, c.s)) != KC_OK) return r;
            if (th == kThetas[0] || ms < best_ms) {
                best_ms = ms;
                theta = th;
            }
        }
        remember_theta(sig, theta);
    }
    if ((r = solve(theta, nullptr)) != KC_OK) return r;
    for (int i = 0; i < count; ++i)
        if (!dev_cen[i])
            KC_CUDA(cudaMemcpyAsync(centers[i], B.per[i].cen, (size_t)std::min<int64_t>(k[i], n[i]) * sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, c.s),
                    "copy centers out");
    if (!dev_kout)
        KC_CUDA(cudaMemcpyAsync(k_out, B.kout_dev, (size_t)count * sizeof(int32_t), cudaMemcpyDeviceToHost, c.s),
                "copy k_out");
    if (!dev_rad)
        KC_CUDA(cudaMemcpyAsync(radii, B.rad_dev, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost, c.s),
                "copy radii");
    if (c.async) return KC_OK;
    return finish(c.arena, c.s);
}

}  // extern "C"

// ------------------------------------------------------------ batch plans
struct kc_batch_plan {
    int dev = 0;
    char *mem = nullptr;
    DevStatus *st = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t last = nullptr;
    bool ran = false;
    double theta = 0;
    int nheavy = 0, gheavy = 0, grid = 0;
};

namespace {

void plan_free(kc_batch_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->mem) cudaFree(p->mem);
    delete p;
}

// Build one plan: its own device allocation (outside the per-stream arena,
// so later calls cannot move it), descriptors uploaded once, and the solve
// captured into a CUDA graph.
kc_status plan_build(BatchShape &b, double theta, int32_t count, const void *const *pts, const int64_t *n,
                     const int32_t *d, const int32_t *k, int64_t *const *centers, int32_t *k_out, double *radii,
                     const kc_opts &o, kc_batch_plan **out) {
    batch_policy(b, n, d, k, theta);
    std::vector<char> dev_pts((size_t)count, 1), dev_cen((size_t)count, 1);
    BatchBufs B;
    Carve sizing(nullptr);
    sizing.take<DevStatus>(1);
    batch_layout(sizing, b, B, n, d, k, centers, k_out, radii, dev_pts.data(), dev_cen.data(), true, true);
    kc_batch_plan *p = new kc_batch_plan();
    KC_CUDA(cudaGetDevice(&p->dev), "cudaGetDevice");
    cudaError_t e = cudaMalloc(&p->mem, sizing.off + 256);
    if (e != cudaSuccess) {
        cudaGetLastError();
        plan_free(p);
        return fail(KC_ERR_OOM, "plan allocation of %zu bytes failed", sizing.off + 256);
    }
    Carve cv(p->mem);
    p->st = cv.take<DevStatus>(1);
    batch_layout(cv, b, B, n, d, k, centers, k_out, radii, dev_pts.data(), dev_cen.data(), true, true);
    B.st = p->st;
    size_t up_bytes = 0;
    std::vector<char> host = batch_descriptors(b, B, pts, n, d, k, dev_pts.data(), &up_bytes);
    cudaStream_t cs = nullptr;
    kc_status r = KC_OK;
    do {
        if ((e = cudaMemset(p->st, 0, sizeof(DevStatus))) != cudaSuccess ||
            (e = cudaMemcpy(B.segs_dev, host.data(), up_bytes, cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
            r = cuda_fail(e, "plan setup");
            break;
        }
        r = batch_enqueue(b, B, timeout_cycles(o), false, cs);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        if (r != KC_OK) {
            if (g) cudaGraphDestroy(g);
            break;
        }
        if (e != cudaSuccess) {
            r = cuda_fail(e, "graph capture");
            break;
        }
        p->graph = g;
        if ((e = cudaGraphInstantiate(&p->exec, g, 0)) != cudaSuccess) r = cuda_fail(e, "graph instantiation");
    } while (false);
    if (cs) cudaStreamDestroy(cs);
    if (r != KC_OK) {
        plan_free(p);
        return r;
    }
    p->theta = theta;
    p->nheavy = b.nheavy;
    p->gheavy = b.gheavy;
    p->grid = b.grid;
    *out = p;
    return KC_OK;
}

kc_status plan_status(kc_batch_plan *p) {
    DevStatus h;
    KC_CUDA(cudaMemcpy(&h, p->st, sizeof h, cudaMemcpyDeviceToHost), "status read-back");
    if (h.code != 0) {
        KC_CUDA(cudaMemset(p->st, 0, sizeof(DevStatus)), "status reset");
        return status_text(h);
    }
    return KC_OK;
}

}  // namespace

extern "C" {

kc_status kc_batch_plan_create(int32_t count, const void *const *pts, const int64_t *n, const int32_t *d,
                               const int32_t *k, int64_t *const *centers, int32_t *k_out, double *radii,
                               const kc_opts *opts, kc_batch_plan **plan) {
    g_err.clear();
    if (!plan) return fail(KC_ERR_ARG, "null plan pointer");
    *plan = nullptr;
    BatchShape b;
    kc_status r = batch_check(count, pts, n, d, k, centers, k_out, radii, opts ? *opts : default_opts(), b);
    if (r != KC_OK) return r;
    CallCtx c;
    if ((r = begin(opts, c, KC_AUTOTUNE)) != KC_OK) return r;
    if (!is_device_ptr(k_out, c.dev) || !is_device_ptr(radii, c.dev))
        return fail(KC_ERR_ARG, "a plan needs device memory for k_out and radii");
    for (int i = 0; i < count; ++i)
        if (!is_device_ptr(pts[i], c.dev) || !is_device_ptr(centers[i], c.dev))
            return fail(KC_ERR_ARG, "instance %d: a plan needs device memory for points and centers", i);
    const uint64_t sig = batch_signature(b, n, d, k);
    double theta = kThetaDefault;
    const bool known = pick_theta(sig, &theta);
    if ((c.o.flags & KC_AUTOTUNE) && !known) {
        // Time each candidate's graph (one warm-up replay, then the fastest of
        // five replays timed one by one: a mean of a few replays let one slow
        // replay pick a slower split) and keep the fastest plan.
        kc_batch_plan *best = nullptr;
        float best_ms = 0.f;
        cudaEvent_t e0, e1;
        KC_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
        KC_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
        for (double th : kThetas) {
            kc_batch_plan *p = nullptr;
            if ((r = plan_build(b, th, count, pts, n, d, k, centers, k_out, radii, c.o, &p)) != KC_OK) break;
            float ms = 0.f;
            cudaError_t e = cudaGraphLaunch(p->exec, c.s);
            for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
                float one = 0.f;
                e = cudaEventRecord(e0, c.s);
                if (e == cudaSuccess) e = cudaGraphLaunch(p->exec, c.s);
                if (e == cudaSuccess) e = cudaEventRecord(e1, c.s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&one, e0, e1);
                if (e == cudaSuccess && (rep == 0 || one < ms)) ms = one;
            }
            if (e != cudaSuccess) {
                r = cuda_fail(e, "plan timing");
                plan_free(p);
                break;
            }
            if ((r = plan_status(p)) != KC_OK) {
                plan_free(p);
                break;
            }
            if (!best || ms < best_ms) {
                plan_free(best);
                best = p;
                best_ms = ms;
            } else {
                plan_free(p);
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (r != KC_OK) {
            plan_free(best);
            return r;
        }
        remember_theta(sig, best->theta);
        *plan = best;
        return KC_OK;
    }
    return plan_build(b, theta, count, pts, n, d, k, centers, k_out, radii, c.o, plan);
}

kc_status kc_batch_plan_run(kc_batch_plan *plan, void *stream) {
    g_err.clear();
    if (!plan) return fail(KC_ERR_ARG, "null plan");
    int dev = 0;
    KC_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != plan->dev) return fail(KC_ERR_ARG, "the plan belongs to device %d, current device is %d", plan->dev, dev);
    KC_CUDA(cudaGraphLaunch(plan->exec, (cudaStream_t)stream), "graph launch");
    plan->last = (cudaStream_t)stream;
    plan->ran = true;
    note_launches(3);
    return KC_OK;
}

kc_status kc_batch_plan_wait(kc_batch_plan *plan) {
    g_err.clear();
    if (!plan) return fail(KC_ERR_ARG, "null plan");
    if (!plan->ran) return KC_OK;
    KC_CUDA(cudaStreamSynchronize(plan->last), "cudaStreamSynchronize");
    return plan_status(plan);
}

kc_status kc_batch_plan_info(const kc_batch_plan *plan, double *theta, int32_t *nheavy, int32_t *gheavy,
                             int32_t *grid) {
    g_err.clear();
    if (!plan) return fail(KC_ERR_ARG, "null plan");
    if (theta) *theta = plan->theta;
    if (nheavy) *nheavy = plan->nheavy;
    if (gheavy) *gheavy = plan->gheavy;
    if (grid) *grid = plan->grid;
    return KC_OK;
}

kc_status kc_batch_plan_destroy(kc_batch_plan *plan) {
    g_err.clear();
    if (!plan) return KC_OK;
    if (plan->ran) cudaStreamSynchronize(plan->last);
    plan_free(plan);
    return KC_OK;
}

}  // extern "C"
