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
    TraceStep(const char *name, cudaStream_t s_) : on(g_trace_on.load() != 0), s(s_) {
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

kc_opts default_opts() {
    kc_opts o;
    memset(&o, 0, sizeof o);
    o.dtype = KC_F32;
    o.phi = 6.0;
    return o;
}

long long timeout_cycles(const kc_opts &o) {
    int dev = 0, khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
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

kc_status begin(const kc_opts *opts, CallCtx &c) {
    c.o = opts ? *opts : default_opts();
    if (c.o.dtype != KC_F32 && c.o.dtype != KC_I32) return fail(KC_ERR_ARG, "dtype must be KC_F32 or KC_I32");
    if (c.o.flags & ~KC_ASYNC) return fail(KC_ERR_ARG, "unknown flags 0x%x", c.o.flags);
    if (c.o.sweep < KC_SWEEP_F32 || c.o.sweep > KC_SWEEP_FP8) return fail(KC_ERR_ARG, "unknown sweep %d", c.o.sweep);
    c.s = (cudaStream_t)c.o.stream;
    c.async = (c.o.flags & KC_ASYNC) != 0;
    KC_CUDA(cudaGetDevice(&c.dev), "cudaGetDevice");
    return arena_for(c.s, &c.arena);
}

// Input points: device pointer as is, else copied into `staging`.
kc_status stage_points(const CallCtx &c, const void *pts, size_t bytes, bool dev_in, void *staging,
                       const void **out) {
    if (dev_in) {
        *out = pts;
        return KC_OK;
    }
    KC_CUDA(cudaMemcpyAsync(staging, pts, bytes, cudaMemcpyHostToDevice, c.s), "copy points to device");
    *out = staging;
    return KC_OK;
}

// Low-precision sweep kind for a call: only float points use it.
int lp_of(const kc_opts &o) { return o.dtype == KC_F32 ? o.sweep : 0; }

// Scratch of the mixed-precision sweep over one packed array of n points.
struct LPBufs {
    uint32_t *lp = nullptr;
    float *eblk = nullptr, *ept = nullptr, *scale = nullptr;
    unsigned *colmax = nullptr;
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
}

// Tensor-core radius filter scratch for kc centers over n float points
// (left null, i.e. CUDA cores, for int32 points, d > 128, tiny center sets,
// or KC_RADIUS_TC=0 in the environment).
void take_tc(Carve &cv, RadiusArgs &ra, int dtype, int64_t n, int d, int kc) {
    bool use = dtype == KC_F32 && tc_supported(d) && (int64_t)kc * d >= 8192;
    if (const char *env = getenv("KC_RADIUS_TC")) use = dtype == KC_F32 && tc_supported(d) && atoi(env) != 0;
    if (!use) {
        ra.tc_at = nullptr;
        return;
    }
    ra.tc_at = cv.take<char>(tc_point_bytes(n, d));
    ra.tc_an = cv.take<float>((size_t)tc_point_rows(n));
    ra.tc_ae = cv.take<float>((size_t)tc_point_rows(n));
    ra.tc_bt = cv.take<char>(tc_center_bytes(kc, d));
    ra.tc_cn = cv.take<float>((size_t)tc_center_tiles(kc) * 256);
    ra.tc_ce = cv.take<float>((size_t)tc_center_tiles(kc) * 256);
    ra.tc_maxes = cv.take<unsigned>(2);
    ra.tc_absmax = cv.take<unsigned>(1);
    ra.tc_mlo = cv.take<float>((size_t)n);
    ra.tc_mhi = cv.take<float>((size_t)n);
    ra.tc_mlomax = cv.take<unsigned>(1);
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
}  // namespace kc

extern "C" {

const char *kc_version(void) { return "kcenter-gb300 0.1 (sm_103a)"; }

void kc_trace_enable(int32_t on) { g_trace_on = on ? 1 : 0; }

int32_t kc_counters(int64_t *out, int32_t cap) {
    unsigned long long v[4] = {0, 0, 0, 0};
    if (cudaDeviceSynchronize() != cudaSuccess || read_counters(v, true) != cudaSuccess ||
        read_tc_counters(v + 2, true) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    for (int i = 0; i < cap && i < 4; ++i) out[i] = (int64_t)v[i];
    return 4;
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
    kc_status r = begin(opts, c);
    if (r != KC_OK) return r;

    const bool dev_pts = is_device_ptr(pts, c.dev);
    const bool dev_cen = is_device_ptr(centers, c.dev);
    const bool dev_kout = is_device_ptr(k_out, c.dev);
    const bool dev_rad = is_device_ptr(radius, c.dev);
    if (c.async && !(dev_pts && dev_cen && dev_kout && dev_rad))
        return fail(KC_ERR_ARG, "KC_ASYNC needs device pointers for all arguments");

    const int keff = (int)(k < n ? k : n);
    const int lp = lp_of(c.o);
    const int grid = choose_gon_grid(c.o.dtype, d, n, lp);
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
        uint64_t *slots = cv.take<uint64_t>((size_t)keff * grid);
        *zero_bytes = cv.off;
        *staging = dev_pts ? nullptr : cv.take<char>((size_t)n * d * esz);
        void *pk = cv.take<char>((size_t)nb * BLK * d * esz);
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
        if (lp) {
            attach_lp(g.single, LB, lp, cenT, keff, ecmax);
            g.lp_kind = lp;
            ra.eblk = LB.eblk;
            ra.ecmax = ecmax;
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

    KC_CUDA(cudaMemsetAsync(c.arena->dev, 0, zero_bytes, c.s), "scratch clear");
    const void *src;
    r = stage_points(c, pts, (size_t)n * d * esz, dev_pts, staging, &src);
    if (r != KC_OK) return r;
    {
        TraceStep t("pack", c.s);
        KC_CUDA(launch_pack(src, c.o.dtype, n, d, (void *)g.single.pk, (int32_t *)g.single.range2,
                            c.arena->status, c.s),
                "pack launch");
        if (lp)
            KC_CUDA(launch_lp_pack(lp, (const float *)g.single.pk, n, d, LB.colmax, LB.scale, LB.lp, LB.ept,
                                   LB.eblk, c.s),
                    "low-precision pack");
    }
    {
        TraceStep t("gonzalez", c.s);
        KC_CUDA(launch_gon(g, c.s), "gonzalez launch");
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

    const bool dev_pts = is_device_ptr(pts, c.dev);
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
        zero_bytes = cv.off;
        staging = dev_pts ? nullptr : cv.take<char>((size_t)n * d * esz);
        ra.pk = cv.take<char>((size_t)nb * BLK * d * esz);
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

    KC_CUDA(cudaMemsetAsync(c.arena->dev, 0, zero_bytes, c.s), "scratch clear");
    const void *src;
    r = stage_points(c, pts, (size_t)n * d * esz, dev_pts, staging, &src);
    if (r != KC_OK) return r;
    if (!dev_cin)
        KC_CUDA(cudaMemcpyAsync((void *)cin_dev, centers, (size_t)kc * sizeof(int64_t), cudaMemcpyHostToDevice, c.s),
                "copy centers in");
    {
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

kc_status kc_mrg(const void *pts, int64_t n, int32_t d, int32_t k, int32_t m, const int64_t *offsets,
                 int64_t *centers, int32_t *k_out, double *radius, const kc_opts *opts) {
    g_err.clear();
    if (!pts || !centers || !k_out || !radius) return fail(KC_ERR_ARG, "null pointer argument");
    if (n < 1 || n > (int64_t)N_MAX) return fail(KC_ERR_ARG, "n=%lld outside [1, 2^32-2]", (long long)n);
    if (d < 1) return fail(KC_ERR_ARG, "d=%d must be >= 1", d);
    if (k < 1) return fail(KC_ERR_ARG, "k=%d must be >= 1", k);
    if (m < 1 || m > n) return fail(KC_ERR_ARG, "m=%d must be in [1, n]", m);
    CallCtx c;
    kc_status r = begin(opts, c);
    if (r != KC_OK) return r;
    const bool dev_pts = is_device_ptr(pts, c.dev);
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

    // Round-1 CTA groups: proportional to each part's work n_i * k_i, at least
    // one CTA, at most one per 32 blocks (one block per warp), within the
    // co-resident grid.  More parts than CTAs: one CTA per part from a queue.
    const int lp = lp_of(c.o);
    const int maxg = gon_max_grid(c.o.dtype, d, lp);
    const int W = gon_warps_per_cta();
    std::vector<int> G((size_t)m, 1), ki((size_t)m);
    std::vector<int64_t> slot_off((size_t)m + 1, 0);
    const bool queue1 = m > maxg;
    {
        double tot = 0;
        std::vector<double> work((size_t)m);
        for (int i = 0; i < m; ++i) {
            const int64_t ni = off[i + 1] - off[i];
            ki[i] = (int)(k < ni ? k : ni);
            work[i] = (double)ni * ki[i];
            tot += work[i];
        }
        if (!queue1) {
            std::vector<int> cap((size_t)m);
            int sum = 0;
            for (int i = 0; i < m; ++i) {
                const int64_t nbi = nblocks(off[i + 1] - off[i]) + 1;
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
        for (int i = 0; i < m; ++i) slot_off[i + 1] = slot_off[i] + (queue1 ? 0 : (int64_t)ki[i] * G[i]);
    }
    int grid1 = 0;
    for (int i = 0; i < m; ++i) grid1 += G[i];
    if (queue1) grid1 = gon_queue_grid(c.o.dtype, d, lp);
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
        int64_t *c1, *U;
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
        Lo.slots2 = cv.take<uint64_t>((size_t)k * G2);
        Lo.zero_bytes = cv.off;
        Lo.staging = dev_pts ? nullptr : cv.take<char>((size_t)n * d * esz);
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
    r = stage_points(c, pts, (size_t)n * d * esz, dev_pts, Lo.staging, &src);
    if (r != KC_OK) return r;
    r = upload(c.arena, c.s, h1.data(), h1.size() * sizeof(GonInst), Lo.insts1);
    if (r != KC_OK) return r;
    const long long tmo = timeout_cycles(c.o);
    {
        TraceStep t("pack", c.s);
        KC_CUDA(launch_pack(src, c.o.dtype, n, d, Lo.pk, Lo.range2, st, c.s), "pack launch");
        if (lp)
            KC_CUDA(launch_lp_pack(lp, (const float *)Lo.pk, n, d, LB.colmax, LB.scale, LB.lp, LB.ept, LB.eblk, c.s),
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
        g.queue = queue1 ? 1 : 0;
        g.counter = Lo.counter;
        g.lp_kind = lp;
        KC_CUDA(launch_gon(g, c.s), "mrg round 1 launch");
    }
    {
        TraceStep t("mrg_union", c.s);
        KC_CUDA(launch_mrg_union(Lo.c1, Lo.k1, m, k, Lo.U, Lo.nU, c.s), "union launch");
        KC_CUDA(launch_gather_pack(Lo.pk, c.o.dtype, d, Lo.U, Lo.nU, ucap, Lo.pkU, c.s), "gather launch");
        KC_CUDA(launch_mrg_round2_prep(Lo.inst2, proto, Lo.nU, k, c.s), "round 2 prep");
    }
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
        Lo.slots = cv.take<uint64_t>((size_t)keff_max * grid);
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
        const bool tcp = c.o.dtype == KC_F32 && tc_supported(d) && !(getenv("KC_PRUNE_TC") && !atoi(getenv("KC_PRUNE_TC")));
        Ptc.tc_at = nullptr;
        if (tcp) {   // tiles for up to n points of R and n centers of S
            Ptc.tc_at = cv.take<char>(tc_point_bytes(n, d));
            Ptc.tc_an = cv.take<float>((size_t)tc_point_rows(n));
            Ptc.tc_ae = cv.take<float>((size_t)tc_point_rows(n));
            Ptc.tc_bt = cv.take<char>(tc_center_bytes(n, d));
            Ptc.tc_cn = cv.take<float>((size_t)tc_center_tiles(n) * 256);
            Ptc.tc_ce = cv.take<float>((size_t)tc_center_tiles(n) * 256);
            Ptc.tc_maxes = cv.take<unsigned>(2);
            Ptc.tc_absmax = cv.take<unsigned>(1);
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

kc_status kc_gonzalez_batch(int32_t count, const void *const *pts, const int64_t *n, const int32_t *d,
                            const int32_t *k, int64_t *const *centers, int32_t *k_out, double *radii,
                            const kc_opts *opts) {
    g_err.clear();
    if (count < 1) return fail(KC_ERR_ARG, "count=%d must be >= 1", count);
    if (!pts || !n || !d || !k || !centers || !k_out || !radii) return fail(KC_ERR_ARG, "null pointer argument");
    for (int i = 0; i < count; ++i) {
        if (!pts[i] || !centers[i]) return fail(KC_ERR_ARG, "instance %d: null pointer", i);
        if (n[i] < 1 || n[i] > (int64_t)N_MAX) return fail(KC_ERR_ARG, "instance %d: n outside [1, 2^32-2]", i);
        if (d[i] < 1) return fail(KC_ERR_ARG, "instance %d: d must be >= 1", i);
        if (k[i] < 1) return fail(KC_ERR_ARG, "instance %d: k must be >= 1", i);
    }
    CallCtx c;
    kc_status r = begin(opts, c);
    if (r != KC_OK) return r;
    const bool dev_kout = is_device_ptr(k_out, c.dev);
    const bool dev_rad = is_device_ptr(radii, c.dev);
    std::vector<char> dev_pts((size_t)count), dev_cen((size_t)count);
    bool all_dev = dev_kout && dev_rad;
    int dmax = 0, dcommon = d[0];
    for (int i = 0; i < count; ++i) {
        dev_pts[i] = is_device_ptr(pts[i], c.dev);
        dev_cen[i] = is_device_ptr(centers[i], c.dev);
        all_dev = all_dev && dev_pts[i] && dev_cen[i];
        dmax = std::max(dmax, (int)d[i]);
        if (d[i] != dcommon) dcommon = 0;
    }
    if (c.async && !all_dev) return fail(KC_ERR_ARG, "KC_ASYNC needs device pointers for all arguments");
    const int dc = (dcommon == 3 || dcommon == 8 || dcommon == 32) && c.o.dtype == KC_F32 ? dcommon : 0;
    const int lp = lp_of(c.o);
    if (lp == KC_SWEEP_FP8)
        return fail(KC_ERR_ARG, "the batched form takes KC_SWEEP_F32 or KC_SWEEP_BF16 (fp8 needs per-instance scales)");

    // Longest processing time first: instances ordered by n * k * d.
    std::vector<int> order((size_t)count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const double wa = (double)n[a] * std::min<int64_t>(k[a], n[a]) * d[a];
        const double wb = (double)n[b] * std::min<int64_t>(k[b], n[b]) * d[b];
        return wa > wb;
    });

    const size_t esz = 4;
    struct Per {
        void *staging, *pk;
        uint32_t *mind;
        int64_t *cen;
        int32_t *range2;
        uint32_t *lpw;
        float *ept, *eblk, *cenT, *ecmax;
    };
    std::vector<Per> per((size_t)count);
    int32_t *kout_dev = nullptr;
    double *rad_dev = nullptr;
    uint64_t *fkeys = nullptr;
    int *counter = nullptr;
    PackSeg *segs_dev = nullptr;
    GonInst *insts_dev = nullptr;
    LpSeg *lsegs_dev = nullptr;
    size_t zero_bytes = 0;
    auto layout = [&](Carve &cv) {
        counter = cv.take<int>(1);
        for (int i = 0; i < count; ++i) per[i].range2 = cv.take<int32_t>(2);
        zero_bytes = cv.off;
        kout_dev = dev_kout ? k_out : cv.take<int32_t>((size_t)count);
        rad_dev = dev_rad ? radii : cv.take<double>((size_t)count);
        fkeys = cv.take<uint64_t>((size_t)count);
        segs_dev = cv.take<PackSeg>((size_t)count);
        insts_dev = cv.take<GonInst>((size_t)count);
        lsegs_dev = cv.take<LpSeg>(lp ? (size_t)count : 0);
        for (int i = 0; i < count; ++i) {
            const int64_t nbi = nblocks(n[i]);
            const int ki = (int)std::min<int64_t>(k[i], n[i]);
            per[i].staging = dev_pts[i] ? nullptr : cv.take<char>((size_t)n[i] * d[i] * esz);
            per[i].pk = cv.take<char>((size_t)nbi * BLK * d[i] * esz);
            per[i].mind = cv.take<uint32_t>((size_t)nbi * BLK);
            per[i].cen = dev_cen[i] ? centers[i] : cv.take<int64_t>((size_t)ki);
            if (lp) {
                per[i].lpw = cv.take<uint32_t>((size_t)nbi * lp_ngroups(lp, d[i]) * BLK);
                per[i].ept = cv.take<float>((size_t)nbi * BLK);
                per[i].eblk = cv.take<float>((size_t)nbi);
                per[i].cenT = cv.take<float>((size_t)ki * d[i]);
                per[i].ecmax = cv.take<float>(1);
            }
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

    // Descriptors: PackSeg[count], GonInst[count] and LpSeg[count] (LPT
    // order), contiguous in the arena, one upload.
    const size_t gi_off = (char *)insts_dev - (char *)segs_dev;
    const size_t ls_off = (char *)lsegs_dev - (char *)segs_dev;
    const size_t up_bytes = lp ? ls_off + sizeof(LpSeg) * count : gi_off + sizeof(GonInst) * count;
    std::vector<char> host(up_bytes + 256);
    PackSeg *hs = reinterpret_cast<PackSeg *>(host.data());
    GonInst *hg = reinterpret_cast<GonInst *>(host.data() + gi_off);
    LpSeg *hl = reinterpret_cast<LpSeg *>(host.data() + ls_off);
    int64_t blk0 = 0;
    for (int q = 0; q < count; ++q) {
        const int i = order[q];
        PackSeg &S = hs[q];
        memset(&S, 0, sizeof S);
        S.src = dev_pts[i] ? pts[i] : per[i].staging;
        S.dst = per[i].pk;
        S.range2 = per[i].range2;
        S.n = n[i];
        S.blk0 = blk0;
        S.d = d[i];
        if (lp) {
            LpSeg &Ls = hl[q];
            memset(&Ls, 0, sizeof Ls);
            Ls.pk = (const float *)per[i].pk;
            Ls.lp = per[i].lpw;
            Ls.ept = per[i].ept;
            Ls.eblk = per[i].eblk;
            Ls.n = n[i];
            Ls.blk0 = blk0;
            Ls.d = d[i];
        }
        blk0 += nblocks(n[i]);
        GonInst &I = hg[q];
        memset(&I, 0, sizeof I);
        I.pk = per[i].pk;
        I.mind = per[i].mind;
        I.slots = nullptr;
        I.centers = per[i].cen;
        I.k_out = kout_dev + i;
        I.final_key = fkeys + i;
        I.map = nullptr;
        I.range2 = per[i].range2;
        I.radius_out = rad_dev + i;
        I.lo = 0;
        I.n = n[i];
        I.base = 0;
        I.first = 0;
        I.d = d[i];
        I.k = (int)std::min<int64_t>(k[i], n[i]);
        I.cta0 = 0;
        I.G = 1;
        I.kcap = I.k;
        if (lp) {
            I.lp = per[i].lpw;
            I.eblk = per[i].eblk;
            I.ept = per[i].ept;
            I.scale = nullptr;
            I.cenT = per[i].cenT;
            I.ecmax_out = per[i].ecmax;
            I.lp_kind = lp;
        }
    }
    KC_CUDA(cudaMemsetAsync(c.arena->dev, 0, zero_bytes, c.s), "scratch clear");
    for (int i = 0; i < count; ++i)
        if (!dev_pts[i])
            KC_CUDA(cudaMemcpyAsync(per[i].staging, pts[i], (size_t)n[i] * d[i] * esz, cudaMemcpyHostToDevice, c.s),
                    "copy points to device");
    r = upload(c.arena, c.s, host.data(), up_bytes, segs_dev);
    if (r != KC_OK) return r;
    {
        TraceStep t("pack", c.s);
        KC_CUDA(launch_pack_many(segs_dev, count, blk0, c.o.dtype, st, c.s), "pack launch");
        if (lp) KC_CUDA(launch_lp_pack_many(lsegs_dev, count, blk0, c.s), "low-precision pack");
    }
    {
        TraceStep t("gonzalez_batch", c.s);
        GonArgs g{};
        g.insts = insts_dev;
        g.ninst = count;
        g.dtype = c.o.dtype;
        g.dc = dc;
        g.dmax = dmax;
        g.st = st;
        g.timeout_cycles = timeout_cycles(c.o);
        g.grid = std::min(gon_queue_grid(c.o.dtype, dc, lp), count);
        g.queue = 1;
        g.counter = counter;
        g.lp_kind = lp;
        KC_CUDA(launch_gon(g, c.s), "batch launch");
    }
    {
        TraceStep t("radius_batch", c.s);
        KC_CUDA(launch_batch_radius(insts_dev, count, c.o.dtype, st, c.s), "batch radius launch");
    }
    for (int i = 0; i < count; ++i)
        if (!dev_cen[i])
            KC_CUDA(cudaMemcpyAsync(centers[i], per[i].cen, (size_t)std::min<int64_t>(k[i], n[i]) * sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, c.s),
                    "copy centers out");
    if (!dev_kout)
        KC_CUDA(cudaMemcpyAsync(k_out, kout_dev, (size_t)count * sizeof(int32_t), cudaMemcpyDeviceToHost, c.s),
                "copy k_out");
    if (!dev_rad)
        KC_CUDA(cudaMemcpyAsync(radii, rad_dev, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost, c.s),
                "copy radii");
    if (c.async) return KC_OK;
    return finish(c.arena, c.s);
}

}  // extern "C"
