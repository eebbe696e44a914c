// kc_internal.cuh -- device helpers and internal launch interfaces shared by
// the CUDA translation units of the library (not part of the public ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/kcenter.h"

namespace kc {

// Points are repacked into blocks of BLK points, coordinate-major inside a
// block ("AoSoA"): element (point i, coordinate j) sits at
//   ((i / BLK) * d + j) * BLK + i % BLK.
// A warp streams one block: lane l owns points 4l..4l+3 and reads them with
// one 16-byte load per coordinate, so every warp load is 512 contiguous bytes.
constexpr int BLK = 128;
constexpr uint32_t N_MAX = 0xFFFFFFFEu;

__host__ __device__ inline int64_t nblocks(int64_t n) { return (n + BLK - 1) / BLK; }
__host__ __device__ inline int64_t pk_index(int64_t i, int64_t j, int d) {
    return ((i / BLK) * d + j) * BLK + (i % BLK);
}
// Coordinate j of float point i: from the packed array, or the row-major
// one when pk is null.
__device__ __forceinline__ float point_at(const float *__restrict__ pk, const float *__restrict__ rm, int64_t i, int j,
                                          int d) {
    return pk ? pk[pk_index(i, j, d)] : rm[i * d + j];
}


// A count that an earlier kernel writes on the device (e.g. k_out), clamped
// to [0, cap]: after a kernel that gave up (a timeout) the word may still
// hold whatever the caller's buffer held, and no later kernel may index past
// the `cap` entries its buffers were sized for.
__device__ __forceinline__ int64_t dev_count(const int32_t *cnt_dev, int64_t cap) {
    if (!cnt_dev) return cap;
    const int64_t v = *cnt_dev;
    return v < 0 ? 0 : (v > cap ? cap : v);
}

// Device status word (first error wins).
struct DevStatus {
    int32_t code;
    int32_t where;
    int64_t info;
};

__device__ __forceinline__ void set_status(DevStatus *st, int code, int where, int64_t info) {
    if (atomicCAS(&st->code, 0, code) == 0) {
        st->where = where;
        st->info = info;
    }
}

// ------------------------------------------------------- checked build
// Compiled with -DKC_CHECKS (a separate library, libkcenter_checks.so, built
// by build.build(checks=True)), kernels test the indices they are about to
// use against the extent of the buffer they address and, on a miss, record
// KC_ERR_BOUNDS (where = the site, info = the index) and skip the access
// instead of making it.  This stands in for compute-sanitizer where that tool
// is not available.  In the regular build the test is the constant true.
#ifdef KC_CHECKS
__device__ __forceinline__ bool kc_in_range(DevStatus *st, int64_t i, int64_t extent, int where) {
    if (i >= 0 && i < extent) return true;
    set_status(st, KC_ERR_BOUNDS, where, i);
    return false;
}
#define KC_IN_RANGE(st, i, extent, where) kc::kc_in_range((st), (int64_t)(i), (int64_t)(extent), (where))
#else
#define KC_IN_RANGE(st, i, extent, where) true
#endif
// Sites of the checked build (DevStatus.where).
enum {
    KC_AT_CENTER_LOAD = 11,   // a GON winner's index, before its coordinates are read
    KC_AT_RESIDENT_SMEM = 12, // a resident kernel's shared-memory column
    KC_AT_CANDIDATE = 13,     // a mixed-precision candidate buffer entry
    KC_AT_RECHECK = 14,       // a point index of an exact recheck
    KC_AT_CENTER_COPY = 15,   // a center slot of the transposed FP32 center copy
    KC_AT_EIM_INDEX = 16,     // an index into the points in EIM's kernels
    KC_AT_RADIUS_LIST = 17,   // an entry of the radius recheck's point list
    KC_AT_SLOT = 18           // a GON exchange slot
};

// ---------------------------------------------------------------- keys
// A 64-bit argmax key: the 32-bit value (float bits of a non-negative float,
// which order like unsigned integers, or an unsigned integer) in the high
// word and 0xFFFFFFFF - index in the low word.  The unsigned maximum of keys
// is the largest value, lowest index among equals.  Real points have keys
// >= 1 because index <= N_MAX.
__device__ __forceinline__ uint64_t make_key(uint32_t v, uint32_t idx) {
    return ((uint64_t)v << 32) | (uint64_t)(0xFFFFFFFFu - idx);
}
__device__ __forceinline__ uint32_t key_idx(uint64_t k) { return 0xFFFFFFFFu - (uint32_t)k; }
__device__ __forceinline__ uint32_t key_val(uint64_t k) { return (uint32_t)(k >> 32); }

__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = umax64(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int32_t ld_volatile_i32(const int32_t *p) {
    return *(const volatile int32_t *)p;
}

// ------------------------------------------------------- squared distance
// Canonical FP32 term: t = x - c rounded to float, acc = fma(t, t, acc).
// Zero-padded coordinates (x = c = 0) leave acc unchanged, so padding never
// alters the value.
__device__ __forceinline__ float sq_step(float acc, float x, float c) {
    float t = __fsub_rn(x, c);
    return __fmaf_rn(t, t, acc);
}
// Exact int32 term in 32-bit unsigned arithmetic (the caller guarantees
// d * range^2 < 2^32, so neither the difference nor the sum wraps).
__device__ __forceinline__ uint32_t sq_step(uint32_t acc, int32_t x, int32_t c) {
    uint32_t t = (uint32_t)(x - c);
    return acc + t * t;
}

// Canonical FP32 squared distance of float point i (packed, or row-major when
// pk is null) and the center row c.  v4: d % 4 == 0, c 16-byte aligned and
// (row-major) rm too; the center row, which differs between the lanes of a
// warp, is then read with 16-byte loads (a quarter of the L1 wavefronts).
__device__ __forceinline__ float point_row_dist(const float *__restrict__ pk, const float *__restrict__ rm, int64_t i,
                                                int d, const float *__restrict__ c, bool v4) {
    float acc = 0.f;
    if (v4) {
        const float4 *c4 = reinterpret_cast<const float4 *>(c);
        const float4 *x4 = pk ? nullptr : reinterpret_cast<const float4 *>(rm + i * d);
        for (int q = 0; q < d / 4; ++q) {
            const float4 cc = c4[q];
            float4 xx;
            if (x4) {
                xx = x4[q];
            } else {
                xx.x = pk[pk_index(i, 4 * q, d)];
                xx.y = pk[pk_index(i, 4 * q + 1, d)];
                xx.z = pk[pk_index(i, 4 * q + 2, d)];
                xx.w = pk[pk_index(i, 4 * q + 3, d)];
            }
            acc = sq_step(acc, xx.x, cc.x);
            acc = sq_step(acc, xx.y, cc.y);
            acc = sq_step(acc, xx.z, cc.z);
            acc = sq_step(acc, xx.w, cc.w);
        }
    } else {
        for (int j = 0; j < d; ++j) acc = sq_step(acc, point_at(pk, rm, i, j, d), c[j]);
    }
    return acc;
}

template <typename T> struct AccOf;
template <> struct AccOf<float> { using type = float; };
template <> struct AccOf<int32_t> { using type = uint32_t; };

__device__ __forceinline__ uint32_t acc_bits(float a) { return __float_as_uint(a); }
__device__ __forceinline__ uint32_t acc_bits(uint32_t a) { return a; }

// int32 exactness check: d * (max - min)^2 < 2^32, where range2 holds the
// pack kernel's order-preserving maxima of ~bias(v) and bias(v).
__device__ __forceinline__ bool int_range_ok(const int32_t *range2, int d) {
    const uint32_t *r = (const uint32_t *)range2;
    const int64_t mn = (int64_t)(int32_t)((0xFFFFFFFFu - r[0]) ^ 0x80000000u);
    const int64_t mx = (int64_t)(int32_t)(r[1] ^ 0x80000000u);
    const uint64_t span = (uint64_t)(mx - mn);
    if (span >= 65536u) return false;
    return (uint64_t)d * span * span < (1ull << 32);
}

// FP64 squared distance in coordinate order, separate multiply and add.
__device__ __forceinline__ double sq_step64(double acc, float x, float c) {
    double t = __dsub_rn((double)x, (double)c);
    return __dadd_rn(acc, __dmul_rn(t, t));
}

// Relative error bound of the canonical FP32 squared distance against the
// exact value: (d + 2) u / (1 - (d + 2) u), u = 2^-24 (one rounding in the
// difference, squared, and one per accumulation).
__host__ __device__ inline double f32_gamma(int d) {
    const double u = 5.9604644775390625e-08;
    const double m = (double)(d + 2) * u;
    return m / (1.0 - m);
}

// --------------------------------------------------------- launchers
// Every launcher reports the number of kernels it launched (tracing and the
// process-wide launch counter).
void note_launches(int kernels);

// Repack row-major points into the AoSoA layout (zero padding), checking
// finiteness (float) or accumulating the coordinate range (int32).
cudaError_t launch_pack(const void *src, int dtype, int64_t n, int d, void *dst, int32_t *range2,
                        DevStatus *st, cudaStream_t s);
// int32 only: record KC_ERR_RANGE unless squared distances fit 32 bits.
cudaError_t launch_range_check(const int32_t *range2, int d, DevStatus *st, cudaStream_t s);

// One Gonzalez instance solved by a group of CTAs [cta0, cta0 + G) of a
// persistent launch.  Indices inside an instance are local (0..n-1); the
// centers written out are base + local index (or map[local] when map is set).
struct GonInst {
    const void *pk;          // packed points of this instance (block aligned)
    // per-step counters of the group's shared tail of blocks ([k], zeroed),
    // or nullptr: every block stays with its CTA (FP32 group kernels only)
    int *tail;
    // FP32 rows of the instance's points, row of local index 0 (row-major,
    // d floats per row), or nullptr: the exact rechecks of the mixed-precision
    // sweep then read the packed copy (one point's coordinates 512 bytes
    // apart) instead of one contiguous row
    const float *rm;
    uint32_t *mind;          // [nblocks(n) * BLK] running minimum (value bits)
    uint64_t *slots;         // [k * G] per-step, per-CTA argmax keys (zeroed)
    int64_t *centers;        // [k] out
    int32_t *k_out;          // out
    uint64_t *final_key;     // out: key of the largest final minimum
    const int64_t *map;      // optional local -> global index map (nullptr: base + local)
    const int32_t *range2;   // int32 only: [min, max] coordinate maxima of the pack
    double *radius_out;      // batched form: this instance's covering radius
    // mixed-precision sweep (lp_kind != 0): low-precision words of the same
    // packed array, per-block error bounds (indexed like blocks of pk),
    // per-point bounds, fp8 column scales, the selected centers' FP32
    // coordinates transposed ([d][kcap]) and the largest center bound (out)
    const uint32_t *lp;
    const float *eblk;
    const float *ept;
    const float *scale;
    float *cenT;
    float *ecmax_out;
    // exact FP32 memo of the recheck, per point of the packed array: m32 is
    // the canonical minimum over centers [0, stamp) (stamp zeroed by the
    // low-precision pack), so a recheck evaluates only the newer centers
    uint32_t *m32;
    uint32_t *stamp;
    int32_t lp_kind;
    int32_t kcap;
    int64_t lo;              // first point of the range in the packed array
    int64_t n;
    int64_t base;
    int64_t first;           // local index of the first center
    int32_t d;
    int32_t k;
    int32_t cta0;
    int32_t G;
};

struct GonArgs {
    GonInst single;          // used when insts == nullptr
    const GonInst *insts;    // device array [ninst], sorted by cta0 (group mode)
    int ninst;
    int dtype;
    int dc;                  // common d for the compile-time specialisation (0 = mixed)
    int dmax;                // largest d of any instance (shared-memory size)
    DevStatus *st;
    long long timeout_cycles;
    int grid;                // CTAs
    int queue;               // 1: one CTA per instance, instances taken from *counter
    int *counter;            // queue mode: next instance (zeroed)
    int nheavy;              // queue mode: insts[0, nheavy) are solved by CTA groups first
    int gheavy;              // queue mode: CTAs of those groups (the first gheavy of the grid)
    int lp_kind;             // 0: FP32 sweep; KC_SWEEP_BF16 / _FP16 / _FP8 (float points)
    // mixed-precision sweep of a CTA group: 1 = each CTA filters its exact
    // rechecks against its own largest lower bound (no extra exchange per
    // step); 0 = the group first exchanges the CTAs' bounds and filters
    // against the group's largest
    int lp_local_t;
    // testing hook (KC_TEST_WITHHOLD): 1 + the step at which the last CTA of
    // a group does not publish its exchange slot, so that the group's waits
    // run out of their budget; 0 = never
    int withhold;
    // testing hook of the checked build (KC_TEST_BAD_INDEX): the first
    // winner index is replaced by one past the instance; 0 = never
    int bad_index;
    // FP32 group kernels of large instances: the instantiation that claims
    // blocks and shares the tail (gon_solve's DYN); 0 = the plain loop
    int dyn;
    // resident form (single instance, gon_resident_kernel): points per
    // coordinate held in each CTA's shared memory; 0 = the streaming kernels
    int res_cap;
};
cudaError_t launch_gon(GonArgs &a, cudaStream_t s);
// Resident form for one instance of n points (row-major rows in device
// memory): the grid (0 when the instance does not fit on chip or d has no
// specialisation), with the shared-memory columns per coordinate in *cap and
// the exchange-slot words per (step, CTA) in *slot_words.
int gon_resident_plan(int dtype, int d, int64_t n, int *cap, int *slot_words);
// Mixed-precision diagnostics (synchronous): exact rechecks, overflows.
cudaError_t read_counters(unsigned long long out[8], bool reset);
int gon_max_grid(int dtype, int d, int lp = 0);
int gon_queue_grid(int dtype, int d, int lp = 0);
int gon_threads();
// SM clock rate of a device in kHz (queried once per device: the query
// costs a few hundred microseconds on some hosts).
int device_clock_khz(int dev);
// Exchange slots: per step a row of G 8-byte words (one per CTA of the
// group); words for k steps, twice that for the mixed-precision sweep (keys,
// then the CTAs' lower bounds).
__host__ __device__ inline int64_t slot_stride(int G) { return (int64_t)G; }
inline int64_t slot_words(int64_t k, int G, bool lp) { return k * slot_stride(G) * (lp ? 2 : 1); }
int gon_queue_warps();
int gon_warps_per_cta();

// Arguments for plain GON: one instance over the whole packed array, solved
// by all `grid` CTAs.
inline void gon_single(GonArgs &g, const void *pk, int dtype, int64_t n, int d, int k, int64_t first,
                       uint32_t *mind, uint64_t *slots, int64_t *centers, int32_t *k_out,
                       uint64_t *final_key, const int32_t *range2, int grid) {
    GonInst &I = g.single;
    I.pk = pk;
    I.tail = nullptr;
    I.rm = nullptr;
    I.mind = mind;
    I.slots = slots;
    I.centers = centers;
    I.k_out = k_out;
    I.final_key = final_key;
    I.map = nullptr;
    I.range2 = range2;
    I.radius_out = nullptr;
    I.lp = nullptr;
    I.eblk = nullptr;
    I.ept = nullptr;
    I.scale = nullptr;
    I.cenT = nullptr;
    I.ecmax_out = nullptr;
    I.m32 = nullptr;
    I.stamp = nullptr;
    I.lp_kind = 0;
    I.kcap = k;
    I.lo = 0;
    I.n = n;
    I.base = 0;
    I.first = first;
    I.d = d;
    I.k = k;
    I.cta0 = 0;
    I.G = grid;
    g.insts = nullptr;
    g.ninst = 1;
    g.dtype = dtype;
    g.dc = d;
    g.dmax = d;
    g.grid = grid;
    g.queue = 0;
    g.counter = nullptr;
    g.lp_kind = 0;
    g.lp_local_t = 0;
}

// Bounds on sqrt(m32) from the approximate minimum m~ (value bits), the
// absolute slack delta = e_x + E and opg = 1 + g, omg = 1 - g (see the
// mixed-precision sweep in kc_gon.cu); directed rounding keeps them sound.
__device__ __forceinline__ float lp_upper(uint32_t mbits, float delta, float opg) {
    const float r = __fsqrt_ru(__uint_as_float(mbits));
    return __fmul_ru(opg, __fadd_ru(__fmul_ru(r, opg), delta));
}
__device__ __forceinline__ float lp_lower(uint32_t mbits, float delta, float omg) {
    const float r = __fsqrt_rd(__uint_as_float(mbits));
    return __fmul_rd(omg, __fsub_rd(__fmul_rd(r, omg), delta));
}
__host__ __device__ inline float lp_slack(int d) { return (float)(f32_gamma(d) + 0x1p-20); }

// --------------------------------------------- low-precision sweep data
// Coordinates per 32-bit word of the low-precision copy (bf16, fp16: 2;
// fp8: 4).
__host__ __device__ constexpr int lp_group(int kind) { return kind == KC_SWEEP_FP8 ? 4 : 2; }
__host__ __device__ inline int lp_ngroups(int kind, int d) { return (d + lp_group(kind) - 1) / lp_group(kind); }
// Build the low-precision copy of a packed FP32 array: words `lp`
// [nblocks*ng*BLK], per-point bounds `ept` [nblocks*BLK], per-block maxima
// `eblk` [nblocks]; fp8 also fills `scale` [ng*4] from the column maxima
// (`colmax` [d] scratch).
// stamp ([nblocks(n) * BLK]) is zeroed: the recheck memo starts empty.
cudaError_t launch_lp_pack(int kind, const float *pk, int64_t n, int d, unsigned *colmax, float *scale, uint32_t *lp,
                           float *ept, float *eblk, uint32_t *stamp, cudaStream_t s);
// bf16 copies of many packed arrays (batched form).
struct LpSeg {
    const float *pk;
    uint32_t *lp;
    float *ept;
    float *eblk;
    uint32_t *stamp;
    int64_t n;
    int64_t blk0;
    int32_t d;
    int32_t pad;
};
cudaError_t launch_lp_pack_many(const LpSeg *segs, int nseg, int64_t total_blocks, cudaStream_t s);

// ------------------------------------------------ MRG and batched helpers
// One row-major array to pack; its blocks are [blk0, blk0 + nblocks(n)) of
// the launch.
struct PackSeg {
    const void *src;
    void *dst;
    int32_t *range2;         // int32: this array's coordinate range (zeroed)
    int64_t n;
    int64_t blk0;
    int32_t d;
    int32_t pad;
};
cudaError_t launch_pack_many(const PackSeg *segs, int nseg, int64_t total_blocks, int dtype, DevStatus *st,
                             cudaStream_t s);
cudaError_t launch_mrg_union(const int64_t *c1, const int32_t *k1, int m, int k, int64_t *U, int64_t *nU,
                             cudaStream_t s);
cudaError_t launch_gather_pack(const void *pk, int dtype, int d, const int64_t *U, const int64_t *nU,
                               int64_t cap, void *out, cudaStream_t s);
cudaError_t launch_mrg_round2_prep(GonInst *inst, const GonInst &proto, const int64_t *nU, int kmax,
                                   cudaStream_t s);
cudaError_t launch_batch_radius(const GonInst *insts, int ninst, int dtype, const DevStatus *st,
                                cudaStream_t s);

// ------------------------------------------------------------------ EIM
cudaError_t launch_eim_iota(uint32_t *R, int64_t n, cudaStream_t s);
cudaError_t launch_eim_sample(const uint32_t *R, int64_t rn, uint64_t seed, int it, double pS, double pH,
                              uint8_t *inS, uint32_t *S, unsigned long long *sn, uint32_t *H, unsigned long long *hn,
                              int64_t hcap, DevStatus *st, cudaStream_t s);
cudaError_t launch_eim_gather_rows(const void *src, int dtype, int d, const uint32_t *idx, int64_t from, int64_t to,
                                   void *out, cudaStream_t s);
cudaError_t launch_eim_dist_hs(int dtype, const void *Hc, int64_t hn, const void *Sc, int64_t sn, int d, uint32_t *dH,
                               cudaStream_t s);
cudaError_t launch_eim_select(const uint32_t *H, const uint32_t *dH, int64_t hn, int64_t p, uint32_t *thr, uint32_t *v,
                              cudaStream_t s);
cudaError_t launch_eim_prune(int dtype, const void *src, int d, const uint32_t *R, int64_t rn, const uint8_t *inS,
                             const void *Sc, int64_t sn, const uint32_t *thr, uint32_t *Rn, unsigned long long *rnn,
                             cudaStream_t s);
cudaError_t launch_eim_drop_sampled(const uint32_t *R, int64_t rn, const uint8_t *inS, uint32_t *Rn,
                                    unsigned long long *rnn, cudaStream_t s);
cudaError_t launch_eim_mark(const uint32_t *R, int64_t rn, uint8_t *mask, cudaStream_t s);
cudaError_t launch_compact(const uint8_t *mask, int64_t n, int *counts, int64_t *offs, int64_t *out, int64_t *total,
                           cudaStream_t s);

struct RadiusArgs {
    const void *pk;
    // float points may come row-major instead ([n][d], pk null): on the
    // tensor-core path, the CUDA-core minimum for d <= 16, and the rechecks;
    // nothing is packed, the coordinates are read in place
    const float *rm;
    int dtype;
    int64_t n;
    int d;
    const int64_t *centers;  // [kc_max] device indices
    const int32_t *kc_dev;   // device count (nullptr: use kc_max)
    int kc_max;
    void *cen;               // scratch [kc_max * d] gathered center coordinates (16-byte aligned)
    uint32_t *mind;          // [nblocks*BLK] values (input if have_mind)
    unsigned long long *key32;   // argmax key of mind (input if have_mind)
    unsigned long long *max64;   // scratch
    unsigned long long *arg64;   // scratch
    double *m64;             // scratch [n] FP64 values of flagged points
    double *radius_out;      // device out
    int64_t *argmax_out;     // device out (may be null)
    DevStatus *st;
    bool have_mind;          // mind/key32 already hold the FP32 minima
    // set when mind holds a mixed-precision sweep's approximate minima: the
    // flag test then uses the upper bound U(x) (eblk per block, *ecmax)
    const float *eblk;
    const float *ecmax;
    // fp16 sweep: the device word holding its power-of-two scale (the
    // bounds above are in the scaled units); nullptr = 1
    const float *lpscale;
    // tensor-core filter scratch (float points, d <= 128); tc_at null: CUDA cores
    void *tc_at, *tc_bt;
    float *tc_an, *tc_ae, *tc_cn, *tc_ce, *tc_mlo, *tc_mhi;
    unsigned *tc_maxes, *tc_absmax, *tc_mlomax;
    uint8_t *tc_rin;         // prune only: per point row, 1 when the point is in S
    // radius: the points that can reach the maximum ([n] slots and their
    // count); the FP64 recheck then visits only these
    uint32_t *tc_flist;
    unsigned long long *tc_fcount;
    // float points: with these set (flagged: [n] slots; flagged_n and done
    // zeroed before the launch) the FP64 recheck, the argmax and the result
    // are one launch (recheck_kernel); null: three launches
    uint32_t *flagged;
    unsigned *flagged_n, *done;
};

// ------------------------------------------------- tensor-core blocks
// Scratch of one tensor-core block: fp16 point tiles (at) with norms and
// bounds, fp16 center tiles (bt) with norms and bounds, their maxima, the
// coordinate maximum that fixes the scale, and the radius outputs.
struct TcBufs {
    void *at, *bt;
    float *an, *ae, *cn, *ce;
    unsigned *maxes, *absmax;
    float *mlo, *mhi;
    unsigned *mlomax;
    uint8_t *rin;   // prune: per point row, 1 when the point is in S (null for the radius)
    uint32_t *flist;              // radius: points that can reach the maximum
    unsigned long long *fcount;   // and their count
};
inline TcBufs tc_bufs(const RadiusArgs &a) {
    return TcBufs{a.tc_at, a.tc_bt, a.tc_an, a.tc_ae, a.tc_cn, a.tc_ce, a.tc_maxes, a.tc_absmax, a.tc_mlo, a.tc_mhi,
                  a.tc_mlomax, a.tc_rin, a.tc_flist, a.tc_fcount};
}
bool tc_supported(int d);
cudaError_t read_tc_counters(unsigned long long out[6], bool reset);
int tc_center_tiles(int64_t kc);
size_t tc_center_bytes(int64_t kc, int d);
size_t tc_point_bytes(int64_t n, int d);
int64_t tc_point_rows(int64_t n);
cudaError_t launch_tc_absmax(const float *pk, int64_t n, int d, unsigned *absmax, cudaStream_t s);
// Points from the packed array pk, or (pk null) from the row-major array rm,
// which is then also checked as the pack would (NaN/Inf, magnitude).
cudaError_t launch_tc_radius(const float *pk, const float *rm, int64_t n, int d, const float *cen,
                             const int32_t *kc_dev, int kc, const TcBufs &B, uint32_t *mind,
                             unsigned long long *key32, DevStatus *st, cudaStream_t s);
// Deferred exact checks of the tensor-core prune: the (row, center) pairs
// its bounds leave undecided, per-row flags, the rows they decide, and the
// counters of both lists.  pairs holds pcap entries; rows beyond it get a
// full exact scan instead.  flag and hit hold one byte per row of R.
struct PruneBufs {
    uint2 *pairs;
    int64_t pcap;
    uint8_t *flag, *hit;
    uint32_t *pend;
    unsigned long long *npairs, *npend;
};
// B.absmax must already hold the coordinate maximum over a superset of R and S.
cudaError_t launch_tc_prune(const float *src, int d, const uint32_t *R, int64_t rn, const uint8_t *inS, const float *Scen,
                            int64_t sn, const TcBufs &B, const PruneBufs &P, const uint32_t *thr, uint32_t *Rn,
                            unsigned long long *rnn, DevStatus *st, cudaStream_t s);
cudaError_t launch_radius(RadiusArgs &a, cudaStream_t s);

}  // namespace kc
