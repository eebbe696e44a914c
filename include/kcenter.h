/*
 * kcenter.h -- C ABI of the GB300 k-center library.
 *
 * The library computes the k-center method of McClintock & Wirth, "Efficient
 * Parallel Algorithms for k-Center Clustering" (arXiv 1604.03228): pick at
 * most k of the n input points as centers so that the largest distance from
 * any point to its nearest center (the covering radius) is small.  Its hot
 * path is the farthest-point step of Gonzalez's algorithm (Section 3.1): the
 * distance from every point to the newest center, a running minimum, and a
 * global argmax with the lowest index winning ties.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Points are row-major n x d (point i's coordinates at pts[i*d .. i*d+d-1]),
 *    float32 (KC_F32) or int32 (KC_I32) as opts->dtype says.  The distance is
 *    Euclidean; squared distances are compared and a radius is returned as a
 *    distance (square root) in double.
 *  - Every pointer may be host memory (pageable or pinned) or device memory
 *    of the current CUDA device; the library tells them apart with
 *    cudaPointerGetAttributes and copies host inputs in and host outputs out
 *    itself.  The caller owns all memory it passes; the library never frees
 *    it.  Scratch memory is allocated by the library on first use, cached per
 *    (device, stream) and released by kc_release().
 *  - Calls are ordered on opts->stream (a cudaStream_t; NULL = the legacy
 *    default stream).  Without KC_ASYNC a call waits for its work and returns
 *    the final status.  With KC_ASYNC (all pointers must then be device
 *    pointers) a call only enqueues work; errors found on the device are kept
 *    in a status word that kc_sync() returns.
 *  - Selection is exact for int32 points (squared distances in 32-bit
 *    unsigned arithmetic, which the library checks is exact: d * (max - min)^2
 *    must be below 2^32, else KC_ERR_RANGE).  For float32 points every argmax
 *    is taken on the canonical FP32 squared distance: for j = 0..d-1,
 *    t = x_j - c_j rounded to float, acc = fma(t, t, acc) from acc = 0.  The
 *    returned radius is then recomputed in FP64 (coordinates widened, terms
 *    summed in coordinate order without fused multiply-add) for the point(s)
 *    that can reach the maximum, so it equals the plain FP64 covering radius
 *    of the chosen centers.
 *  - Ties between equally far points go to the lowest point index.  When
 *    every point is at distance 0 from the chosen centers, selection stops
 *    early and *k_out < k ("at most k centers", Section 1.1).
 *  - n must be in [1, 2^32 - 2]; d >= 1; k >= 1.  Non-finite float
 *    coordinates give KC_ERR_NONFINITE.  Spin-waits inside persistent kernels
 *    give up after a time budget and return KC_ERR_TIMEOUT; nothing traps.
 *  - Every failure is a status code; kc_last_error() describes the last one
 *    on the calling thread.  No function aborts the process.
 *
 * Environment (tuning and testing; none of these changes a result)
 * ----------------------------------------------------------------
 *  KC_RADIUS_TC=0|1          covering radius on CUDA cores / on the tensor-core
 *                            blocks (default: tensor cores for float points
 *                            with d <= 128 when k * d >= 8192, or when
 *                            k * d >= 1536 and n >= 262144)
 *  KC_PRUNE_TC=0|1           EIM prune on CUDA cores / tensor cores (default:
 *                            tensor cores for float points, 16 <= d <= 128,
 *                            |S| >= 256)
 *  KC_TC_STREAM_CENTERS=1    tensor-core blocks stream the center tiles through
 *                            a two-stage ring even when all of them fit in
 *                            shared memory
 *  KC_TC_PAIR=0              streamed center tiles feed one point tile each
 *                            (default: two, for d <= 93)
 *  KC_PRUNE_PAIR_CAP=N       capacity of the tensor-core prune's buffer of
 *                            undecided pairs (rows past it get a full exact
 *                            scan)
 *  KC_GON_GRID=G             CTAs of a single Gonzalez launch (clamped to the
 *                            co-resident maximum)
 *  KC_GON_RESIDENT=0         single FP32 / int32 Gonzalez instances always
 *                            stream their points (default: held on chip when
 *                            they fit, d = 8 or 10)
 *  KC_GON_RESIDENT_PTS=P     points per CTA the resident form aims for
 *                            (default 4096)
 *  KC_GON_TAIL=0             no shared tail of blocks in large streaming FP32
 *                            Gonzalez launches
 *  KC_LP_LOCAL_T=1           mixed-precision sweeps recheck against each CTA's
 *                            own bound instead of the group's
 *  KC_BATCH_THETA=x|inf      the batch split of kc_gonzalez_batch and batch
 *                            plans (see there); overrides the tuned value
 */
#ifndef KCENTER_H
#define KCENTER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KC_OK = 0,
    KC_ERR_ARG = 1,        /* invalid argument (sizes, indices, flags) */
    KC_ERR_CUDA = 2,       /* a CUDA runtime call failed */
    KC_ERR_OOM = 3,        /* device scratch allocation failed */
    KC_ERR_TIMEOUT = 4,    /* a device spin-wait ran out of its time budget */
    KC_ERR_RANGE = 5,      /* int32 squared distances would not fit 32 bits */
    KC_ERR_NONFINITE = 6,  /* a float coordinate is NaN or infinite */
    KC_ERR_BOUNDS = 7      /* checked build only (libkcenter_checks.so, compiled with
                              -DKC_CHECKS): a kernel found an index outside the
                              buffer it was about to address and skipped the access */
} kc_status;

typedef enum { KC_F32 = 0, KC_I32 = 1 } kc_dtype;

/*
 * Storage precision of the Gonzalez sweep for float points (kc_opts.sweep).
 * KC_SWEEP_BF16 / KC_SWEEP_FP16 / KC_SWEEP_FP8 stream a bf16 (or fp16 with
 * one power-of-two scale for all coordinates, chosen from the largest
 * magnitude so that nothing overflows; or fp8 e4m3 with a per-column scale
 * max|x_j| / 448) copy of the points and keep, per point, an error bound
 * e_x >= ||decoded(x) - x||_2.  Every candidate whose low-precision distance
 * could reach the step's maximum is recomputed in canonical FP32 from the
 * FP32 points, so the selected centers, k_out and radius are identical to
 * KC_SWEEP_F32.  fp16 streams as many bytes as bf16 with 3 more mantissa
 * bits, so far fewer candidates need the recheck.  Ignored for int32 points.
 */
typedef enum { KC_SWEEP_F32 = 0, KC_SWEEP_BF16 = 1, KC_SWEEP_FP8 = 2, KC_SWEEP_FP16 = 3 } kc_sweep;

/* Flags for kc_opts.flags. */
#define KC_ASYNC 1u        /* enqueue only; see kc_sync() */
#define KC_AUTOTUNE 2u     /* batched form only: time launch shapes, keep the fastest */
/* Testing only (kc_gonzalez): in the first step the last CTA of the launch
 * does not publish its exchange slot, so every CTA's wait for the step's
 * slots runs out of its budget (kc_opts.timeout_ms) and the call returns
 * KC_ERR_TIMEOUT.  Exercises the abort path of the persistent kernel
 * without faulting or hanging the GPU; has no effect when the launch has a
 * single CTA (no exchange). */
#define KC_TEST_WITHHOLD 0x80000000u
/* Testing only, checked build only (kc_gonzalez; the regular build rejects
 * it with KC_ERR_ARG): the first winner's index is replaced by one past the
 * last point, so that the kernel's own check records KC_ERR_BOUNDS instead
 * of reading past the points.  Selects the streaming kernel. */
#define KC_TEST_BAD_INDEX 0x40000000u

typedef struct {
    int32_t dtype;          /* kc_dtype of the points */
    uint32_t flags;         /* KC_ASYNC, KC_AUTOTUNE (batched form) or 0 */
    int32_t sweep;          /* kc_sweep (float points only) */
    int32_t reserved;       /* must be 0 */
    uint64_t seed;          /* EIM sampling seed */
    double phi;             /* EIM Select parameter (Section 4.2); <= 0 means 6 */
    void *stream;           /* cudaStream_t, NULL = legacy default stream */
    int64_t timeout_ms;     /* device spin-wait budget; <= 0 means 2000 ms */
} kc_opts;

/*
 * kc_gonzalez -- GON, Section 3.1 (the factor-2 greedy of Gonzalez): start
 * from point `first`, then repeatedly add the point farthest from the centers
 * chosen so far, until k centers exist.  Cost O(k n) distance evaluations
 * (Section 5.1).
 *   pts      [n*d] points (see conventions); read only.
 *   first    index of the first center, 0 <= first < n.
 *   centers  [k] int64 out: chosen point indices in selection order; entries
 *            past *k_out are left untouched.
 *   k_out    int32 out: number of centers chosen (k, or fewer on early stop).
 *   radius   double out: covering radius of the chosen centers over all points.
 * Errors: KC_ERR_ARG for bad sizes or `first`; KC_ERR_RANGE, KC_ERR_NONFINITE,
 * KC_ERR_TIMEOUT, KC_ERR_OOM, KC_ERR_CUDA as above.  Outputs are undefined on
 * error.
 */
kc_status kc_gonzalez(const void *pts, int64_t n, int32_t d, int32_t k, int64_t first,
                      int64_t *centers, int32_t *k_out, double *radius, const kc_opts *opts);

/*
 * kc_radius -- covering radius of a given center set, the "solution value"
 * reported throughout Section 7 (the objective of Section 1.1, read as the
 * largest distance from a point to its nearest center):
 * max over x of min over c of d(x, c).
 *   centers       [kc] int64 indices into the points, each in [0, n).
 *   radius        double out: the covering radius.
 *   argmax_point  int64 out (may be NULL): the farthest point, lowest index on
 *                 ties.
 * For float points with d <= 128 and kc * d >= 8192 (kc * d >= 1536 from
 * n = 262144 on) the n x kc block runs on the tensor cores (fp16 products with per-point bounds; every point that can
 * reach the maximum is recomputed in canonical FP32, then FP64), reading the
 * row-major points where they lie; the result is the same as the CUDA-core
 * path's (KC_RADIUS_TC selects either).  On the CUDA cores float points with
 * d <= 16 are read row-major too (no packed copy); host points are copied to
 * the device first on both row-major paths.
 * Errors: KC_ERR_ARG if kc < 1 or an index is out of range; others as above.
 */
kc_status kc_radius(const void *pts, int64_t n, int32_t d, const int64_t *centers, int32_t kc,
                    double *radius, int64_t *argmax_point, const kc_opts *opts);

/*
 * kc_mrg -- MRG, the two-round MapReduce Gonzalez of Algorithm 1 (Section
 * 3.1) with its 4-approximation (Lemma 2).  Round 1: the points are split into
 * m parts with contiguous index ranges; GON runs on every part (first center =
 * the part's lowest index) and returns up to k centers per part.  Round 2: the
 * union of those centers, in ascending index order, runs GON (first center =
 * its lowest index).  On one GPU the m "reducers" of round 1 run side by side
 * in one persistent launch, each part on a group of CTAs sized to its work.
 *   offsets  [m+1] int64 part boundaries (part i = [offsets[i], offsets[i+1]),
 *            offsets[0] = 0, offsets[m] = n, every part non-empty), host or
 *            device; NULL = balanced split offsets[i] = floor(i n / m), so no
 *            part exceeds ceil(n/m) points as Algorithm 1 asks.
 *   centers  [k] int64 out: round-2 selection (point indices, in order).
 *   k_out    int32 out: number of centers; radius: covering radius over all n.
 * Errors: KC_ERR_ARG for m outside [1, n] or bad offsets; others as kc_gonzalez.
 */
kc_status kc_mrg(const void *pts, int64_t n, int32_t d, int32_t k, int32_t m, const int64_t *offsets,
                 int64_t *centers, int32_t *k_out, double *radius, const kc_opts *opts);

/*
 * kc_mrg_rounds -- MRG with a machine capacity: Algorithm 1 with its while
 * loop (Section 3.2, Lemma 3).  Round 1 is kc_mrg's (GON on the m parts);
 * while the union S of the returned centers (in ascending index) holds more
 * than `capacity` points, S is split into ceil(|S| / capacity) contiguous
 * parts -- part i holds positions [floor(i |S| / m'), floor((i+1) |S| / m'))
 * of S -- each part runs GON from its lowest index, and S becomes the union
 * of their centers; finally GON on S from its lowest index.  Each round
 * beyond the second adds 2 to the approximation factor.  With
 * capacity >= m k this is kc_mrg.
 *   capacity  points one machine holds; must be >= 2k (else KC_ERR_ARG: the
 *             union could stop shrinking).
 *   rounds    int32 out, host memory, may be NULL: rounds run, the final
 *             GON included.
 * Other arguments and errors as kc_mrg.  With more than two rounds the call
 * reads |S| back after each round (a host loop) and does not take KC_ASYNC.
 * Rounds after the first sweep in FP32 whatever opts->sweep says (same
 * selections).
 */
kc_status kc_mrg_rounds(const void *pts, int64_t n, int32_t d, int32_t k, int32_t m, const int64_t *offsets,
                        int64_t capacity, int64_t *centers, int32_t *k_out, double *radius, int32_t *rounds,
                        const kc_opts *opts);

/*
 * kc_eim -- EIM: the sampling scheme of Ene, Im and Moseley as generalised in
 * Section 4 (EIM-MapReduce-Sample, Algorithm 2, with Select, Algorithm 3, and
 * the parameter phi), followed by GON on the returned sample (Section 4.2).
 *   S = {}, R = all points; log is the natural logarithm, n fixed.
 *   while |R| > (4/eps) k n^eps log n:
 *     every x in R joins S with probability min(1, 9 k n^eps log n / |R|) and
 *     H with probability min(1, 4 n^eps log n / |R|);
 *     v = the point at position p = min(|H|, max(1, ceil(phi log n))) of H
 *     sorted by distance to S (farthest first, lower index first on ties);
 *     every x in R with d(x, S) <= d(v, S) leaves R (equality removes, so R
 *     shrinks and sampled points always leave, Section 4.1); with H or S
 *     empty, only the new S members leave.
 *   C = S u R in ascending index order; GON(C, k) from C's lowest index.
 * Randomness: U(seed, it, x, stream) = splitmix64 output number
 * (it<<33 | x<<1 | stream) + 1 of the stream seeded opts->seed, top 53 bits
 * over 2^53; x joins S when U(.., 0) < pS and H when U(.., 1) < pH.
 * opts->phi (<= 0: 6, the paper's choice) and opts->seed are used.  Distances
 * are compared exactly as in kc_gonzalez (canonical FP32 or exact int32).
 * The call runs a host loop (one synchronisation per sampling round) and
 * does not take KC_ASYNC.  Errors: KC_ERR_ARG for eps outside (0, 1); others
 * as kc_gonzalez.
 */
kc_status kc_eim(const void *pts, int64_t n, int32_t d, int32_t k, double eps, int64_t *centers, int32_t *k_out,
                 double *radius, const kc_opts *opts);

/*
 * kc_gonzalez_batch -- GON on `count` independent instances in one
 * persistent launch (the simulated parallel machines of Section 7.1, one
 * instance per machine).  Instance i has points pts[i] (row-major n[i] x d[i],
 * host or device), selects up to k[i] centers from its point 0, and writes
 * centers[i][0 .. k_out[i]) (indices local to the instance) and radii[i].
 * n, d, k, pts and centers are host arrays of `count` entries; k_out and radii
 * are [count] arrays in host or device memory.
 * Launch shape: instances are ordered longest-first by modelled work
 * n k (d b + 8) bytes (b = 4 for FP32, 2 for the bf16 sweep).  An instance
 * whose work exceeds theta times the fair share of one resident CTA is solved
 * by a group of CTAs sized to its work (cooperative launch); the others go
 * through a queue, one CTA each, longest first.  theta is 1 by default; with
 * KC_AUTOTUNE in opts->flags the first call for a batch shape (count, dtype,
 * sweep and every (n, d, k)) solves the batch once per candidate theta
 * (plain queue, 4, 2, 1, 0.5), keeps the fastest for later calls in the
 * process, and returns the result of a final solve with it.  Every launch
 * shape selects the same centers.  KC_AUTOTUNE does not combine with
 * KC_ASYNC.  Errors: as kc_gonzalez, per instance; KC_ERR_ARG for the fp8
 * sweep (it needs per-instance column scales).
 */
kc_status kc_gonzalez_batch(int32_t count, const void *const *pts, const int64_t *n, const int32_t *d,
                            const int32_t *k, int64_t *const *centers, int32_t *k_out, double *radii,
                            const kc_opts *opts);

/*
 * Batch plans -- the batched form prepared once and replayed as a CUDA graph.
 * The paper has no counterpart (it simulates its parallel machines one after
 * another, Section 7.1); a plan is for callers that solve the same batch
 * shape repeatedly on changing point values, e.g. inside a serving loop.
 *
 * kc_batch_plan_create takes the arguments of kc_gonzalez_batch, all of them
 * device memory of the current device (KC_ERR_ARG otherwise), checks them,
 * picks the launch shape (KC_AUTOTUNE: builds and times a plan per candidate
 * theta: a warm-up replay, then the fastest of five, and keeps the fastest), allocates the plan's
 * own scratch (freed by kc_batch_plan_destroy), uploads the instance
 * descriptors and captures pack + GON + radius into a CUDA graph.  The
 * pointers are bound at creation: each run reads the current contents of
 * pts[i] and writes centers[i], k_out and radii.
 * kc_batch_plan_run enqueues one replay on `stream` (a cudaStream_t; the
 * plan's device must be current) and returns at once.  Runs of one plan
 * must not overlap (they share scratch): order them on one stream.
 * kc_batch_plan_wait waits for the last run and returns its device status
 * (KC_ERR_RANGE, KC_ERR_NONFINITE, KC_ERR_TIMEOUT as kc_gonzalez).
 * kc_batch_plan_info reports the chosen theta, the number of group-solved
 * instances, their CTAs, and the grid size.
 * kc_batch_plan_destroy waits for the last run and frees the plan (NULL is
 * accepted).
 */
typedef struct kc_batch_plan kc_batch_plan;
kc_status kc_batch_plan_create(int32_t count, const void *const *pts, const int64_t *n, const int32_t *d,
                               const int32_t *k, int64_t *const *centers, int32_t *k_out, double *radii,
                               const kc_opts *opts, kc_batch_plan **plan);
kc_status kc_batch_plan_run(kc_batch_plan *plan, void *stream);
kc_status kc_batch_plan_wait(kc_batch_plan *plan);
kc_status kc_batch_plan_info(const kc_batch_plan *plan, double *theta, int32_t *nheavy, int32_t *gheavy,
                             int32_t *grid);
kc_status kc_batch_plan_destroy(kc_batch_plan *plan);

/*
 * kc_gonzalez_noalloc -- the same Gonzalez selection as kc_gonzalez, for
 * callers that must not allocate device memory during a call.  The paper has
 * no counterpart; this is a deployment variant.  cudaMalloc/cudaFree can
 * synchronise the whole device (stalling latency-critical loops such as a
 * serving loop), and a process whose HBM is already held by another
 * allocator may not get a fresh allocation at all.  This entry point takes
 * all of its scratch from one static device array of KC_NOALLOC_MAX_BYTES
 * (64 MiB), which every GPU that loads the library keeps until the process
 * exits, and calls no allocating routine.
 *   Arguments and results are those of kc_gonzalez, except: every pointer
 *   must be device memory of the current device; opts->flags must be 0 (the
 *   call always waits and returns the final status); opts->sweep must be
 *   KC_SWEEP_F32 and opts->reserved 0 (else KC_ERR_ARG: the low-precision
 *   copies would not fit the array); inputs needing more
 *   than KC_NOALLOC_MAX_BYTES of scratch (about n * (4 d + 12) bytes for
 *   float points, n * (4 d + 4) for int32) are rejected with KC_ERR_ARG and
 *   a message naming the size, before any work is enqueued.
 *   The first call on a device looks up the array's address
 *   (cudaGetSymbolAddress, with that device current); make that first call
 *   before any stream capture.  All calls share the array and each clears
 *   what must start at zero; calls whose GPU work overlaps in time (other
 *   threads or streams) race on it and must be serialised by the caller.
 */
#define KC_NOALLOC_MAX_BYTES (64 * 1024 * 1024)
kc_status kc_gonzalez_noalloc(const void *pts, int64_t n, int32_t d, int32_t k, int64_t first,
                              int64_t *centers, int32_t *k_out, double *radius, const kc_opts *opts);

/*
 * kc_sync -- wait for all work enqueued on `stream` and return (and clear)
 * the device status word of that stream's scratch: KC_OK, or the first error
 * a kernel recorded since the last kc_sync / synchronous call.
 */
kc_status kc_sync(void *stream);

/*
 * kc_last_fp32_radius -- the error of a result against FP64, for the last
 * kc_gonzalez, kc_mrg, kc_eim or kc_radius call on `stream`: *radius32 is the
 * square root of the largest canonical FP32 squared distance from a point to
 * its nearest chosen center (the values every selection was decided on; exact
 * for int32 points), in double.  Beside the call's returned radius (the same
 * quantity in FP64) it gives the FP32 evaluation's error at that result.
 * Waits for the stream.  KC_ERR_ARG if no such call ran on the stream since
 * kc_release; the value is undefined if that call failed.
 */
kc_status kc_last_fp32_radius(void *stream, double *radius32);

/* kc_last_error -- text describing the last failure on this thread. */
const char *kc_last_error(void);

/* kc_release -- free all cached device scratch of every device and stream.
 * No call may be in flight. */
void kc_release(void);

/* kc_version -- library version string. */
const char *kc_version(void);

/*
 * Tracing (no counterpart in the paper; the paper reports wall-clock time per
 * simulated MapReduce round, Section 7.1).  While tracing is on, each launch
 * step of every call is bracketed by CUDA events recorded on the call's
 * stream.  kc_trace_read waits for the traced work, copies up to `cap`
 * records into `out` (oldest first), clears the list and returns the number
 * of records that were pending.  kc_launch_count returns how many CUDA
 * kernels the library has launched in this process.
 */
typedef struct {
    char name[24];      /* launch step, e.g. "pack", "gonzalez", "radius" */
    int32_t kernels;    /* kernels launched by this step */
    float ms;           /* elapsed device time between the events */
} kc_trace_rec;

void kc_trace_enable(int32_t on);
int32_t kc_trace_read(kc_trace_rec *out, int32_t cap);
int64_t kc_launch_count(void);

/*
 * kc_counters -- diagnostics of the mixed-precision sweep on the current
 * device since the last call (which it resets): out[0] = candidates
 * recomputed exactly in FP32, out[1] = candidate-buffer overflows (a warp
 * rescanned its running minima); and of EIM's tensor-core prune: out[2] =
 * (point, center) pairs left undecided by the bounds and recomputed exactly,
 * out[3] = points processed; and of every EIM prune (tensor cores or CUDA
 * cores, counted on the host for all devices): out[4] = the sum over prune
 * rounds of |R| x |S|, the point-center pairs the prune covers; out[5] =
 * sweep rechecks whose exact-minimum memo lagged more than 4 centers (done by
 * a whole warp); out[6..8] = clock cycles of the persistent GON kernels,
 * summed over CTAs, spent in the sweep, the exact rechecks and the group
 * exchange; out[9], out[10] = the largest per-CTA sweep total and sweep +
 * recheck total; out[11..14] = clock cycles of the tensor-core blocks' MMA-
 * issuing thread, summed over CTAs, spent waiting for a center tile, for a
 * free accumulator, for a point tile, and in all.  Synchronises the device.
 * Returns the number of values (15), or -1 on a CUDA error.
 */
int32_t kc_counters(int64_t *out, int32_t cap);

/*
 * kc_read_sweep -- measurement helper, no counterpart in the paper: enqueue
 * on `stream` one kernel that reads the device buffer `buf` (`bytes` long,
 * both multiples of 16 and 16-byte aligned) `reps` times with 16-byte loads
 * over the whole GPU and folds the words into *sink (device memory).  Timed
 * with events around it, bytes * reps / time is the read bandwidth of the
 * level that holds the buffer: L2 for a buffer well under the L2 size, HBM
 * for one well over it.  This is the roofline denominator of a Gonzalez
 * sweep whose points stay in L2 between its k passes (Section 5.1).
 * Errors: KC_ERR_ARG for bad sizes or alignment, KC_ERR_CUDA on a launch
 * failure.
 */
kc_status kc_read_sweep(const void *buf, size_t bytes, int32_t reps, unsigned long long *sink, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* KCENTER_H */
