/*
 * kc_oracle.c -- plain CPU oracle for k-center (McClintock & Wirth,
 * "Efficient Parallel Algorithms for k-Center Clustering", arXiv 1604.03228).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed
 * CPU baseline of the benchmark may load this file's library.  It shares no
 * code with the CUDA path and reads nothing from it.
 *
 * Everything here is written for a reader to check against the paper by eye:
 * one loop per definition, no blocking, no fusion, no reordering.  Distances
 * are evaluated in one of three metric modes:
 *
 *   ORC_F64  FP32 coordinates widened to double; squared distance summed in
 *            coordinate order with separate multiply and add (the library is
 *            compiled with -ffp-contract=off so no fused multiply-add sneaks in).
 *   ORC_F32  the "canonical FP32" squared distance: for j = 0..d-1,
 *            t = x_j - c_j (float), acc = fmaf(t, t, acc) starting from 0.
 *            The paper does not fix a precision; this mode lets the oracle
 *            take argmax decisions in the same precision as a float kernel.
 *   ORC_I64  int32 coordinates, exact int64 sum of squared differences.
 *
 * Values are carried as double.  For ORC_F32 a float converts exactly; for
 * ORC_I64 the caller guarantees every squared distance is below 2^53 (the
 * Python wrapper checks d * range^2 < 2^53), so comparisons in double are
 * exactly the comparisons in the native type.
 *
 * Squared distances are compared; a radius is the square root of the largest
 * squared distance (sqrt is monotone, so the argmax is unchanged).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_F64 = 0, ORC_F32 = 1, ORC_I64 = 2 };

typedef struct {
    const void *pts; /* row-major n x d, float (F64/F32 modes) or int32 (I64) */
    int64_t n;
    int32_t d;
    int32_t mode;
} orc_metric;

/* Squared distance between global points a and b (the metric of Section 1.1,
 * Euclidean, computed on demand from coordinates as in Section 7.2). */
static double orc_d2(const orc_metric *M, int64_t a, int64_t b)
{
    const int32_t d = M->d;
    if (M->mode == ORC_F64) {
        const float *x = (const float *)M->pts + a * d;
        const float *y = (const float *)M->pts + b * d;
        double s = 0.0;
        for (int32_t j = 0; j < d; ++j) {
            double t = (double)x[j] - (double)y[j];
            double sq = t * t;
            s = s + sq;
        }
        return s;
    } else if (M->mode == ORC_F32) {
        const float *x = (const float *)M->pts + a * d;
        const float *y = (const float *)M->pts + b * d;
        float acc = 0.0f;
        for (int32_t j = 0; j < d; ++j) {
            float t = x[j] - y[j];
            acc = fmaf(t, t, acc);
        }
        return (double)acc;
    } else {
        const int32_t *x = (const int32_t *)M->pts + a * d;
        const int32_t *y = (const int32_t *)M->pts + b * d;
        int64_t s = 0;
        for (int32_t j = 0; j < d; ++j) {
            int64_t t = (int64_t)x[j] - (int64_t)y[j];
            s += t * t;
        }
        return (double)s;
    }
}

static inline int64_t orc_global(const int64_t *subset, int64_t pos)
{
    return subset ? subset[pos] : pos;
}

/*
 * GON, Section 3.1: start from an arbitrary point (here the one at position
 * `first_pos`), then repeatedly mark as a new center the point farthest from
 * the centers chosen so far, until k centers exist.
 *
 * Readings of points the paper leaves open:
 *  - ties among equally far points go to the lowest position (positions are
 *    in ascending global index order, so this is the lowest global index);
 *  - if every point is already at distance 0 from the centers, stop early
 *    (the definition in Section 1.1 asks for "at most k" centers).
 *
 * subset: NULL for all n points, else n ascending global indices.
 * Outputs: centers[k] (global indices, selection order), sel2[k] (squared
 * distance of each center to the earlier centers when it was chosen; 0 for
 * the first), *radius2 = max over the subset of the squared distance to the
 * nearest center.  Returns the number of centers chosen.
 */
int64_t orc_gon(const orc_metric *M, const int64_t *subset, int64_t n, int64_t k,
                int64_t first_pos, int64_t *centers, double *sel2, double *radius2)
{
    if (n <= 0 || k <= 0) { *radius2 = 0.0; return 0; }
    double *mind = (double *)malloc((size_t)n * sizeof(double));
    int64_t c = orc_global(subset, first_pos);
    int64_t kout = 0;
    centers[kout] = c;
    if (sel2) sel2[kout] = 0.0;
    kout++;
    for (int64_t p = 0; p < n; ++p) mind[p] = orc_d2(M, orc_global(subset, p), c);
    while (kout < k) {
        int64_t best = 0;
        double bestv = mind[0];
        for (int64_t p = 1; p < n; ++p)
            if (mind[p] > bestv) { bestv = mind[p]; best = p; }
        if (bestv == 0.0) break;
        c = orc_global(subset, best);
        centers[kout] = c;
        if (sel2) sel2[kout] = bestv;
        kout++;
        for (int64_t p = 0; p < n; ++p) {
            double t = orc_d2(M, orc_global(subset, p), c);
            if (t < mind[p]) mind[p] = t;
        }
    }
    double r = 0.0;
    for (int64_t p = 0; p < n; ++p) if (mind[p] > r) r = mind[p];
    *radius2 = r;
    free(mind);
    return kout;
}

/*
 * Covering radius (the "solution value" of Section 7, and the objective of
 * Section 1.1 read as max over points of the distance to the nearest
 * center): max_x min_{c in C} d(x, c) over points x of the subset.  The
 * argmax goes to the lowest index among equal maxima.  Returns the squared
 * radius; *argmax gets the global index of the farthest point.
 */
double orc_radius(const orc_metric *M, const int64_t *subset, int64_t n,
                  const int64_t *C, int64_t kc, int64_t *argmax)
{
    double best = -1.0;
    int64_t besti = -1;
    for (int64_t p = 0; p < n; ++p) {
        int64_t x = orc_global(subset, p);
        double m = INFINITY;
        for (int64_t i = 0; i < kc; ++i) {
            double t = orc_d2(M, x, C[i]);
            if (t < m) m = t;
        }
        if (m > best) { best = m; besti = x; }
    }
    if (argmax) *argmax = besti;
    return best < 0.0 ? 0.0 : best;
}

/*
 * For a given center sequence C[0..kc-1] over all n points: max2[j] is the
 * largest squared distance from any point to {C[0..j-1]} (so max2[j] is the
 * value GON's j-th selection should attain) and sel2[j] is the squared
 * distance of C[j] to {C[0..j-1]}; max2[0] = sel2[0] = 0; max2[kc] is the
 * squared covering radius of the whole sequence.  Used to check a float
 * selection step by step against the exact step maximum.
 */
void orc_eval_sequence(const orc_metric *M, const int64_t *C, int64_t kc,
                       double *sel2, double *max2)
{
    const int64_t n = M->n;
    double *mind = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t p = 0; p < n; ++p) mind[p] = INFINITY;
    sel2[0] = 0.0;
    max2[0] = 0.0;
    for (int64_t j = 0; j < kc; ++j) {
        if (j > 0) {
            double mx = 0.0;
            for (int64_t p = 0; p < n; ++p) if (mind[p] > mx) mx = mind[p];
            max2[j] = mx;
            sel2[j] = mind[C[j]];
        }
        for (int64_t p = 0; p < n; ++p) {
            double t = orc_d2(M, p, C[j]);
            if (t < mind[p]) mind[p] = t;
        }
    }
    double mx = 0.0;
    for (int64_t p = 0; p < n; ++p) if (mind[p] > mx) mx = mind[p];
    max2[kc] = mx;
    free(mind);
}

/*
 * MRG with two rounds, Algorithm 1 when the point set fits the capacity
 * (Lemma 2):
 *   round 1: part i = global indices [off[i], off[i+1]) runs GON with its
 *            lowest index as the first center and returns up to k centers C_i;
 *   round 2: S = union of the C_i, taken in ascending global index order,
 *            runs GON with its lowest index as the first center.
 * Outputs: round1[m*k] (part i's centers at round1[i*k ..], padded with -1),
 * round1_k[m], centers[k] (round-2 selection), returns the number chosen;
 * *radius2 is the squared covering radius of the final centers over all n.
 */
static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

int64_t orc_mrg(const orc_metric *M, int64_t k, int64_t m, const int64_t *off,
                int64_t *round1, int64_t *round1_k, int64_t *centers, double *radius2)
{
    int64_t *subset = (int64_t *)malloc((size_t)M->n * sizeof(int64_t));
    int64_t *S = (int64_t *)malloc((size_t)(m * k) * sizeof(int64_t));
    int64_t sn = 0;
    double r2;
    for (int64_t i = 0; i < m; ++i) {
        int64_t lo = off[i], hi = off[i + 1];
        for (int64_t p = lo; p < hi; ++p) subset[p - lo] = p;
        int64_t *Ci = round1 + i * k;
        for (int64_t j = 0; j < k; ++j) Ci[j] = -1;
        int64_t ki = orc_gon(M, subset, hi - lo, k, 0, Ci, NULL, &r2);
        round1_k[i] = ki;
        for (int64_t j = 0; j < ki; ++j) S[sn++] = Ci[j];
    }
    qsort(S, (size_t)sn, sizeof(int64_t), cmp_i64);
    int64_t kout = orc_gon(M, S, sn, k, 0, centers, NULL, &r2);
    *radius2 = orc_radius(M, NULL, M->n, centers, kout, NULL);
    free(subset);
    free(S);
    return kout;
}

/*
 * MRG with a machine capacity c (Algorithm 1 with its while loop).  The first
 * round runs GON on the m given parts (as orc_mrg).  While the union S of the
 * returned centers, in ascending index, holds more than c points, S is split
 * into m' = ceil(|S| / c) contiguous parts -- part i holds positions
 * [floor(i |S| / m'), floor((i + 1) |S| / m')) of S, at most c points -- each
 * part runs GON from its lowest index, and S becomes the union of their
 * centers.  Finally GON on S from its lowest index.  Each extra round adds 2
 * to the approximation factor (Lemma 3).  Needs c >= 2k, so that S shrinks
 * (the machine count of inequality (1) falls below 2 only when 2k < c).
 * sizes[r] (at most max_rounds entries) gets |S| after round r + 1;
 * *rounds the number of rounds including the final one.  Returns k_out, or
 * -1 when c < 2k or the rounds exceed max_rounds.
 */
int64_t orc_mrg_rounds(const orc_metric *M, int64_t k, int64_t m, const int64_t *off, int64_t c,
                       int64_t max_rounds, int64_t *sizes, int64_t *rounds, int64_t *centers, double *radius2)
{
    if (c < 2 * k) return -1;
    int64_t cap = m * k > 1 ? m * k : 1;
    int64_t *subset = (int64_t *)malloc((size_t)M->n * sizeof(int64_t));
    int64_t *S = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    int64_t *T = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    int64_t *Ci = (int64_t *)malloc((size_t)k * sizeof(int64_t));
    int64_t sn = 0, r = 0, kout = -1;
    double r2;
    for (int64_t i = 0; i < m; ++i) {
        int64_t lo = off[i], hi = off[i + 1];
        for (int64_t p = lo; p < hi; ++p) subset[p - lo] = p;
        int64_t ki = orc_gon(M, subset, hi - lo, k, 0, Ci, NULL, &r2);
        for (int64_t j = 0; j < ki; ++j) S[sn++] = Ci[j];
    }
    qsort(S, (size_t)sn, sizeof(int64_t), cmp_i64);
    if (r < max_rounds) sizes[r] = sn;
    ++r;
    while (sn > c) {
        if (r >= max_rounds) goto done;
        int64_t mp = (sn + c - 1) / c, tn = 0;
        for (int64_t i = 0; i < mp; ++i) {
            int64_t lo = (int64_t)((__int128)i * sn / mp), hi = (int64_t)((__int128)(i + 1) * sn / mp);
            int64_t ki = orc_gon(M, S + lo, hi - lo, k, 0, Ci, NULL, &r2);
            for (int64_t j = 0; j < ki; ++j) T[tn++] = Ci[j];
        }
        qsort(T, (size_t)tn, sizeof(int64_t), cmp_i64);
        int64_t *tmp = S;
        S = T;
        T = tmp;
        sn = tn;
        sizes[r] = sn;
        ++r;
    }
    kout = orc_gon(M, S, sn, k, 0, centers, NULL, &r2);
    *radius2 = orc_radius(M, NULL, M->n, centers, kout, NULL);
    ++r;
done:
    *rounds = r;
    free(subset);
    free(S);
    free(T);
    free(Ci);
    return kout;
}

/*
 * Uniform draw U(seed, it, x, stream) in [0, 1) for EIM's Bernoulli samples.
 * The paper leaves the random source open; this is a counter-based
 * splitmix64 (Steele, Lea, Flood 2014): counter = it<<33 | x<<1 | stream,
 * h = mix64(seed + (counter + 1) * 0x9E3779B97F4A7C15), u = (h >> 11) / 2^53.
 */
static uint64_t orc_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double orc_uniform(uint64_t seed, uint64_t it, uint64_t x, uint64_t stream)
{
    uint64_t ctr = (it << 33) | (x << 1) | stream;
    uint64_t h = orc_mix64(seed + (ctr + 1ULL) * 0x9E3779B97F4A7C15ULL);
    return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

/* d(x, S) = min over s in S of the (squared) distance; +inf for empty S. */
static double orc_dist_to_set(const orc_metric *M, int64_t x, const int64_t *S, int64_t sn)
{
    double m = INFINITY;
    for (int64_t i = 0; i < sn; ++i) {
        double t = orc_d2(M, x, S[i]);
        if (t < m) m = t;
    }
    return m;
}

typedef struct { double dist; int64_t idx; } orc_hkey;

/* Order for Select (Algorithm 3): farthest first, lower index first on ties. */
static int cmp_hkey(const void *a, const void *b)
{
    const orc_hkey *x = (const orc_hkey *)a, *y = (const orc_hkey *)b;
    if (x->dist > y->dist) return -1;
    if (x->dist < y->dist) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/*
 * EIM: EIM-MapReduce-Sample (Algorithm 2) with Select (Algorithm 3) and the
 * paper's parameter phi, then GON on the returned sample (Section 4.2).
 *
 *   S = {}, R = V;  n = |V| throughout;  log is the natural logarithm.
 *   while |R| > (4/eps) k n^eps log n:
 *       each x in R joins S with probability min(1, 9 k n^eps log n / |R|)
 *       and joins H with probability min(1, 4 n^eps log n / |R|);
 *       v = Select(H, S): sort H by d(., S) farthest first (lower index first
 *           on ties) and take position p = min(|H|, max(1, ceil(phi log n)))
 *           (1-based);
 *       remove from R every x with d(x, S) <= d(v, S)   (Section 4.1: "equal"
 *           is removed too, so R shrinks and sampled points always leave R);
 *       if H or S is empty there is no pivot: only the new S members leave R.
 *   C = S u R in ascending index order; GON(C, k) from the lowest index.
 *
 * Outputs: centers[k], returns the number chosen; *radius2 over all points;
 * stats[0] = loop iterations, stats[1] = |S|, stats[2] = |R| at exit,
 * stats[3] = |C|.  If sample_out is non-NULL it receives C (size n).
 * If trace is non-NULL, iteration it < trace_cap writes 8 doubles at
 * trace[8*it]: pS, pH, |S| after sampling, |H|, pivot v (-1 if none),
 * d(v,S)^2 (-1 if none), |R| after pruning, and the 1-based position p used.
 */
int64_t orc_eim(const orc_metric *M, int64_t k, double eps, double phi, uint64_t seed,
                int64_t *centers, double *radius2, int64_t *stats, int64_t *sample_out,
                double *trace, int64_t trace_cap)
{
    const int64_t n = M->n;
    const double ne = pow((double)n, eps);
    const double ln = log((double)n);
    const double base = ne * ln;
    const double limit = (4.0 / eps) * (double)k * base;
    const int64_t pos = (int64_t)ceil(phi * ln);

    int64_t *R = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *Rn = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *S = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *H = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    unsigned char *inS = (unsigned char *)calloc((size_t)n, 1);
    int64_t rn = n, sn = 0, it = 0;
    for (int64_t x = 0; x < n; ++x) R[x] = x;

    while ((double)rn > limit) {
        const double pS = fmin(1.0, 9.0 * (double)k * base / (double)rn);
        const double pH = fmin(1.0, 4.0 * base / (double)rn);
        int64_t hn = 0;
        for (int64_t i = 0; i < rn; ++i) {
            int64_t x = R[i];
            if (orc_uniform(seed, (uint64_t)it, (uint64_t)x, 0) < pS) inS[x] = 1;
            if (orc_uniform(seed, (uint64_t)it, (uint64_t)x, 1) < pH) H[hn++] = x;
        }
        sn = 0;
        for (int64_t x = 0; x < n; ++x) if (inS[x]) S[sn++] = x;

        int64_t rnn = 0;
        if (hn > 0 && sn > 0) {
            orc_hkey *hk = (orc_hkey *)malloc((size_t)hn * sizeof(orc_hkey));
            for (int64_t i = 0; i < hn; ++i) {
                hk[i].dist = orc_dist_to_set(M, H[i], S, sn);
                hk[i].idx = H[i];
            }
            qsort(hk, (size_t)hn, sizeof(orc_hkey), cmp_hkey);
            int64_t p = pos < 1 ? 1 : pos;
            if (p > hn) p = hn;
            const double thr = hk[p - 1].dist;
            if (trace && it < trace_cap) {
                trace[8 * it + 4] = (double)hk[p - 1].idx;
                trace[8 * it + 5] = thr;
                trace[8 * it + 7] = (double)p;
            }
            free(hk);
            for (int64_t i = 0; i < rn; ++i) {
                int64_t x = R[i];
                if (orc_dist_to_set(M, x, S, sn) > thr) Rn[rnn++] = x;
            }
        } else {
            for (int64_t i = 0; i < rn; ++i) if (!inS[R[i]]) Rn[rnn++] = R[i];
        }
        if (trace && it < trace_cap) {
            trace[8 * it + 0] = pS;
            trace[8 * it + 1] = pH;
            trace[8 * it + 2] = (double)sn;
            trace[8 * it + 3] = (double)hn;
            trace[8 * it + 6] = (double)rnn;
            if (!(hn > 0 && sn > 0)) {
                trace[8 * it + 4] = -1.0;
                trace[8 * it + 5] = -1.0;
                trace[8 * it + 7] = 0.0;
            }
        }
        int64_t *tmp = R; R = Rn; Rn = tmp;
        rn = rnn;
        it++;
    }

    /* C = S u R, ascending (R and S are disjoint once pruned; mark both). */
    int64_t cn = 0;
    for (int64_t i = 0; i < rn; ++i) inS[R[i]] = 1;
    for (int64_t x = 0; x < n; ++x) if (inS[x]) H[cn++] = x;
    double r2;
    int64_t kout = orc_gon(M, H, cn, k, 0, centers, NULL, &r2);
    *radius2 = orc_radius(M, NULL, n, centers, kout, NULL);
    if (stats) { stats[0] = it; stats[1] = sn; stats[2] = rn; stats[3] = cn; }
    if (sample_out) memcpy(sample_out, H, (size_t)cn * sizeof(int64_t));
    free(R); free(Rn); free(S); free(H); free(inS);
    return kout;
}

/* Squared distance of every point to its nearest center (assignment values). */
void orc_mind(const orc_metric *M, const int64_t *C, int64_t kc, double *out)
{
    for (int64_t x = 0; x < M->n; ++x) {
        double m = INFINITY;
        for (int64_t i = 0; i < kc; ++i) {
            double t = orc_d2(M, x, C[i]);
            if (t < m) m = t;
        }
        out[x] = m;
    }
}
