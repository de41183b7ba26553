/*
 * zsort_oracle.c -- plain, slow, sequential CPU restatement of zSort
 * (Jain, Sabale, Shastri, Thakkar, Londhe: "zSort: Stable Distribution Sort
 * using Z-Score Partitioning", arXiv 2605.14419).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the package's smoke() check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header or constant
 * with the CUDA library: every step below is written from the paper's text.
 *
 * Contents
 *   oracle_stats             Alg. 1, statistics loops (min, mean, population sd)
 *   oracle_zsort_pairs       Alg. 1 + zsortRec (section "Proposed Work"), on
 *                            (uint64 key, uint32 payload) pairs, stable
 *   oracle_zsort_pairs_rec   the same, also recording every zsortRec
 *                            sub-problem's meanEst, mean, sd and Zmin (R9)
 *   oracle_zsort_segmented   the same, applied to each segment of a batch
 *   oracle_key_from_i64/f64  order-preserving key encodings (not in the paper;
 *                            definitions of two's-complement order and of the
 *                            IEEE-754 totalOrder predicate)
 *   oracle_splitmix64, oracle_sample_positions, oracle_pwl_train,
 *   oracle_pwl_bucket        the learned monotone piecewise-linear bucket map
 *                            that replaces the z-score map (not in the paper;
 *                            restated from its written definition)
 *   oracle_split_train, oracle_split_bucket
 *                            the learned map with exact-key breakpoints, the
 *                            second choice when the FP32 normalisation of the
 *                            first collapses the keys (not in the paper;
 *                            reading R12)
 *   oracle_mlp_train, oracle_mlp_bucket
 *                            the alternative learned map: a 2-layer MLP with
 *                            positive weights fitted to the same quantile
 *                            knots (not in the paper; restated from its
 *                            written definition below)
 *
 * Readings of the paper where it is silent or garbled (each repeated where
 * it is used):
 *   R1  Statistics are taken on d = key - min (exact unsigned subtraction,
 *       then conversion to double).  The z-score is shift invariant, so the
 *       map is unchanged; the paper's raw sum of 64-bit keys would overflow.
 *   R2  The early exit "min == mean" is restated as "min == max".
 *   R3  Eq. 1 adds z_min, "the minimum z-score", which is negative; Alg. 1
 *       uses Zmin = |(min - mean)/std|.  The absolute value is taken.
 *   R4  Buckets are floor(h) clipped to [0, k-1]; the paper clips only the
 *       top, the bottom clip only guards rounding.
 *   R5  k = max(2, floor(alpha * sqrt(n))) with alpha = 0.6 (the tuned value
 *       of the alpha sensitivity study, Table 2); scale = k/4; both fixed
 *       for every recursion level.
 *   R6  A cluster with more than `leaf` (96) elements recurses, otherwise it
 *       is insertion sorted.
 *   R7  The counting-sort switch (range < 65000) is checked on entry to
 *       every (sub)problem, after the early exit.
 *   R8  The scatter statement of Alg. 1 is missing its right-hand side; it
 *       is read as a stable scatter of the (key, payload) pair.
 *   R9  zsortRec takes mean = meanEst and recomputes min, max, the standard
 *       deviation about meanEst and Zmin over its own sub-array.
 *   R10 Progress guard (the paper's depth argument assumes every level
 *       shrinks the largest part): if a level puts every element of a
 *       sub-problem with min < max into one cluster, or the depth reaches
 *       `guard_depth`, that level uses the range map
 *       b = floor(d * k / (range + 1)) in exact 128-bit integer arithmetic.
 *   R11 The learned map is not in the paper; it is a fitted model whose
 *       parameters are the breakpoints q[0..P] and one slope per piece,
 *       r[s] = fl32(1 / (q[s+1] - q[s])), fixed when the model is trained.
 *       Inference multiplies by the stored slope, frac = fl32(fl32(u - q[s])
 *       * r[s]), instead of dividing by the width for every key.  Both forms
 *       are monotone in u inside a piece (a rounded product or quotient by a
 *       fixed positive number), so either sorts exactly; they can differ in
 *       the last bit of frac and so in the bucket of a key that sits on a
 *       sub-bucket edge.  The stored-slope form is the definition here.
 *   R12 The learned map's second form, for keys that binary32 normalisation
 *       collapses, keeps R11's model (the same 256 quantiles of the same
 *       sample) but holds its breakpoints as keys: b[0] = min, b[P] = max,
 *       b[j] = the sample key of rank j m / P, and r[s] = fl32(1 /
 *       fl32(b[s+1] - b[s])) (0 for an empty piece).  A key's piece is the
 *       last b[j] <= key among j = 1..P-1, and it is interpolated from its
 *       piece's own lower key, frac = fl32(fl32(key - b[s]) * r[s]), clipped
 *       to [0, 1 - 2^-24]; bucket = s * (k/P) + min(k/P - 1, floor(frac *
 *       k/P)).  Monotone in the key inside a piece for the same reason as
 *       R11, and across pieces because the pieces' buckets are ordered.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* Counters describing one oracle run (returned to the caller). */
typedef struct {
    uint64_t partitions;      /* partition passes executed (all levels)      */
    uint64_t max_depth;       /* deepest recursion level reached (top = 0)   */
    uint64_t guard_levels;    /* levels that used the range map (R10)        */
    uint64_t counting_sorts;  /* sub-problems finished by counting sort (R7) */
    uint64_t insertion_sorts; /* clusters finished by insertion sort (R6)    */
    uint64_t equal_exits;     /* sub-problems finished by min == max (R2)    */
    uint64_t k;               /* number of clusters (R5)                     */
    double scale;             /* Eq. 1 scale (R5)                            */
} oracle_trace;

/* One zsortRec sub-problem as it was partitioned (R9): the cluster j of the
 * parent it came from, its size and minimum, meanEst in the parent's frame
 * (d-units above the parent's minimum), and the mean (meanEst moved into
 * its own frame), standard deviation about that mean and Zmin it used. */
typedef struct {
    uint64_t depth, parent_bucket, size, min, parent_min;
    double est_parent_d, mean, sd, zmin;
} oracle_sub_rec;

typedef struct {
    uint64_t k;
    double scale;
    uint64_t leaf;        /* insertion-sort cutoff, 96 in the paper        */
    uint64_t count_range; /* counting-sort switch, 65000 in the paper      */
    uint64_t guard_depth; /* depth from which R10 always applies           */
    uint64_t *count;      /* counting-sort histogram, count_range entries  */
    oracle_trace *tr;
    oracle_sub_rec *rec;  /* optional record of the sub-problems (R9)      */
    uint64_t rec_cap, rec_n;
} zs_ctx;

/* ------------------------------------------------------------------------ */
/* Alg. 1, statistics: one pass for the sum and the minimum, one pass for the
 * sum of squared deviations; std = sqrt(var / size) (population).  Computed
 * on d = key - min (R1).  Also returns the maximum (needed by R2, R7). */
void oracle_stats(const uint64_t *keys, uint64_t n, uint64_t *min_out,
                  uint64_t *max_out, double *mean_d_out, double *sd_out)
{
    uint64_t mn = keys[0], mx = keys[0];
    for (uint64_t i = 1; i < n; i++) {
        if (keys[i] < mn) mn = keys[i];
        if (keys[i] > mx) mx = keys[i];
    }
    double sum = 0.0;
    for (uint64_t i = 0; i < n; i++) sum += (double)(keys[i] - mn);
    double mean = sum / (double)n;
    double var = 0.0;
    for (uint64_t i = 0; i < n; i++) {
        double res = (double)(keys[i] - mn) - mean;
        var += res * res;
    }
    *min_out = mn;
    *max_out = mx;
    *mean_d_out = mean;
    *sd_out = sqrt(var / (double)n);
}

/* Stable insertion sort of n pairs in place (Alg. 1, small clusters). */
static void insertion_sort(uint64_t *k, uint32_t *v, uint64_t n)
{
    for (uint64_t i = 1; i < n; i++) {
        uint64_t ck = k[i];
        uint32_t cv = v[i];
        uint64_t j = i;
        while (j > 0 && k[j - 1] > ck) { /* strict: equal keys keep order */
            k[j] = k[j - 1];
            v[j] = v[j - 1];
            j--;
        }
        k[j] = ck;
        v[j] = cv;
    }
}

/* Stable counting sort by d = key - mn over [0, range] (R7). */
static void counting_sort(zs_ctx *c, const uint64_t *sk, const uint32_t *sv,
                          uint64_t *dk, uint32_t *dv, uint64_t n, uint64_t mn,
                          uint64_t range)
{
    uint64_t *cnt = c->count;
    memset(cnt, 0, (size_t)(range + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < n; i++) cnt[sk[i] - mn]++;
    uint64_t run = 0;
    for (uint64_t r = 0; r <= range; r++) {
        uint64_t t = cnt[r];
        cnt[r] = run;
        run += t;
    }
    for (uint64_t i = 0; i < n; i++) {
        uint64_t p = cnt[sk[i] - mn]++;
        dk[p] = sk[i];
        dv[p] = sv[i];
    }
}

/* Eq. 1 with R3, R4: h = ((d - mean)/std + Zmin) * scale, b = clip(floor h). */
static uint64_t zmap(double d, double mean, double sd, double zmin,
                     double scale, uint64_t k)
{
    double h = ((d - mean) / sd + zmin) * scale;
    if (!(h >= 0.0)) return 0;
    if (h >= (double)(k - 1)) return k - 1;
    return (uint64_t)h; /* floor for h >= 0 */
}

/* R10: range map, exact: floor(d * k / (range + 1)). */
static uint64_t rmap(uint64_t d, uint64_t range, uint64_t k)
{
    return (uint64_t)(((u128)d * (u128)k) / ((u128)range + 1));
}

/*
 * One zSort (sub)problem: sorts src[0..size) stably into dst[0..size).
 * src is consumed; tmp is the single auxiliary "clustersArr" of Alg. 1.
 * have_est == 0: top level, mean computed (Alg. 1).
 * have_est != 0: zsortRec, mean = meanEst, given in the parent's d-frame
 *                (relative to parent_min) (R9).
 */
static void zs_rec(zs_ctx *c, uint64_t *sk, uint32_t *sv, uint64_t *dk,
                   uint32_t *dv, uint64_t *tk, uint32_t *tv, uint64_t size,
                   int have_est, double est_parent_d, uint64_t parent_min,
                   uint64_t parent_bucket, uint64_t depth)
{
    oracle_trace *tr = c->tr;
    if (depth > tr->max_depth) tr->max_depth = depth;
    if (size == 0) return;
    if (size == 1) {
        dk[0] = sk[0];
        dv[0] = sv[0];
        return;
    }

    /* Alg. 1 first loop: sum and min (here also max, R2/R7). */
    uint64_t mn = sk[0], mx = sk[0];
    for (uint64_t i = 1; i < size; i++) {
        if (sk[i] < mn) mn = sk[i];
        if (sk[i] > mx) mx = sk[i];
    }
    /* R2: a set of identical keys is already sorted. */
    if (mn == mx) {
        memcpy(dk, sk, (size_t)size * sizeof(uint64_t));
        memcpy(dv, sv, (size_t)size * sizeof(uint32_t));
        tr->equal_exits++;
        return;
    }
    uint64_t range = mx - mn;
    /* R7: counting sort for small key ranges. */
    if (range < c->count_range) {
        counting_sort(c, sk, sv, dk, dv, size, mn, range);
        tr->counting_sorts++;
        return;
    }

    double mean;
    if (!have_est) {
        double sum = 0.0;
        for (uint64_t i = 0; i < size; i++) sum += (double)(sk[i] - mn);
        mean = sum / (double)size;
    } else {
        /* R9: meanEst moved from the parent's frame into this one. */
        mean = est_parent_d - (double)(mn - parent_min);
    }
    /* Alg. 1 second loop: var = sum (x - mean)^2, std = sqrt(var/size). */
    double var = 0.0;
    for (uint64_t i = 0; i < size; i++) {
        double res = (double)(sk[i] - mn) - mean;
        var += res * res;
    }
    double sd = sqrt(var / (double)size);
    double zmin = fabs((0.0 - mean) / sd); /* R3: Zmin = |(min - mean)/std| */
    if (have_est && c->rec) {
        if (c->rec_n < c->rec_cap) {
            oracle_sub_rec *r = &c->rec[c->rec_n];
            r->depth = depth;
            r->parent_bucket = parent_bucket;
            r->size = size;
            r->min = mn;
            r->parent_min = parent_min;
            r->est_parent_d = est_parent_d;
            r->mean = mean;
            r->sd = sd;
            r->zmin = zmin;
        }
        c->rec_n++;
    }
    uint64_t k = c->k;
    double scale = c->scale;

    uint64_t *counts = (uint64_t *)calloc((size_t)k, sizeof(uint64_t));
    uint64_t *offs = (uint64_t *)malloc((size_t)k * sizeof(uint64_t));
    int guard = depth >= c->guard_depth;
    for (int attempt = 0; attempt < 2; attempt++) {
        memset(counts, 0, (size_t)k * sizeof(uint64_t));
        /* Histogram of clusters (Alg. 1). */
        for (uint64_t i = 0; i < size; i++) {
            uint64_t d = sk[i] - mn;
            uint64_t b = guard ? rmap(d, range, k)
                               : zmap((double)d, mean, sd, zmin, scale, k);
            counts[b]++;
        }
        if (guard) break;
        /* R10: a level that made no progress is redone with the range map. */
        int stuck = 0;
        for (uint64_t b = 0; b < k; b++)
            if (counts[b] == size) stuck = 1;
        if (!stuck) break;
        guard = 1;
    }
    if (guard) tr->guard_levels++;
    tr->partitions++;

    /* Exclusive scan of counts into offsets (Alg. 1). */
    uint64_t run = 0;
    for (uint64_t b = 0; b < k; b++) {
        offs[b] = run;
        run += counts[b];
    }
    /* Stable scatter in input order into the single auxiliary array (R8). */
    for (uint64_t i = 0; i < size; i++) {
        uint64_t d = sk[i] - mn;
        uint64_t b = guard ? rmap(d, range, k)
                           : zmap((double)d, mean, sd, zmin, scale, k);
        uint64_t p = offs[b]++;
        tk[p] = sk[i];
        tv[p] = sv[i];
    }

    /* Per-cluster dispatch with running offset lbSum (Alg. 1). */
    uint64_t lb = 0;
    for (uint64_t b = 0; b < k; b++) {
        uint64_t cnt = counts[b];
        if (cnt == 0) continue;
        if (cnt > c->leaf) {
            /* meanEst = ((j + 0.5)/scale - Zmin) * std + mean (zsortRec). */
            double est = (((double)b + 0.5) / scale - zmin) * sd + mean;
            if (guard) {
                /* The range map has no z-space; use the cluster midpoint. */
                est = ((double)b + 0.5) * ((double)range + 1.0) / (double)k;
            }
            /* The cluster in tmp is the child's source; src is free now and
             * serves as the child's auxiliary array. */
            zs_rec(c, tk + lb, tv + lb, dk + lb, dv + lb, sk + lb, sv + lb, cnt,
                   1, est, mn, b, depth + 1);
        } else {
            memcpy(dk + lb, tk + lb, (size_t)cnt * sizeof(uint64_t));
            memcpy(dv + lb, tv + lb, (size_t)cnt * sizeof(uint32_t));
            insertion_sort(dk + lb, dv + lb, cnt);
            tr->insertion_sorts++;
        }
        lb += cnt;
    }
    free(counts);
    free(offs);
}

/*
 * Sorts n (key, payload) pairs in place, ascending by key, stably.
 * alpha: cluster-count factor (k = max(2, floor(alpha*sqrt(n)))), 0.6 in the
 * paper; leaf: insertion-sort cutoff (96); count_range: counting-sort switch
 * (65000); guard_depth: depth from which the range map is always used.
 * Returns 0, or -1 on allocation failure.
 */
int oracle_zsort_pairs_rec(uint64_t *keys, uint32_t *vals, uint64_t n,
                           double alpha, uint64_t leaf, uint64_t count_range,
                           uint64_t guard_depth, oracle_trace *trace,
                           oracle_sub_rec *rec, uint64_t rec_cap,
                           uint64_t *rec_count)
{
    oracle_trace local;
    oracle_trace *tr = trace ? trace : &local;
    memset(tr, 0, sizeof(*tr));
    if (rec_count) *rec_count = 0;
    if (n <= 1) return 0;
    zs_ctx c;
    uint64_t k = (uint64_t)floor(alpha * sqrt((double)n));
    if (k < 2) k = 2;
    c.k = k;
    c.scale = (double)k / 4.0;
    c.leaf = leaf;
    c.count_range = count_range;
    c.guard_depth = guard_depth;
    c.tr = tr;
    c.rec = rec;
    c.rec_cap = rec ? rec_cap : 0;
    c.rec_n = 0;
    tr->k = k;
    tr->scale = c.scale;
    c.count = (uint64_t *)malloc((size_t)(count_range ? count_range : 1) *
                                 sizeof(uint64_t));
    uint64_t *bk = (uint64_t *)malloc((size_t)n * 2 * sizeof(uint64_t));
    uint32_t *bv = (uint32_t *)malloc((size_t)n * 2 * sizeof(uint32_t));
    if (!c.count || !bk || !bv) {
        free(c.count);
        free(bk);
        free(bv);
        return -1;
    }
    /* src = a copy of the input (consumed), dst = the caller's arrays. */
    memcpy(bk, keys, (size_t)n * sizeof(uint64_t));
    memcpy(bv, vals, (size_t)n * sizeof(uint32_t));
    zs_rec(&c, bk, bv, keys, vals, bk + n, bv + n, n, 0, 0.0, 0, 0, 0);
    if (rec_count) *rec_count = c.rec_n;
    free(c.count);
    free(bk);
    free(bv);
    return 0;
}

int oracle_zsort_pairs_ex(uint64_t *keys, uint32_t *vals, uint64_t n,
                          double alpha, uint64_t leaf, uint64_t count_range,
                          uint64_t guard_depth, oracle_trace *trace)
{
    return oracle_zsort_pairs_rec(keys, vals, n, alpha, leaf, count_range,
                                  guard_depth, trace, NULL, 0, NULL);
}

int oracle_zsort_pairs(uint64_t *keys, uint32_t *vals, uint64_t n,
                       oracle_trace *trace)
{
    return oracle_zsort_pairs_ex(keys, vals, n, 0.6, 96, 65000, 32, trace);
}

/* Segment i is [off[i], off[i+1]); each is sorted on its own. */
int oracle_zsort_segmented(uint64_t *keys, uint32_t *vals, const uint64_t *off,
                           uint64_t nseg)
{
    for (uint64_t s = 0; s < nseg; s++) {
        uint64_t a = off[s], b = off[s + 1];
        if (b < a) return -5;
        if (oracle_zsort_pairs(keys + a, vals + a, b - a, NULL) != 0) return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Key encodings.  Two's complement order: flipping the sign bit maps int64
 * order onto uint64 order.  IEEE-754 totalOrder: negative values (sign bit
 * set) have all bits inverted, non-negative values get the sign bit set. */
void oracle_key_from_i64(const int64_t *in, uint64_t *out, uint64_t n)
{
    for (uint64_t i = 0; i < n; i++)
        out[i] = (uint64_t)in[i] ^ 0x8000000000000000ull;
}

void oracle_key_to_i64(const uint64_t *in, int64_t *out, uint64_t n)
{
    for (uint64_t i = 0; i < n; i++)
        out[i] = (int64_t)(in[i] ^ 0x8000000000000000ull);
}

void oracle_key_from_f64(const double *in, uint64_t *out, uint64_t n)
{
    for (uint64_t i = 0; i < n; i++) {
        uint64_t b;
        memcpy(&b, &in[i], 8);
        out[i] = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
    }
}

void oracle_key_to_f64(const uint64_t *in, double *out, uint64_t n)
{
    for (uint64_t i = 0; i < n; i++) {
        uint64_t u = in[i];
        uint64_t b = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
        memcpy(&out[i], &b, 8);
    }
}

/* ------------------------------------------------------------------------ */
/* Learned piecewise-linear CDF bucket map (the z-score map's replacement). */

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the output of generator state
 * x + 1 step, i.e. mix(x + golden gamma). */
uint64_t oracle_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* Stratified sample: stratum i = [floor(i*len/m), floor((i+1)*len/m)); one
 * position drawn in it by splitmix64(seed + i) mod stratum width.  len >= m. */
void oracle_sample_positions(uint64_t seed, uint64_t len, uint64_t m,
                             uint64_t *pos)
{
    for (uint64_t i = 0; i < m; i++) {
        uint64_t lo = (uint64_t)(((u128)i * len) / m);
        uint64_t hi = (uint64_t)(((u128)(i + 1) * len) / m);
        uint64_t w = hi - lo;
        pos[i] = lo + (w ? oracle_splitmix64(seed + i) % w : 0);
    }
}

/* Bit length of r (r >= 1): the E of the normalisation u = fl32(d) * 2^-E. */
static int bitlen64(uint64_t r)
{
    int e = 0;
    while (r) {
        e++;
        r >>= 1;
    }
    return e;
}

/* FP32-normalised key: u = fl32(key - mn) * 2^-E, E = bitlen(mx - mn).
 * The scaling by a power of two is exact, so u lies in [0, 1]. */
float oracle_pwl_normalise(uint64_t key, uint64_t mn, uint64_t mx)
{
    int e = bitlen64(mx - mn);
    volatile float f = (float)(key - mn);
    return f * ldexpf(1.0f, -e);
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

static int cmp_float(const void *a, const void *b)
{
    float x = *(const float *)a, y = *(const float *)b;
    return (x > y) - (x < y);
}

/* Training: breakpoints q[0..P] of the empirical CDF of the normalised sample.
 * q[0] = u(min) = 0, q[P] = u(max), q[j] = j-th P-quantile of the sorted
 * sample, sorted[floor(j*m/P)], for 0 < j < P.  Non-decreasing by
 * construction, so the map below is monotone. */
void oracle_pwl_train(const uint64_t *sample, uint64_t m, uint64_t mn,
                      uint64_t mx, uint32_t P, float *q)
{
    float *u = (float *)malloc((size_t)m * sizeof(float));
    for (uint64_t i = 0; i < m; i++) u[i] = oracle_pwl_normalise(sample[i], mn, mx);
    qsort(u, (size_t)m, sizeof(float), cmp_float);
    q[0] = 0.0f;
    for (uint32_t j = 1; j < P; j++) q[j] = u[(uint64_t)j * m / P];
    q[P] = oracle_pwl_normalise(mx, mn, mx);
    free(u);
}

/* Inference: piece s = #{ 0 < j < P : q[j] <= u }; within it the linear
 * interpolation frac = (u - q[s]) * r[s] with the stored slope (R11)
 * r[s] = fl32(1 / (q[s+1] - q[s])) (0 for an empty piece), clipped to
 * [0, 1 - 2^-24]; bucket = s*K + min(K-1, floor(frac * K)), K = k / P.
 * All arithmetic is IEEE binary32 with round-to-nearest; frac is monotone
 * in u inside a piece and every piece owns its own K buckets, so the map is
 * monotone non-decreasing. */
uint32_t oracle_pwl_bucket(uint64_t key, uint64_t mn, uint64_t mx,
                           const float *q, uint32_t P, uint32_t k)
{
    float u = oracle_pwl_normalise(key, mn, mx);
    uint32_t s = 0;
    for (uint32_t j = 1; j < P; j++)
        if (q[j] <= u) s = j;
    uint32_t K = k / P;
    volatile float lo = q[s], hi = q[s + 1];
    float frac = 0.0f;
    if (hi > lo) {
        volatile float den = hi - lo;
        volatile float r = 1.0f / den;
        volatile float num = u - lo;
        frac = num * r;
    }
    if (frac < 0.0f) frac = 0.0f;
    if (frac > 0.99999994f) frac = 0.99999994f; /* 1 - 2^-24 */
    volatile float t = frac * (float)K;
    uint32_t w = (uint32_t)t;
    if (w > K - 1) w = K - 1;
    return s * K + w;
}

/* Learned map with exact-key breakpoints.  The piecewise-linear map above
 * normalises keys to binary32 first, so keys closer together than the
 * binary32 spacing at their distance from the minimum become one value (a
 * dense interval of width 2^20 near 2^63 collapses to a single u).  This map
 * keeps the breakpoints as keys: b[0] = mn, b[P] = mx, b[j] = the j-th
 * P-quantile key of the sorted sample, sorted[floor(j*m/P)], for 0 < j < P.
 * Piece s = #{ 0 < j < P : b[j] <= key } (keys below mn take piece 0, keys
 * above mx piece P-1); inside it the interpolation is binary32 relative to
 * the piece's own lower key: frac = fl32(fl32(key - b[s]) * r[s]) with the
 * stored slope r[s] = fl32(1 / fl32(b[s+1] - b[s])) (0 for an empty piece),
 * clipped to [0, 1 - 2^-24]; bucket = s*K + min(K-1, floor(frac*K)),
 * K = k / P.  Monotone: the piece is, and each piece owns its K buckets. */
void oracle_split_train(const uint64_t *sample, uint64_t m, uint64_t mn, uint64_t mx, uint32_t P,
                        uint64_t *b, float *r)
{
    uint64_t *srt = (uint64_t *)malloc((size_t)m * sizeof(uint64_t));
    memcpy(srt, sample, (size_t)m * sizeof(uint64_t));
    qsort(srt, (size_t)m, sizeof(uint64_t), cmp_u64);
    b[0] = mn;
    for (uint32_t j = 1; j < P; j++) b[j] = srt[(uint64_t)j * m / P];
    b[P] = mx;
    for (uint32_t j = 0; j < P; j++) {
        if (b[j + 1] > b[j]) {
            volatile float w = (float)(b[j + 1] - b[j]);
            r[j] = 1.0f / w;
        } else {
            r[j] = 0.0f;
        }
    }
    free(srt);
}

uint32_t oracle_split_bucket(uint64_t key, const uint64_t *b, const float *r, uint32_t P, uint32_t k)
{
    uint32_t s = 0;
    for (uint32_t j = 1; j < P; j++)
        if (b[j] <= key) s = j;
    uint32_t K = k / P;
    volatile float d = (float)(key > b[s] ? key - b[s] : 0);
    volatile float frac = d * r[s];
    float f = frac;
    if (f < 0.0f) f = 0.0f;
    if (f > 0.99999994f) f = 0.99999994f; /* 1 - 2^-24 */
    volatile float t = f * (float)K;
    uint32_t w = (uint32_t)t;
    if (w > K - 1) w = K - 1;
    return s * K + w;
}

void oracle_split_buckets(const uint64_t *keys, uint64_t n, const uint64_t *b, const float *r, uint32_t P,
                          uint32_t k, uint32_t *out)
{
    for (uint64_t i = 0; i < n; i++) out[i] = oracle_split_bucket(keys[i], b, r, P, k);
}

/* Level-1 cluster of every key under Eq. 1 (Alg. 1 statistics, R1-R5), as
 * the top level of oracle_zsort_pairs computes it before any guard. */
void oracle_level1_buckets(const uint64_t *keys, uint64_t n, uint64_t k,
                           uint64_t *out)
{
    uint64_t mn, mx;
    double mean, sd;
    oracle_stats(keys, n, &mn, &mx, &mean, &sd);
    double scale = (double)k / 4.0;
    double zmin = fabs((0.0 - mean) / sd);
    for (uint64_t i = 0; i < n; i++)
        out[i] = zmap((double)(keys[i] - mn), mean, sd, zmin, scale, k);
}

/* The learned-map bucket of each of n keys (the same map as above). */
void oracle_pwl_buckets(const uint64_t *keys, uint64_t n, uint64_t mn, uint64_t mx,
                        const float *q, uint32_t P, uint32_t k, uint32_t *out)
{
    for (uint64_t i = 0; i < n; i++) out[i] = oracle_pwl_bucket(keys[i], mn, mx, q, P, k);
}


/* ---------------------------------------------------------------- MLP map
 * Monotone 2-layer MLP: f(u) = sum_{h<H} a_h * clamp(w_h * u + b_h, 0, 1)
 * with a_h = alpha_h^2 and w_h = omega_h^2, so every weight is >= 0 and f is
 * non-decreasing in u by construction; also in binary32, since each step
 * (a product by a non-negative factor, an addition, a clamp, the sum taken
 * in the fixed order h = 0, 1, ...) is a monotone rounding of a monotone
 * function.  The map: g = (f(u) - f(0)) * inv, inv = 1 / (f(u_max) - f(0)),
 * clipped to [0, 1 - 2^-24], bucket = min(k - 1, trunc(g * k)).
 *
 * Training on the P + 1 knots (x_j, y_j) = (q[j], j / P) of the
 * piecewise-linear map (the exact sample quantiles): the squared error
 * sum_j (f(x_j) - y_j)^2 minimised by full-batch resilient gradient descent
 * (each parameter moves by its own step against the sign of its gradient;
 * the step grows by 1.2 while the sign holds and halves, without a move,
 * when it flips), `iters` iterations.  Only gradient signs are used, so the
 * positive factors 2 and a_h of the exact gradients are dropped; a gradient
 * through a unit with a_h = 0 is zero.  Start: unit h is the linear ramp
 * from knot h P/H to knot (h+1) P/H with weight 1/H, i.e. f starts as the
 * H-piece interpolation of the knots.
 *
 * params: omega[H], beta[H], alpha[H], f0, inv (3H + 2 floats).
 * Every operation is an IEEE binary32 operation with round-to-nearest, in
 * the order written (the file is compiled without contraction). */
#define ORACLE_MLP_H 32

static float mlp_forward(const float *om, const float *be, const float *al, float u)
{
    float f = 0.0f;
    for (int h = 0; h < ORACLE_MLP_H; h++) {
        volatile float w = om[h] * om[h];
        volatile float t = w * u;
        volatile float t2 = t + be[h];
        float c = fminf(fmaxf(t2, 0.0f), 1.0f);
        volatile float a = al[h] * al[h];
        volatile float term = a * c;
        f = f + term;
    }
    return f;
}

static void rprop(float *p, float *step, int *sprev, float g)
{
    int sg = (g > 0.0f) - (g < 0.0f);
    if (sg * *sprev < 0) {
        *step = *step * 0.5f;
        *sprev = 0;
        return;
    }
    if (sg * *sprev > 0) *step = *step * 1.2f;
    if (sg > 0) *p = *p - *step;
    if (sg < 0) *p = *p + *step;
    *sprev = sg;
}

void oracle_mlp_train(const float *q, uint32_t P, uint32_t iters, float *params)
{
    const int H = ORACLE_MLP_H;
    float om[ORACLE_MLP_H], be[ORACLE_MLP_H], al[ORACLE_MLP_H];
    float so[ORACLE_MLP_H], sb[ORACLE_MLP_H], sa[ORACLE_MLP_H];
    int po[ORACLE_MLP_H], pb[ORACLE_MLP_H], pa[ORACLE_MLP_H];
    float *r = (float *)malloc((size_t)(P + 1) * sizeof(float));
    for (int h = 0; h < H; h++) {
        float lo = q[(uint64_t)h * P / H], hi = q[(uint64_t)(h + 1) * P / H];
        volatile float den = hi - lo;
        float w = hi > lo ? 1.0f / den : 1048576.0f;
        om[h] = sqrtf(w);
        volatile float lw = lo * w;
        be[h] = -lw;
        al[h] = sqrtf(1.0f / (float)H);
        so[h] = 0.001f * om[h];
        sb[h] = 0.001f;
        sa[h] = 0.001f * al[h];
        po[h] = pb[h] = pa[h] = 0;
    }
    for (uint32_t it = 0; it < iters; it++) {
        for (uint32_t j = 0; j <= P; j++) {
            volatile float y = (float)j / (float)P;
            r[j] = mlp_forward(om, be, al, q[j]) - y;
        }
        for (int h = 0; h < H; h++) {
            volatile float w = om[h] * om[h];
            volatile float a = al[h] * al[h];
            float ga = 0.0f, gw = 0.0f, gb = 0.0f;
            for (uint32_t j = 0; j <= P; j++) {
                volatile float t = w * q[j];
                volatile float t2 = t + be[h];
                float c = fminf(fmaxf(t2, 0.0f), 1.0f);
                volatile float rc = r[j] * c;
                ga = ga + rc;
                if (t2 > 0.0f && t2 < 1.0f) {
                    volatile float rx = r[j] * q[j];
                    gw = gw + rx;
                    gb = gb + r[j];
                }
            }
            if (!(a > 0.0f)) gw = gb = 0.0f;
            volatile float dom = gw * om[h];
            volatile float dal = ga * al[h];
            rprop(&om[h], &so[h], &po[h], dom);
            rprop(&be[h], &sb[h], &pb[h], gb);
            rprop(&al[h], &sa[h], &pa[h], dal);
        }
    }
    for (int h = 0; h < H; h++) {
        params[h] = om[h];
        params[H + h] = be[h];
        params[2 * H + h] = al[h];
    }
    float f0 = mlp_forward(om, be, al, 0.0f);
    float f1 = mlp_forward(om, be, al, q[P]);
    volatile float span = f1 - f0;
    params[3 * H] = f0;
    params[3 * H + 1] = f1 > f0 ? 1.0f / span : 0.0f;
    free(r);
}

uint32_t oracle_mlp_bucket(uint64_t key, uint64_t mn, uint64_t mx, const float *params, uint32_t k)
{
    const int H = ORACLE_MLP_H;
    float u = oracle_pwl_normalise(key, mn, mx);
    float f = mlp_forward(params, params + H, params + 2 * H, u);
    volatile float d = f - params[3 * H];
    volatile float g = d * params[3 * H + 1];
    float gc = fminf(fmaxf(g, 0.0f), 0.99999994f); /* 1 - 2^-24 */
    volatile float t = gc * (float)k;
    uint32_t b = (uint32_t)t;
    return b > k - 1 ? k - 1 : b;
}

void oracle_mlp_buckets(const uint64_t *keys, uint64_t n, uint64_t mn, uint64_t mx, const float *params,
                        uint32_t k, uint32_t *out)
{
    for (uint64_t i = 0; i < n; i++) out[i] = oracle_mlp_bucket(keys[i], mn, mx, params, k);
}

/* f(u) of trained parameters (for the pins: monotonicity, the start state). */
float oracle_mlp_eval(const float *params, float u)
{
    return mlp_forward(params, params + ORACLE_MLP_H, params + 2 * ORACLE_MLP_H, u);
}
