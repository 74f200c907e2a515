/*
 * FP64 CPU oracle for PALMAD discord discovery (Zymbler & Kraeva,
 * "High-performance Time Series Anomaly Discovery on Graphics Processor").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header
 * or constant with the CUDA library: it reads the same float32 series and
 * nothing else.
 *
 * Everything is double precision and deliberately plain:
 *   - window mean / standard deviation:  Eq. 4, evaluated two-pass
 *     (mu = sum/m, sigma^2 = sum (x-mu)^2 / m, algebraically Eq. 4's
 *     (1/m) sum x^2 - mu^2, chosen for FP64 accuracy);
 *   - distance: Eq. 5 applied to the z-normalised windows of Eq. 4
 *     (NOT the dot-product form of Eq. 6, which the GPU uses);
 *   - non-self match |i - j| >= m (Sec. 2.1), range discord
 *     min Dist >= r (Sec. 2.1);
 *   - brute-force non-self-match nearest neighbour ("matrix profile");
 *   - range discords at r (Sec. 2.1), evaluated from their definition
 *     window by window; this is the set one DRAG call (Algorithm 2)
 *     returns;
 *   - MERLIN's threshold schedule over lengths minL..maxL, as the prose
 *     of Sec. 2.2 describes it;
 *   - greedy top-K and the discord heatmap of Eq. 10;
 *   - the k-th non-self neighbour variant (reading R14) by brute force.
 *
 * Readings of the paper taken here (the paper is garbled or silent):
 *   R1  r is in distance units; every comparison is d < r on the plain
 *       (not squared) z-normalised Euclidean distance.
 *   R2  A window whose sigma <= 2^-22 |mu| is flat.  Two flat windows are at
 *       distance 0; a flat and a non-flat window are at distance sqrt(2m)
 *       (correlation taken as 0 in Eq. 6).
 *   R3  A window with no non-self match (possible when n - m + 1 < 2m) has
 *       no nearest neighbour and is never a discord.
 *   R4  One DRAG call at r outputs the range discords at r (Sec. 2.1), each
 *       with its exact nearest-neighbour distance.  The refine phase of
 *       Algorithm 2 adds a candidate to its output while the scan is still
 *       running; that is read as keeping the candidate until the scan ends.
 *   R5  Top-K per length: the range discords sorted by (nnDist desc, index
 *       asc), taken greedily; with `exclusive` set, a pick must be at least
 *       m away from every earlier pick.
 *   R6  A DRAG call "succeeds" when R5 yields K picks; nnDist_m (the value
 *       fed to the schedule) is the distance of the K-th pick.
 *   R7  Sec. 2.2, lengths two to five: the first try is 1% below the
 *       previous length's nnDist and each failure takes off another 1% of
 *       the current r (r <- 0.99 r).  Later lengths: the first try is
 *       mean - 2 sd of the last five nnDist (sample deviation, n-1), and
 *       each failure subtracts sd; no try repeats an unchanged r.  If sd is
 *       0 the step is 0.01 mean.
 *   R8  Loop guards (not in the paper): after 60 halvings, 3000 shrinks of
 *       1%, or any r <= 0, the call is made with r = 0, where every window
 *       with a non-self match qualifies; fewer than K picks are then
 *       returned as they are.
 *   R9  Heatmap (Eq. 10): row m, column i holds nnDist^2 / (2m) for the
 *       range discords at the final r of that length and 0 elsewhere; the
 *       row width is n - minL + 1.
 *   R14 k-th neighbour variant (the top-k discord definition of Sec. 2.1,
 *       read literally): the k-distance of window i is the k-th smallest
 *       distance to its non-self matches j (|i - j| >= m), every such j
 *       counted, so neighbours may overlap one another.  k = 1 is the
 *       nearest-neighbour distance.  A window with fewer than k non-self
 *       matches has no k-distance and is never a discord.  The range
 *       k-discords at r are the windows whose k-distance is >= r; MERLIN
 *       runs unchanged on the k-distance.
 *   R13 Discord interest (Eq. 11, Sec. 5): the interest of index i is the
 *       largest heatmap value over the lengths, and its length the smallest
 *       m reaching it.  The top-k interesting discords are taken greedily
 *       by (interest desc, index asc) among indices of positive interest;
 *       with `exclusive` set, a pick's window [i, i + m) must not overlap an
 *       earlier pick's window.
 *
 * Parallelism: the brute-force nearest neighbour and the range-discord
 * test run their windows in parallel; each window's result depends on that
 * window alone, so the output equals the serial loop's.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_FLAT_REL 2.384185791015625e-07 /* 2^-22 */

/* ---------- window statistics (Eq. 4) ---------- */

static void window_stats(const float *T, int64_t i, int32_t m, double *mu, double *sd) {
    double s = 0.0;
    for (int32_t k = 0; k < m; ++k) s += (double)T[i + k];
    double mean = s / (double)m;
    double v = 0.0;
    for (int32_t k = 0; k < m; ++k) {
        double d = (double)T[i + k] - mean;
        v += d * d;
    }
    *mu = mean;
    *sd = sqrt(v / (double)m);
}

static int is_flat(double mu, double sd) { return sd <= ORACLE_FLAT_REL * fabs(mu); }

int oracle_stats(const float *T, int64_t n, int32_t m, double *mu, double *sd) {
    if (!T || !mu || !sd || m < 1 || n < m) return -1;
    int64_t N = n - m + 1;
    for (int64_t i = 0; i < N; ++i) window_stats(T, i, m, &mu[i], &sd[i]);
    return 0;
}

/* ---------- distance (Eq. 5 on the z-normalised windows of Eq. 4) ---------- */

/* Squared z-normalised Euclidean distance (Eq. 5 on Eq. 4). */
static double zdist2(const float *T, int32_t m, int64_t i, int64_t j, double mui, double sdi,
                     double muj, double sdj) {
    int fi = is_flat(mui, sdi), fj = is_flat(muj, sdj);
    if (fi && fj) return 0.0;
    if (fi || fj) return 2.0 * (double)m;
    double s = 0.0;
    for (int32_t k = 0; k < m; ++k) {
        double a = ((double)T[i + k] - mui) / sdi;
        double b = ((double)T[j + k] - muj) / sdj;
        double d = a - b;
        s += d * d;
    }
    return s;
}

double oracle_dist(const float *T, int64_t n, int32_t m, int64_t i, int64_t j) {
    if (!T || m < 1 || i < 0 || j < 0 || i + m > n || j + m > n) return NAN;
    double mui, sdi, muj, sdj;
    window_stats(T, i, m, &mui, &sdi);
    window_stats(T, j, m, &muj, &sdj);
    return sqrt(zdist2(T, m, i, j, mui, sdi, muj, sdj));
}

/* ---------- brute-force nearest non-self match ---------- */

int oracle_mp(const float *T, int64_t n, int32_t m, double *mp, int64_t *mpidx) {
    if (!T || !mp || m < 1 || n < m) return -1;
    int64_t N = n - m + 1;
    double *mu = (double *)malloc(sizeof(double) * N), *sd = (double *)malloc(sizeof(double) * N);
    if (!mu || !sd) { free(mu); free(sd); return -2; }
    oracle_stats(T, n, m, mu, sd);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i) {
        double best = INFINITY;
        int64_t arg = -1;
        for (int64_t j = 0; j < N; ++j) {
            if (llabs(i - j) < m) continue;
            double d2 = zdist2(T, m, i, j, mu[i], sd[i], mu[j], sd[j]);
            if (d2 < best) { best = d2; arg = j; }
        }
        mp[i] = sqrt(best);
        if (mpidx) mpidx[i] = arg;
    }
    free(mu);
    free(sd);
    return 0;
}

/* Nearest non-self match of one window (one row of the brute force above). */
int oracle_nn_one(const float *T, int64_t n, int32_t m, int64_t i, double *nn, int64_t *nnidx) {
    if (!T || !nn || m < 1 || n < m || i < 0 || i > n - m) return -1;
    int64_t N = n - m + 1;
    double mui, sdi;
    window_stats(T, i, m, &mui, &sdi);
    double best = INFINITY;
    int64_t arg = -1;
#pragma omp parallel
    {
        double lb = INFINITY;
        int64_t la = -1;
#pragma omp for schedule(static)
        for (int64_t j = 0; j < N; ++j) {
            if (llabs(i - j) < m) continue;
            double muj, sdj;
            window_stats(T, j, m, &muj, &sdj);
            double d2 = zdist2(T, m, i, j, mui, sdi, muj, sdj);
            if (d2 < lb || (d2 == lb && j < la)) { lb = d2; la = j; }
        }
#pragma omp critical
        {
            if (lb < best || (lb == best && la >= 0 && la < arg)) { best = lb; arg = la; }
        }
    }
    *nn = sqrt(best);
    if (nnidx) *nnidx = arg;
    return 0;
}

/* ---------- k-th non-self neighbour (reading R14) ---------- */

static int cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* knn[i] = the k-th smallest distance from window i to its non-self
 * matches, by brute force (all distances of the row, sorted); INFINITY when
 * the window has fewer than k non-self matches. */
int oracle_knn(const float *T, int64_t n, int32_t m, int32_t k, double *knn) {
    if (!T || !knn || m < 1 || n < m || k < 1) return -1;
    int64_t N = n - m + 1;
    double *mu = (double *)malloc(sizeof(double) * N), *sd = (double *)malloc(sizeof(double) * N);
    if (!mu || !sd) { free(mu); free(sd); return -2; }
    oracle_stats(T, n, m, mu, sd);
    int bad = 0;
#pragma omp parallel
    {
        double *row = (double *)malloc(sizeof(double) * N);
        if (!row) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < N; ++i) {
            if (!row) continue;
            int64_t cnt = 0;
            for (int64_t j = 0; j < N; ++j) {
                if (llabs(i - j) < m) continue;
                row[cnt++] = zdist2(T, m, i, j, mu[i], sd[i], mu[j], sd[j]);
            }
            if (cnt < k) { knn[i] = INFINITY; continue; }
            qsort(row, (size_t)cnt, sizeof(double), cmp_double);
            knn[i] = sqrt(row[k - 1]);
        }
        free(row);
    }
    free(mu);
    free(sd);
    return bad ? -2 : 0;
}

/* Range k-discords at r (reading R14): the windows whose k-distance is
 * finite and >= r (every finite one when r <= 0), ascending; up to `cap`
 * written, *count receives the full number.  `knn` may hold the profile
 * from oracle_knn, or be NULL to compute it here. */
int oracle_drag_knn(const float *T, int64_t n, int32_t m, int32_t k, double r, const double *knn,
                    int64_t *out_idx, double *out_nn, int64_t cap, int64_t *count) {
    if (!T || m < 1 || n < m || k < 1 || !count) return -1;
    int64_t N = n - m + 1;
    double *own = NULL;
    if (!knn) {
        own = (double *)malloc(sizeof(double) * N);
        if (!own) return -2;
        int rc = oracle_knn(T, n, m, k, own);
        if (rc) { free(own); return rc; }
        knn = own;
    }
    int64_t c = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (!isfinite(knn[i]) || (r > 0.0 && knn[i] < r)) continue;
        if (c < cap) {
            if (out_idx) out_idx[c] = i;
            if (out_nn) out_nn[c] = knn[i];
        }
        ++c;
    }
    *count = c;
    free(own);
    return 0;
}

/* ---------- range discords (Sec. 2.1) ---------- */

/*
 * The range discords of length m at threshold r: the windows whose nearest
 * non-self match lies at distance >= r, each with that distance (nnDist).
 * DRAG (Algorithm 2) computes exactly this set; here it is evaluated from
 * the definition, one window at a time.  Window i is compared with its
 * non-self matches j in ascending order.  A j with Dist(i, j) < r shows that
 * i is not a range discord (the "for every non-self match" of the definition
 * fails there), and the test of i ends.  Otherwise nnDist(i) is the minimum
 * over every j.  With r <= 0 every window with a non-self match qualifies
 * (R8); a window with none never does (R3).
 *
 * Writes up to `cap` (index, nnDist) pairs in ascending index order;
 * *count receives the full number.  Returns 0, or a negative value on bad
 * arguments / allocation failure.
 */
/* The definition applied to window i: its nnDist when it is a range
 * discord at r, NAN otherwise. */
static double range_discord_test(const float *T, int32_t m, int64_t N, int64_t i, double r, const double *mu,
                                 const double *sd) {
    double best = INFINITY;
    for (int64_t j = 0; j < N; ++j) {
        if (llabs(i - j) < m) continue;
        double d = sqrt(zdist2(T, m, i, j, mu[i], sd[i], mu[j], sd[j]));
        if (r > 0.0 && d < r) return NAN;
        if (d < best) best = d;
    }
    return isfinite(best) ? best : NAN;
}

int oracle_range_discords(const float *T, int64_t n, int32_t m, double r, int64_t *out_idx, double *out_nn,
                          int64_t cap, int64_t *count) {
    if (!T || m < 1 || n < m || !count) return -1;
    int64_t N = n - m + 1;
    double *mu = (double *)malloc(sizeof(double) * N), *sd = (double *)malloc(sizeof(double) * N);
    double *nn = (double *)malloc(sizeof(double) * N);  /* nnDist, or NAN: not a range discord */
    if (!mu || !sd || !nn) { free(mu); free(sd); free(nn); return -2; }
    oracle_stats(T, n, m, mu, sd);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < N; ++i) nn[i] = range_discord_test(T, m, N, i, r, mu, sd);
    int64_t c = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (isnan(nn[i])) continue;
        if (c < cap) {
            if (out_idx) out_idx[c] = i;
            if (out_nn) out_nn[c] = nn[i];
        }
        ++c;
    }
    *count = c;
    free(mu); free(sd); free(nn);
    return 0;
}

/* The same test for the listed windows only: out_nn[q] is the nnDist of
 * window idx[q] when it is a range discord at r, NAN otherwise. */
int oracle_range_discord_windows(const float *T, int64_t n, int32_t m, double r, const int64_t *idx, int64_t count,
                                 double *out_nn) {
    if (!T || m < 1 || n < m || (count > 0 && (!idx || !out_nn))) return -1;
    int64_t N = n - m + 1;
    for (int64_t q = 0; q < count; ++q)
        if (idx[q] < 0 || idx[q] >= N) return -1;
    double *mu = (double *)malloc(sizeof(double) * N), *sd = (double *)malloc(sizeof(double) * N);
    if (!mu || !sd) { free(mu); free(sd); return -2; }
    oracle_stats(T, n, m, mu, sd);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < count; ++q) out_nn[q] = range_discord_test(T, m, N, idx[q], r, mu, sd);
    free(mu); free(sd);
    return 0;
}

/* ---------- greedy top-K (reading R5) ---------- */

typedef struct { int64_t idx; double nn; } pick_t;

static int cmp_pick(const void *a, const void *b) {
    const pick_t *x = (const pick_t *)a, *y = (const pick_t *)b;
    if (x->nn > y->nn) return -1;
    if (x->nn < y->nn) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

int oracle_topk(const int64_t *idx, const double *nn, int64_t count, int32_t m, int32_t K, int exclusive,
                int64_t *out_idx, double *out_nn) {
    if (K < 1 || count < 0) return -1;
    pick_t *p = (pick_t *)malloc(sizeof(pick_t) * (count > 0 ? count : 1));
    if (!p) return -2;
    for (int64_t q = 0; q < count; ++q) { p[q].idx = idx[q]; p[q].nn = nn[q]; }
    qsort(p, (size_t)count, sizeof(pick_t), cmp_pick);
    int32_t got = 0;
    for (int64_t q = 0; q < count && got < K; ++q) {
        int ok = 1;
        if (exclusive)
            for (int32_t g = 0; g < got; ++g)
                if (llabs(p[q].idx - out_idx[g]) < m) { ok = 0; break; }
        if (ok) { out_idx[got] = p[q].idx; out_nn[got] = p[q].nn; ++got; }
    }
    for (int32_t g = got; g < K; ++g) { out_idx[g] = -1; out_nn[g] = 0.0; }
    free(p);
    return got;
}

/* ---------- MERLIN over a length range (Sec. 2.2) ---------- */

/* Range discords of one length at one r, into a buffer that grows as needed. */
typedef struct {
    int64_t *idx; double *nn; int64_t cap; int64_t count;
    int32_t knn;           /* k of reading R14 (1: nearest neighbour) */
    const double *prof;    /* k-distances of the current length when knn > 1 */
} discord_set;

static int find_range_discords(const float *T, int64_t n, int32_t m, double r, discord_set *b) {
    for (;;) {
        int64_t cnt = 0;
        int rc = b->knn > 1 ? oracle_drag_knn(T, n, m, b->knn, r, b->prof, b->idx, b->nn, b->cap, &cnt)
                            : oracle_range_discords(T, n, m, r, b->idx, b->nn, b->cap, &cnt);
        if (rc) return rc;
        if (cnt <= b->cap) { b->count = cnt; return 0; }
        free(b->idx); free(b->nn);
        b->cap = cnt;
        b->idx = (int64_t *)malloc(sizeof(int64_t) * cnt);
        b->nn = (double *)malloc(sizeof(double) * cnt);
        if (!b->idx || !b->nn) return -2;
    }
}

/*
 * How Sec. 2.2 chooses r for the length with schedule index l (l = m - minL)
 * from the nnDist values of the lengths before it (prev[0 .. l-1]): the
 * first try, and how a failed try lowers r (next = r * scale - minus).
 *   l = 0      2 sqrt(minL), the largest possible z-normalised distance,
 *              halved per failure;
 *   l = 1..4   the previous length's nnDist less 1%, then 1% of r less per
 *              failure (R7);
 *   l >= 5     mean - 2 sd of the last five nnDist values (sample deviation),
 *              sd less per failure; 0.01 mean when sd is 0 (R7).
 * The try counts after which r drops to 0 are reading R8.
 */
typedef struct { double first, scale, minus; int max_tries; } r_rule;

static r_rule threshold_rule(int32_t l, int32_t minL, const double *prev) {
    r_rule q;
    if (l == 0) {
        q.first = 2.0 * sqrt((double)minL);
        q.scale = 0.5;
        q.minus = 0.0;
        q.max_tries = 60;
    } else if (l < 5) {
        q.first = 0.99 * prev[l - 1];
        q.scale = 0.99;
        q.minus = 0.0;
        q.max_tries = 3000;
    } else {
        const double *last5 = prev + (l - 5);
        double mean = 0.0, ss = 0.0;
        for (int k = 0; k < 5; ++k) mean += last5[4 - k];
        mean /= 5.0;
        for (int k = 0; k < 5; ++k) ss += (last5[4 - k] - mean) * (last5[4 - k] - mean);
        const double sd = sqrt(ss / 4.0);
        q.first = mean - 2.0 * sd;
        q.scale = 1.0;
        q.minus = sd > 0.0 ? sd : 0.01 * mean;
        q.max_tries = 3000;
    }
    return q;
}

/*
 * out_idx/out_nn: [L*K] picks per length (index -1 and 0.0 when fewer);
 * out_count: [L] number of range discords at the final r; out_r: [L] final r;
 * out_calls: [L] range-discord evaluations (DRAG calls) made; out_heat:
 * [L*(n-minL+1)] or NULL.
 *
 * Lengths run in increasing order.  For each, r starts at its rule's first
 * try; a try succeeds when the greedy top-K of the range discords at r
 * (R5) yields K picks (R6).  A try with r <= 0 is the last one.  The K-th
 * pick's nnDist is what later lengths' rules read.
 */
int oracle_merlin_knn(const float *T, int64_t n, int32_t minL, int32_t maxL, int32_t K, int exclusive,
                      int32_t knn, int64_t *out_idx, double *out_nn, int64_t *out_count, double *out_r,
                      int32_t *out_calls, float *out_heat) {
    if (!T || minL < 3 || maxL < minL || n < 2 * (int64_t)maxL || K < 1 || knn < 1) return -1;
    const int32_t L = maxL - minL + 1;
    const int64_t W = n - minL + 1;
    discord_set b = {0};
    b.cap = 1024;
    b.knn = knn;
    b.idx = (int64_t *)malloc(sizeof(int64_t) * b.cap);
    b.nn = (double *)malloc(sizeof(double) * b.cap);
    double *nndist = (double *)malloc(sizeof(double) * L); /* the value each length passes on */
    /* k-distances of one length: every try at that length thresholds them */
    double *prof = knn > 1 ? (double *)malloc(sizeof(double) * (size_t)(n - minL + 1)) : NULL;
    if (!b.idx || !b.nn || !nndist || (knn > 1 && !prof)) {
        free(b.idx); free(b.nn); free(nndist); free(prof);
        return -2;
    }
    if (out_heat) memset(out_heat, 0, sizeof(float) * (size_t)L * (size_t)W);
    int rc = 0;
    for (int32_t l = 0; l < L && !rc; ++l) {
        const int32_t m = minL + l;
        if (knn > 1) {
            rc = oracle_knn(T, n, m, knn, prof);
            if (rc) break;
            b.prof = prof;
        }
        int64_t *pidx = out_idx + (int64_t)l * K;
        double *pnn = out_nn + (int64_t)l * K;
        const r_rule rule = threshold_rule(l, minL, nndist);
        double r = rule.first;
        int tries = 0;
        for (;;) {
            if (tries >= rule.max_tries || r <= 0.0) r = 0.0;
            rc = find_range_discords(T, n, m, r, &b);
            ++tries;
            if (rc) break;
            const int got = oracle_topk(b.idx, b.nn, b.count, m, K, exclusive, pidx, pnn);
            if (got < 0) { rc = got; break; }
            if (got == K || r <= 0.0) break;
            r = rule.minus > 0.0 || rule.scale < 1.0 ? r * rule.scale - rule.minus : 0.0;
        }
        if (rc) break;
        /* the K-th pick's distance, or the last pick's when fewer (R6, R8) */
        int got = 0;
        while (got < K && pidx[got] >= 0) ++got;
        nndist[l] = got > 0 ? pnn[got - 1] : 0.0;
        if (out_count) out_count[l] = b.count;
        if (out_r) out_r[l] = r;
        if (out_calls) out_calls[l] = tries;
        if (out_heat) {
            float *row = out_heat + (int64_t)l * W;
            for (int64_t q = 0; q < b.count; ++q)
                row[b.idx[q]] = (float)(b.nn[q] * b.nn[q] / (2.0 * (double)m));
        }
    }
    free(b.idx); free(b.nn); free(nndist); free(prof);
    return rc;
}

int oracle_merlin(const float *T, int64_t n, int32_t minL, int32_t maxL, int32_t K, int exclusive,
                  int64_t *out_idx, double *out_nn, int64_t *out_count, double *out_r,
                  int32_t *out_calls, float *out_heat) {
    return oracle_merlin_knn(T, n, minL, maxL, K, exclusive, 1, out_idx, out_nn, out_count, out_r, out_calls,
                             out_heat);
}

/* ---------- discord interest across lengths (Eq. 11, reading R13) ---------- */

/*
 * heat: [L * W] row-major by length (row l is length minL + l).
 * score / best_m: [W] per index, or NULL.  out_idx / out_m / out_score: [K]
 * picks, -1 / 0 / 0 past the last one.  Returns the number of picks.
 */
int oracle_interest(const float *heat, int32_t L, int64_t W, int32_t minL, int32_t K, int exclusive, float *score,
                    int32_t *best_m, int64_t *out_idx, int32_t *out_m, float *out_score) {
    if (!heat || L < 1 || W < 1 || K < 1) return -1;
    float *sc = (float *)malloc(sizeof(float) * (size_t)W);
    int32_t *bm = (int32_t *)malloc(sizeof(int32_t) * (size_t)W);
    if (!sc || !bm) { free(sc); free(bm); return -2; }
    for (int64_t i = 0; i < W; ++i) {
        float best = heat[i];
        int32_t at = 0;
        for (int32_t l = 1; l < L; ++l) {
            const float v = heat[(int64_t)l * W + i];
            if (v > best) { best = v; at = l; }
        }
        sc[i] = best;
        bm[i] = minL + at;
    }
    int32_t got = 0;
    for (; got < K; ++got) {
        int64_t pick = -1;
        for (int64_t i = 0; i < W; ++i) {
            if (!(sc[i] > 0.0f)) continue;
            if (pick >= 0 && !(sc[i] > sc[pick])) continue; /* ties keep the lower index */
            int ok = 1;
            for (int32_t g = 0; g < got && ok; ++g) {
                if (out_idx[g] == i) ok = 0;
                else if (exclusive && i < out_idx[g] + out_m[g] && out_idx[g] < i + bm[i]) ok = 0;
            }
            if (ok) pick = i;
        }
        if (pick < 0) break;
        out_idx[got] = pick;
        out_m[got] = bm[pick];
        out_score[got] = sc[pick];
    }
    for (int32_t g = got; g < K; ++g) { out_idx[g] = -1; out_m[g] = 0; out_score[g] = 0.0f; }
    if (score) memcpy(score, sc, sizeof(float) * (size_t)W);
    if (best_m) memcpy(best_m, bm, sizeof(int32_t) * (size_t)W);
    free(sc); free(bm);
    return got;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
