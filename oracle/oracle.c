/*
 * oracle.c -- plain CPU reference for window-pair alignment plots.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code with the CUDA path.
 *
 * What it computes (Krusche & Tiskin, "Computing alignment plots
 * efficiently", Section 2):
 *
 *   For two byte strings x (length m) and y (length n) and a window length w,
 *   the alignment plot holds one value for each pair of w-windows
 *   a = x[i .. i+w) and b = y[j .. j+w), with 0 <= i < m-w and 0 <= j < n-w
 *   (the paper's index ranges {1..m-w} x {1..n-w}, written 0-based).
 *
 *   The value is the best alignment score of a against b, with score
 *   `match` for an aligned pair of equal characters, `mismatch` for an
 *   aligned pair of different characters and 0 for a gap.  Section 2 gets
 *   LCS from the scores (match 1, mismatch 0, gap 0).  It also uses the
 *   scheme (1, 0, -1/2).  Shifting every gap score to zero and doubling gives
 *   the integer scheme (2, 1, 0).  Its optimum is T = S + w, where S is the
 *   score under (1, 0, -1/2).
 *
 *   The score is the textbook dynamic programme over the alignment grid
 *   (Section 2: horizontal and vertical edges score 0, diagonal edges
 *   score the character pair):
 *
 *     D[0][l] = D[k][0] = 0
 *     D[k][l] = max(D[k-1][l], D[k][l-1], D[k-1][l-1] + s(a_k, b_l))
 *
 *   and the plot value is D[w][w].  Repeated for every window pair, this is
 *   the O(m n w^2) method the paper improves on.  Here it is the reference
 *   the fast method is checked against.
 *
 * Work is split over plot rows (or over sample indices) with pthreads.  Each
 * value is computed on its own, so the result does not depend on the thread
 * count.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Best alignment score of a[0..la) against b[0..lb) under (match, mismatch,
 * gap 0), by the recurrence above, keeping one row of D.  `row` must hold
 * lb + 1 ints. */
int64_t oracle_pair_score(const uint8_t *a, int64_t la, const uint8_t *b,
                          int64_t lb, int32_t match, int32_t mismatch,
                          int32_t *row)
{
    for (int64_t l = 0; l <= lb; ++l) row[l] = 0;       /* D[0][l] = 0 */
    for (int64_t k = 1; k <= la; ++k) {
        int32_t diag = row[0];                          /* D[k-1][0] */
        row[0] = 0;                                     /* D[k][0] = 0 */
        for (int64_t l = 1; l <= lb; ++l) {
            int32_t up = row[l];                        /* D[k-1][l] */
            int32_t left = row[l - 1];                  /* D[k][l-1] */
            int32_t s = (a[k - 1] == b[l - 1]) ? match : mismatch;
            int32_t best = diag + s;
            if (up > best) best = up;
            if (left > best) best = left;
            diag = up;                                  /* D[k-1][l] for l+1 */
            row[l] = best;
        }
    }
    return row[lb];
}

typedef struct {
    const uint8_t *x, *y;
    int64_t m, n, w;
    int32_t match, mismatch;
    int32_t *out;
    int64_t ld;
    /* full plot: rows [r0, r1); samples: indices [r0, r1) */
    const int64_t *ii, *jj;
    int64_t r0, r1;
} job_t;

static void *plot_worker(void *arg)
{
    job_t *jb = (job_t *)arg;
    int32_t *row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(jb->w + 1));
    int64_t cols = jb->n - jb->w;
    for (int64_t i = jb->r0; i < jb->r1; ++i)
        for (int64_t j = 0; j < cols; ++j)
            jb->out[i * jb->ld + j] = (int32_t)oracle_pair_score(
                jb->x + i, jb->w, jb->y + j, jb->w, jb->match, jb->mismatch,
                row);
    free(row);
    return NULL;
}

static void *sample_worker(void *arg)
{
    job_t *jb = (job_t *)arg;
    int32_t *row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(jb->w + 1));
    for (int64_t s = jb->r0; s < jb->r1; ++s)
        jb->out[s] = (int32_t)oracle_pair_score(jb->x + jb->ii[s], jb->w,
                                                jb->y + jb->jj[s], jb->w,
                                                jb->match, jb->mismatch, row);
    free(row);
    return NULL;
}

static int run_split(void *(*fn)(void *), job_t base, int64_t total,
                     int nthreads)
{
    if (total <= 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > total) nthreads = (int)total;
    pthread_t th[256];
    job_t jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = base;
        jobs[t].r0 = total * t / nthreads;
        jobs[t].r1 = total * (t + 1) / nthreads;
        if (pthread_create(&th[t], NULL, fn, &jobs[t]) != 0) {
            /* fall back to running this share on the calling thread */
            fn(&jobs[t]);
            th[t] = 0;
        }
    }
    for (int t = 0; t < nthreads; ++t)
        if (th[t]) pthread_join(th[t], NULL);
    return 0;
}

/* Full plot: out[i*ld + j] for 0 <= i < m-w, 0 <= j < n-w.  Returns 0, or -1
 * on bad arguments.  An empty plot (m <= w or n <= w) writes nothing. */
int oracle_plot(const uint8_t *x, int64_t m, const uint8_t *y, int64_t n,
                int64_t w, int32_t match, int32_t mismatch, int32_t *out,
                int64_t ld, int nthreads)
{
    if (w < 1 || m < 0 || n < 0) return -1;
    if (m <= w || n <= w) return 0;
    if (ld < n - w) return -1;
    job_t b;
    memset(&b, 0, sizeof b);
    b.x = x; b.y = y; b.m = m; b.n = n; b.w = w;
    b.match = match; b.mismatch = mismatch; b.out = out; b.ld = ld;
    return run_split(plot_worker, b, m - w, nthreads);
}

/* Sampled plot values: out[s] = plot(ii[s], jj[s]).  Indices must lie in the
 * plot; returns -1 if any does not. */
int oracle_samples(const uint8_t *x, int64_t m, const uint8_t *y, int64_t n,
                   int64_t w, int32_t match, int32_t mismatch,
                   const int64_t *ii, const int64_t *jj, int64_t count,
                   int32_t *out, int nthreads)
{
    if (w < 1) return -1;
    for (int64_t s = 0; s < count; ++s)
        if (ii[s] < 0 || ii[s] >= m - w || jj[s] < 0 || jj[s] >= n - w)
            return -1;
    job_t b;
    memset(&b, 0, sizeof b);
    b.x = x; b.y = y; b.m = m; b.n = n; b.w = w;
    b.match = match; b.mismatch = mismatch; b.out = out;
    b.ii = ii; b.jj = jj;
    return run_split(sample_worker, b, count, nthreads);
}

/* ---------------------------------------------------------------------------
 * Digest of a whole plot without storing it (for plots too large to hold):
 *     result[0]     = sum over cells of P[r][j] * (r*2654435761 + j*40503 + 1)
 *                     mod 2^64
 *     result[1 + v] = number of cells with value v, for v < nbins
 * over plot rows r = 0, 1, ... where row r is the x-window starting at
 * r * step (step 1: the full plot).  Each value is the recurrence above.
 * ------------------------------------------------------------------------- */

typedef struct {
    const uint8_t *x, *y;
    int64_t w, step, cols;
    int32_t match, mismatch;
    int32_t nbins;
    uint64_t *acc;
    int64_t r0, r1;
} digest_job_t;

static void *digest_worker(void *arg)
{
    digest_job_t *jb = (digest_job_t *)arg;
    int32_t *row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(jb->w + 1));
    for (int64_t r = jb->r0; r < jb->r1; ++r) {
        const uint64_t wr = (uint64_t)r * 2654435761ull + 1ull;
        for (int64_t j = 0; j < jb->cols; ++j) {
            const int64_t v = oracle_pair_score(jb->x + r * jb->step, jb->w, jb->y + j, jb->w,
                                                jb->match, jb->mismatch, row);
            jb->acc[0] += (uint64_t)v * (wr + (uint64_t)j * 40503ull);
            if (v >= 0 && v < jb->nbins) jb->acc[1 + v] += 1;
        }
    }
    free(row);
    return NULL;
}

int oracle_plot_digest(const uint8_t *x, int64_t m, const uint8_t *y, int64_t n, int64_t w,
                       int32_t match, int32_t mismatch, int64_t step, int32_t nbins,
                       uint64_t *result, int nthreads)
{
    if (w < 1 || m < 0 || n < 0 || step < 1 || nbins < 0) return -1;
    for (int32_t k = 0; k <= nbins; ++k) result[k] = 0;
    const int64_t rows = m > w ? (m - w + step - 1) / step : 0;
    const int64_t cols = n > w ? n - w : 0;
    if (rows == 0 || cols == 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > rows) nthreads = (int)rows;
    uint64_t *acc = (uint64_t *)calloc((size_t)nthreads * (size_t)(1 + nbins), sizeof(uint64_t));
    pthread_t th[256];
    digest_job_t jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        digest_job_t *jb = &jobs[t];
        jb->x = x; jb->y = y; jb->w = w; jb->step = step; jb->cols = cols;
        jb->match = match; jb->mismatch = mismatch; jb->nbins = nbins;
        jb->acc = acc + (size_t)t * (size_t)(1 + nbins);
        jb->r0 = rows * t / nthreads;
        jb->r1 = rows * (t + 1) / nthreads;
        if (pthread_create(&th[t], NULL, digest_worker, jb) != 0) {
            digest_worker(jb);
            th[t] = 0;
        }
    }
    for (int t = 0; t < nthreads; ++t)
        if (th[t]) pthread_join(th[t], NULL);
    for (int t = 0; t < nthreads; ++t)
        for (int32_t k = 0; k <= nbins; ++k) result[k] += acc[(size_t)t * (size_t)(1 + nbins) + k];
    free(acc);
    return 0;
}
