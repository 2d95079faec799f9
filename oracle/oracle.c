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
