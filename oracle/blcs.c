/*
 * blcs.c -- a second CPU reference for large alignment plots: bit-parallel
 * LCS per window pair.
 *
 * TEST INFRASTRUCTURE ONLY, like oracle.c.  Nothing in the product library
 * calls, links or loads this file, and it shares no code with the CUDA
 * path.  The tests check it against oracle.c's dynamic programme and the
 * brute-force pins before any stored value it writes is trusted.
 *
 * What it computes: the same plot as oracle.c (Krusche & Tiskin, "Computing
 * alignment plots efficiently", Section 2), by a different method.  Section 4
 * compares the paper's method with "BLCS", the bit-parallel LCS algorithm of
 * Crochemore, Iliopoulos, Pinzon and Reid (2001), run once per window pair.
 * That algorithm keeps one bit per character of the first string a:
 *
 *     PM[c]  = bit set of the positions p with a[p] == c
 *     V      = all ones (one bit per character of a)
 *     for every character c of b, in order:
 *         V = (V + (V & PM[c])) | (V & ~PM[c])        (addition with carry)
 *     LLCS(a, b) = number of zero bits among the low |a| bits of V.
 *
 * It costs O(|a| |b| / 64) word operations per pair, against O(|a| |b|) for
 * the dynamic programme, which makes digests of whole 10^10-cell plots
 * affordable on the host.
 *
 * Scores {nu, mu, 0} (0 < mu < nu, or the LCS nu = 1, mu = 0) go through
 * the blow-up of Section 2: every character becomes mu copies of a new
 * character '$' followed by nu - mu copies of itself, and the best
 * {nu, mu, 0} alignment score of two windows is the LLCS of their blown-up
 * forms.  (For {2,1,0} this is the paper's '$' before every character.)
 * '$' is coded as 256, outside the byte alphabet, so no byte value is
 * reserved.  The reduction is checked by brute force in the tests.
 *
 * The plot may take every step-th x-window (Section 3's vertical step h):
 * plot row r is the x-window starting at r * step.
 *
 * Digest of a plot (what the GPU's checksum kernel also reports):
 *     checksum = sum over cells of P[r][j] * (r*2654435761 + j*40503 + 1)
 *                mod 2^64
 *     hist[v]  = number of cells with value v, for v < nbins.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define BLCS_DOLLAR 256          /* the blow-up's extra character */
#define BLCS_SYMS 257
#define BLCS_MAXW 16             /* 64-bit words per blown-up window: 1024 */

typedef struct {
    const uint8_t *x, *y;
    int64_t m, n, w, step, rows, cols;
    int nu, mu, nw;              /* blow-up, words per blown-up window */
    int32_t *out;                /* full plot, or NULL for a digest */
    int64_t ld;
    int nbins;
    uint64_t *acc;               /* this share's checksum + nbins counts */
    int64_t r0, r1;              /* plot rows of this share */
} blcs_job;

/* Characters of the blown-up window of s[0..w): unit k becomes mu '$' then
 * nu - mu copies of s[k]. */
static int blow_window(const uint8_t *s, int64_t w, int nu, int mu, int *outc)
{
    int L = 0;
    for (int64_t k = 0; k < w; ++k) {
        for (int t = 0; t < mu; ++t) outc[L++] = BLCS_DOLLAR;
        for (int t = mu; t < nu; ++t) outc[L++] = s[k];
    }
    return L;
}

/* LLCS of the blown-up a (given by its match table pm, L bits in nw words)
 * and the blown-up window b[0..lb). */
static int64_t blcs_llcs(const uint64_t *pm, int L, int nw, const int *b, int lb)
{
    uint64_t V[BLCS_MAXW];
    for (int q = 0; q < nw; ++q) V[q] = ~(uint64_t)0;
    if (L % 64) V[nw - 1] = ((uint64_t)1 << (L % 64)) - 1;
    for (int t = 0; t < lb; ++t) {
        const uint64_t *M = pm + (size_t)b[t] * (size_t)nw;
        uint64_t carry = 0;
        for (int q = 0; q < nw; ++q) {
            const uint64_t u = V[q] & M[q];
            const uint64_t s1 = V[q] + u;
            const uint64_t c1 = s1 < u;
            const uint64_t s2 = s1 + carry;
            const uint64_t c2 = s2 < carry;
            V[q] = s2 | (V[q] & ~M[q]);
            carry = c1 | c2;
        }
    }
    int64_t ones = 0;
    for (int q = 0; q < nw; ++q) {
        uint64_t v = V[q];
        if (q == nw - 1 && (L % 64)) v &= ((uint64_t)1 << (L % 64)) - 1;
        ones += __builtin_popcountll(v);
    }
    return (int64_t)L - ones;
}

static void *blcs_worker(void *arg)
{
    blcs_job *jb = (blcs_job *)arg;
    const int nw = jb->nw;
    const int Lmax = jb->nu * (int)jb->w;
    uint64_t *pm = (uint64_t *)calloc((size_t)BLCS_SYMS * (size_t)nw, sizeof(uint64_t));
    int *a = (int *)malloc(sizeof(int) * (size_t)Lmax);
    int *b = (int *)malloc(sizeof(int) * (size_t)Lmax);
    for (int64_t r = jb->r0; r < jb->r1; ++r) {
        const int L = blow_window(jb->x + r * jb->step, jb->w, jb->nu, jb->mu, a);
        memset(pm, 0, sizeof(uint64_t) * (size_t)BLCS_SYMS * (size_t)nw);
        for (int p = 0; p < L; ++p) pm[(size_t)a[p] * (size_t)nw + (size_t)(p / 64)] |= (uint64_t)1 << (p % 64);
        const uint64_t wr = (uint64_t)r * 2654435761ull + 1ull;
        for (int64_t j = 0; j < jb->cols; ++j) {
            const int lb = blow_window(jb->y + j, jb->w, jb->nu, jb->mu, b);
            const int64_t v = blcs_llcs(pm, L, nw, b, lb);
            if (jb->out) {
                jb->out[r * jb->ld + j] = (int32_t)v;
            } else {
                jb->acc[0] += (uint64_t)v * (wr + (uint64_t)j * 40503ull);
                if (v < jb->nbins) jb->acc[1 + v] += 1;
            }
        }
    }
    free(pm);
    free(a);
    free(b);
    return NULL;
}

static int blcs_run(blcs_job base, int nthreads)
{
    if (base.rows <= 0 || base.cols <= 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > base.rows) nthreads = (int)base.rows;
    pthread_t th[256];
    blcs_job jobs[256];
    uint64_t *acc = NULL;
    if (!base.out) acc = (uint64_t *)calloc((size_t)nthreads * (size_t)(1 + base.nbins), sizeof(uint64_t));
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = base;
        /* interleaved row blocks: rows cost the same, so any split balances */
        jobs[t].r0 = base.rows * t / nthreads;
        jobs[t].r1 = base.rows * (t + 1) / nthreads;
        if (acc) jobs[t].acc = acc + (size_t)t * (size_t)(1 + base.nbins);
        if (pthread_create(&th[t], NULL, blcs_worker, &jobs[t]) != 0) {
            blcs_worker(&jobs[t]);
            th[t] = 0;
        }
    }
    for (int t = 0; t < nthreads; ++t)
        if (th[t]) pthread_join(th[t], NULL);
    if (acc) {
        for (int k = 0; k <= base.nbins; ++k) base.acc[k] = 0;
        for (int t = 0; t < nthreads; ++t)
            for (int k = 0; k <= base.nbins; ++k) base.acc[k] += acc[(size_t)t * (size_t)(1 + base.nbins) + k];
        free(acc);
    }
    return 0;
}

static int blcs_setup(blcs_job *b, const uint8_t *x, int64_t m, const uint8_t *y, int64_t n,
                      int64_t w, int32_t nu, int32_t mu, int64_t step)
{
    if (w < 1 || m < 0 || n < 0 || step < 1) return -1;
    if (!(nu == 1 && mu == 0) && !(nu >= 2 && mu >= 1 && mu < nu)) return -1;
    const int64_t L = (int64_t)nu * w;
    if (L > 64 * BLCS_MAXW) return -1;
    memset(b, 0, sizeof *b);
    b->x = x; b->y = y; b->m = m; b->n = n; b->w = w; b->step = step;
    b->nu = nu; b->mu = mu;
    b->nw = (int)((L + 63) / 64);
    b->rows = m > w ? (m - w + step - 1) / step : 0;
    b->cols = n > w ? n - w : 0;
    return 0;
}

/* Full plot (every step-th x-window): out[r*ld + j].  Returns 0, or -1 for
 * arguments outside what is built (blown-up windows up to 1024 characters). */
int oracle_blcs_plot(const uint8_t *x, int64_t m, const uint8_t *y, int64_t n, int64_t w,
                     int32_t nu, int32_t mu, int64_t step, int32_t *out, int64_t ld,
                     int nthreads)
{
    blcs_job b;
    if (blcs_setup(&b, x, m, y, n, w, nu, mu, step) != 0) return -1;
    if (b.cols > 0 && ld < b.cols) return -1;
    b.out = out;
    b.ld = ld;
    return blcs_run(b, nthreads);
}

/* Digest of the plot: result[0] = checksum, result[1 + v] = count of value v
 * (v < nbins).  result holds 1 + nbins words. */
int oracle_blcs_digest(const uint8_t *x, int64_t m, const uint8_t *y, int64_t n, int64_t w,
                       int32_t nu, int32_t mu, int64_t step, int32_t nbins, uint64_t *result,
                       int nthreads)
{
    blcs_job b;
    if (blcs_setup(&b, x, m, y, n, w, nu, mu, step) != 0 || nbins < 0) return -1;
    b.nbins = nbins;
    b.acc = result;
    for (int k = 0; k <= nbins; ++k) result[k] = 0;
    return blcs_run(b, nthreads);
}
