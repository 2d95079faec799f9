/*
 * alnplot.h -- C ABI of the GB300 alignment-plot library (libalnplot.so).
 *
 * An alignment plot (Krusche & Tiskin, "Computing alignment plots
 * efficiently", Section 2) holds, for two strings x (length m) and y
 * (length n) and a window length w, one value per pair of w-windows:
 *
 *     P[i][j] = best alignment score of x[i .. i+w) and y[j .. j+w)
 *     for 0 <= i < m - w and 0 <= j < n - w
 *
 * This is the paper's index range {1..m-w} x {1..n-w}, written 0-based.
 * The library computes every value with the seaweed strip sweep of
 * Theorem 3.1 and Section 3, at O(w) per column per strip.  It does not
 * run the O(w^2) dynamic programme once per window pair.
 *
 * Conventions shared by every call:
 *   - Sequences are arrays of bytes; two characters match when their bytes
 *     are equal, so all 256 byte values are ordinary characters.
 *   - Pointers named "device" are CUDA device pointers owned by the caller;
 *     "host" pointers are ordinary host memory.  The library never frees
 *     caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream are stream-ordered: they enqueue
 *     work and return without waiting, unless stated otherwise.
 *   - Every call returns an ap_status and never aborts.  On failure,
 *     ap_last_error() gives a message for the calling thread.
 */
#ifndef ALNPLOT_H
#define ALNPLOT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ap_status {
    AP_OK = 0,
    AP_E_INVAL = 1,        /* bad argument (null pointer, w < 1, ld too small, ...) */
    AP_E_UNSUPPORTED = 2,  /* valid request that this build does not handle */
    AP_E_NOMEM = 3,        /* workspace or budget too small */
    AP_E_OVERFLOW = 4,     /* more dots than the caller's buffer holds */
    AP_E_CUDA = 5,         /* a CUDA runtime call failed */
    AP_E_TIMEOUT = 6,      /* a wait reached its time limit */
    AP_E_BUSY = 7,         /* no free slot right now */
    AP_E_CANCELLED = 8     /* the job was cancelled */
} ap_status;

/*
 * Alignment scores, normalised so that gap = 0 and 0 <= mismatch < match
 * (Section 2: LCS is the scheme with match 1 and mismatch and gap 0).
 * Supported:
 *   {1, 0, 0}  LCS: P = LLCS of the two windows, 0 <= P <= w.
 *   {2, 1, 0}  Section 2's scheme (match 1, mismatch 0, gap -1/2), shifted
 *              so gaps score 0 and doubled: P = T = S + w, w <= T <= 2w,
 *              where S is the (1, 0, -1/2) score.  Computed as the LCS of the
 *              '$'-interleaved windows (Section 2), with Definition 3.2's
 *              (w, 2) restriction.
 *   {m, x, 0}  other small rational scores (Section 2 reduces them to LCS by
 *              enlarging the input strings by a constant factor).  With
 *              g = gcd(m, x), every score under {m, x, 0} is g times its score
 *              under {m/g, x/g, 0}, so the plot is g times the reduced
 *              scheme's plot; the reduced scheme with m/g >= 2 is combed as
 *              the LCS of blown-up windows, every character becoming x/g
 *              copies of '$' followed by m/g - x/g copies of itself.  Built:
 *              m/g <= 8 -- so {m, 0, 0} (m times the LCS, g = m) for any m,
 *              {2k, k, 0}, {3k, k, 0}, {4k, 3k, 0}, {5k, 2k, 0}, {8k, 7k, 0}
 *              and so on.  x w <= P <= m w.  Windows: as LCS for m/g = 1, as
 *              {2,1,0} for m/g = 2, up to 256 for m/g = 3, 4, 192 for 5, 160
 *              for 6, 128 for 7 and 8.
 * A scheme (a, b, c) with c < 0 maps to {a - 2c, b - 2c, 0} after scaling to
 * integers (and the plot value to S - 2wc).  Other normalised pairs
 * (m/g >= 9) return AP_E_UNSUPPORTED; so do plots whose largest value m w
 * exceeds 65535.
 */
typedef struct ap_scores {
    int32_t match;
    int32_t mismatch;
    int32_t gap;
} ap_scores;

/* One dot of a thresholded plot (Section 1: a dot for each window pair whose
 * score passes the threshold).  value = P[i][j]. */
typedef struct ap_dot {
    uint32_t i;
    uint32_t j;
    uint16_t value;
    uint16_t pad;
} ap_dot;

/* How a plot call is carried out (kernel variant and tiling); informational. */
typedef struct ap_plan {
    int32_t lane_bits;        /* 8, 10 or 16: bits per seaweed key lane */
    int32_t strips_per_reg;   /* strips held side by side in one 32-bit register */
    int32_t rows_per_lane;    /* comb rows each thread holds (compile-time) */
    int32_t lanes_per_strip;  /* threads that split one strip's rows */
    int32_t comb_rows;        /* physical comb height: w (LCS) or 2w (score) */
    int32_t chunk;            /* plot columns per tile */
    int64_t tiles;            /* strip groups x column chunks */
    int64_t physical_cells;   /* comb cell updates, warm-up and padding included */
    int64_t logical_cells;    /* (m - w)(n - w) w: window pairs times window length */
    int32_t tables;           /* match tables, taken by warps whose x letters have at
                                 most four values: 0 none; 1 one thread per strip
                                 group; 2, 3 shared by the threads of a strip group,
                                 their row split rounded down (2) or up (3) */
    int32_t smem_per_block;   /* dynamic shared memory of a block of the comb launch
                                 (bytes): exit rings, output stages and tables */
} ap_plan;

/* Library version string. */
const char *ap_version(void);

/* Message for the calling thread's last failed call ("" if none). */
const char *ap_last_error(void);

/* Name of a status code. */
const char *ap_status_string(ap_status s);

/*
 * Plot shape (Section 2): rows = max(0, m - w), cols = max(0, n - w).
 * rows, cols: host pointers, written on success.  AP_E_INVAL if w < 1,
 * m < 0, n < 0 or a pointer is null.
 */
ap_status ap_plot_shape(int64_t m, int64_t n, int32_t w, int64_t *rows,
                        int64_t *cols);

/*
 * The plan ap_alignment_plot would use for these sizes (host only, no GPU
 * work).  `plan`: host pointer, written on success.
 */
ap_status ap_plot_plan(int64_t m, int64_t n, int32_t w,
                       const ap_scores *scores, ap_plan *plan);

/*
 * Tuning: force the number of plot columns per tile (rounded up to a
 * multiple of 32) for later plot and dots calls in this process; 0 restores
 * the automatic choice.  Results do not depend on it (a tile starting at
 * column c0 combs w - 1 warm-up columns, which is exact; Theorem 3.1 applied
 * to the substring of y from c0).  Process-wide; AP_E_INVAL if chunk < 0.
 */
ap_status ap_set_chunk(int64_t chunk);

/*
 * Tuning and testing: force the band height of the banded calls, which comb
 * a plot a band of rows at a time into device memory (ap_alignment_dots,
 * ap_alignment_plot_host, and the jobs that ap_server_submit plans), to
 * `rows` plot rows rounded up to whole strip groups; 0 restores the
 * automatic choice (about 1 GB of plot per band).  Each band combs its rows
 * exactly as one call would (strips are independent, Theorem 3.1), so
 * results do not depend on it; small bands make small plots take the
 * many-band path.  A workspace size queried under one setting serves calls
 * under the same setting.  Process-wide; AP_E_INVAL if rows < 0.
 */
ap_status ap_set_band_rows(int64_t rows);

/*
 * Tuning: ask for a lane format of the LCS comb -- 8 (four strips per
 * register; windows up to 254), 10 (three strips; 121..480) or 16 bits (two
 * strips; any window up to 512) -- for later plot and dots calls in this
 * process; 0 restores the automatic choice (8 bits up to w = 240, then 16).  Honoured where the format
 * covers the window, else the automatic choice is used.  Results do not
 * depend on it.  Process-wide; AP_E_INVAL unless bits is 0, 8, 10 or 16.
 */
ap_status ap_set_lane_bits(int32_t bits);

/*
 * Tuning: ask for `groups` threads per group of strips (the comb rows of one
 * strip are split over them; 0 restores the automatic choice).  Honoured
 * when a compiled variant exists for the window length, else the automatic
 * choice is used.  Results do not depend on it.  Process-wide; AP_E_INVAL
 * unless groups is 0, 1, 2, 4 or 8.
 */
ap_status ap_set_lanes_per_strip(int32_t groups);

/*
 * Full alignment plot (Section 2 definition; Theorem 3.1 / Section 3 method).
 *
 *   x       device, m bytes          y       device, n bytes
 *   w       window length, >= 1
 *   scores  host, {1,0,0}, {2,1,0} or another built {m, x, 0} (see ap_scores)
 *   out     device, rows x ld elements, row-major; out[i*ld + j] = P[i][j]
 *   out_elem_bytes  1 (uint8) or 2 (uint16)
 *   ld      elements between consecutive rows, ld >= cols
 *   stream  cudaStream_t as void*
 *
 * Errors: AP_E_INVAL for null pointers, w < 1, ld < cols, an element size
 * other than 1 or 2, or uint8 output when the largest possible value
 * (match * w) exceeds 255; AP_E_UNSUPPORTED for score schemes not built
 * or w beyond the largest compiled comb height (LCS w <= 512, {2,1,0} and
 * m/g = 3, 4: w <= 256; m/g = 5: 192, 6: 160, 7 and 8: 128);
 * AP_E_CUDA if a launch fails.  If m <= w or n <= w the plot is empty:
 * nothing is written and AP_OK is returned.  Stream-ordered; allocates no
 * device memory.
 */
ap_status ap_alignment_plot(const uint8_t *x, int64_t m, const uint8_t *y,
                            int64_t n, int32_t w, const ap_scores *scores,
                            void *out, int32_t out_elem_bytes, int64_t ld,
                            void *stream);

/*
 * Alignment plot with a vertical step (Section 3: a step size h keeps only
 * the x-windows whose start is a multiple of h; Section 4 uses h = 5): plot
 * row r holds the x-window starting at
 * r * step, for 0 <= r < ceil((m - w) / step), against every y-window:
 *     out[r*ld + j] = P[r * step][j]
 * step = 1 is ap_alignment_plot.  With step > 1 this build covers LCS for
 * w <= 512 and {2,1,0} for w <= 256 (AP_E_UNSUPPORTED otherwise, and for
 * other score schemes).  Other arguments and errors as in
 * ap_alignment_plot; AP_E_INVAL for step < 1.
 */
ap_status ap_alignment_plot_step(const uint8_t *x, int64_t m, const uint8_t *y,
                                 int64_t n, int32_t w, const ap_scores *scores,
                                 int64_t step, void *out, int32_t out_elem_bytes,
                                 int64_t ld, void *stream);

/*
 * Plot into HOST memory (and optionally its dots), end to end: x and y are
 * HOST arrays (pinned memory copies fastest), `out` is a HOST buffer of
 * (m - w) x ld elements, row-major, as in ap_alignment_plot.  The plot is
 * combed band by band into two device band buffers, and each band's copy
 * back to the host overlaps the comb of the next.  So the plot may be larger
 * than device memory, and the copy hides behind the compute.  With ld equal
 * to cols rounded up to a multiple of 32 (the device band's row stride),
 * each band is one contiguous copy.
 *
 *   threshold, dots, dots_cap, dots_count: if dots_count is non-null, the
 *     dots with P >= threshold are also returned (HOST `dots`, row-major as in
 *     ap_alignment_dots; AP_E_OVERFLOW beyond dots_cap, full count reported);
 *     pass dots_count = NULL for the plot alone.
 *   workspace: DEVICE, >= ap_plot_host_workspace_size(...) bytes (the
 *     sequences, two band buffers, row counts, and dots_cap dots).
 *
 * Synchronous: returns when the plot and dots are in host memory.  Errors as
 * in ap_alignment_plot, plus AP_E_NOMEM for a short workspace.
 */
ap_status ap_plot_host_workspace_size(int64_t m, int64_t n, int32_t w,
                                      const ap_scores *scores,
                                      int32_t out_elem_bytes, int64_t dots_cap,
                                      int64_t *bytes);
ap_status ap_alignment_plot_host(const uint8_t *x, int64_t m, const uint8_t *y,
                                 int64_t n, int32_t w, const ap_scores *scores,
                                 void *out, int32_t out_elem_bytes, int64_t ld,
                                 int32_t threshold, ap_dot *dots,
                                 int64_t dots_cap, int64_t *dots_count,
                                 void *workspace, int64_t workspace_bytes,
                                 void *stream);

/*
 * Bytes of device workspace ap_alignment_dots needs for these sizes.
 * bytes: host pointer, written on success.
 */
ap_status ap_dots_workspace_size(int64_t m, int64_t n, int32_t w,
                                 const ap_scores *scores, int64_t *bytes);

/*
 * Thresholded plot: every window pair with P[i][j] >= threshold, as ap_dot
 * records in row-major order (i, then j) -- Section 1's dot plot, with the
 * inclusive threshold on the alignment score.
 *
 *   dots       device, room for `cap` records (may be null when cap = 0)
 *   count      host; receives the total number of qualifying pairs, also
 *              when it exceeds cap
 *   workspace  device, >= ap_dots_workspace_size(...) bytes, caller-owned
 *
 * The plot is computed band by band into the workspace, so no full-size
 * plot is ever allocated.  Returns AP_E_OVERFLOW (after writing the first
 * `cap` dots and the full count) when count > cap.  Synchronises `stream`
 * before returning, because the status depends on the count.
 */
ap_status ap_alignment_dots(const uint8_t *x, int64_t m, const uint8_t *y,
                            int64_t n, int32_t w, const ap_scores *scores,
                            int32_t threshold, ap_dot *dots, int64_t cap,
                            int64_t *count, void *workspace,
                            int64_t workspace_bytes, void *stream);

/*
 * Dots of an existing plot in device memory (same order and overflow rule
 * as ap_alignment_dots).  plot: device, rows x ld elements of elem_bytes
 * (1 or 2).  Workspace: device, >= ap_plot_dots_workspace_size(rows) bytes.
 * Synchronises `stream` before returning.
 */
ap_status ap_plot_dots_workspace_size(int64_t rows, int64_t *bytes);
ap_status ap_plot_dots(const void *plot, int32_t elem_bytes, int64_t rows,
                       int64_t cols, int64_t ld, int32_t threshold,
                       ap_dot *dots, int64_t cap, int64_t *count,
                       void *workspace, int64_t workspace_bytes, void *stream);

/* Largest plot height that ap_plot_dots_noalloc accepts. */
#define AP_PLOT_DOTS_NOALLOC_MAX_ROWS 262144

/*
 * ap_plot_dots with no workspace argument and no device allocation.  The
 * paper has no counterpart; this is an interface convenience.
 *
 * It is for callers that cannot call cudaMalloc, for instance a plug-in
 * running inside a host program that owns the GPU's memory budget, or a
 * service that must not allocate once it has started.  The scratch that
 * ap_plot_dots takes from the caller (12 bytes per plot row: a row count, a
 * row offset, plus a running total) lives in one fixed static device array
 * in the library.  It is sized for AP_PLOT_DOTS_NOALLOC_MAX_ROWS rows (about
 * 3 MiB), and every GPU that loads the library holds it until the process
 * exits.  Taller plots are rejected with AP_E_NOMEM.
 *
 * Every call looks up the array's address on the device current at the
 * call.  The first call in a process on a device also loads the library's
 * module holding the array there, which takes those ~3 MiB of device memory
 * at that moment (and can fail with AP_E_CUDA if the device is full).  So
 * make one call per device at start-up, before any stream capture and
 * before the host program takes the rest of the memory: a call with
 * rows = 0 (plot may then be null) does only that.  All calls share the
 * one array, which keeps the last call's contents.  Each call clears what
 * must start at zero, but calls whose GPU work overlaps (different streams
 * or host threads) race on the array, so the caller must order them.
 *
 * Arguments, results, dot order and the overflow rule are those of
 * ap_plot_dots.  Synchronises `stream` before returning.
 */
ap_status ap_plot_dots_noalloc(const void *plot, int32_t elem_bytes,
                               int64_t rows, int64_t cols, int64_t ld,
                               int32_t threshold, ap_dot *dots, int64_t cap,
                               int64_t *count, void *stream);

/*
 * Checksum and value histogram of a plot in device memory, for checking
 * large plots without copying them:
 *   sum over cells of P[i][j] * (i*2654435761 + j*40503 + 1)  mod 2^64
 * and hist[v] = number of cells with value v, for v < nbins (larger values
 * are not counted).  result: device, 1 + nbins uint64 words (checksum first),
 * overwritten.  Stream-ordered.
 */
ap_status ap_plot_checksum(const void *plot, int32_t elem_bytes, int64_t rows,
                           int64_t cols, int64_t ld, int32_t nbins,
                           uint64_t *result, void *stream);

/*
 * Debug builds only (the library compiled with AP_DEBUG_BOUNDS, as
 * paper_0909_2000_gb300/build.py builds libalnplot_debug.so): every plot
 * store, sequence read, exit-ring slot and match-table read of the comb
 * kernels is checked against its buffer, and a failed check sets a bit in a
 * per-device word and skips the access instead of touching memory outside
 * the buffer.  This call waits for the device, writes that word to *flags
 * (host; 0 = no violation; bits 1 plot store, 2 y read, 4 x read, 8 ring
 * slot, 16 table read) and clears it.  Other builds return
 * AP_E_UNSUPPORTED with *flags = 0.  Not in the paper: a testing aid.
 */
ap_status ap_debug_bounds(uint32_t *flags);

/*
 * Integer issue rate of the current device, the denominator of the comb
 * kernel's roofline (not in the paper: a measurement aid).  A kernel of
 * eight independent accumulators per thread, 64 warps an SM, updates each
 * accumulator `iters` times from two others with one instruction:
 *   kind 0  three-input logic (lop3)      -- the ALU pipe alone
 *   kind 1  32-bit multiply-add (mad.lo)  -- the FMA pipe alone
 *   kind 2  the two alternately           -- both pipes
 * *lane_ops_per_s (host) receives the 32-bit lane operations per second of
 * one timed launch (after one warm-up launch).  Synchronous; allocates
 * nothing (its 16 KB result sink is a file-scope device array).
 * AP_E_INVAL for kind outside 0..2, iters < 1 or a null pointer.
 */
ap_status ap_int_issue_probe(int32_t kind, int64_t iters, double *lane_ops_per_s);

/* ------------------------------------------------------------------------
 * Batched plots: many independent (x, y, w) jobs, run as one CUDA graph of
 * persistent strip-comb kernels.  Not in the paper: it is the many-pairs
 * form of the same computation (every job's plot is exactly the plot
 * ap_alignment_plot would write).
 * ---------------------------------------------------------------------- */

/* One plot job.  All pointers are device pointers owned by the caller; they
 * must stay valid (and keep their contents' meaning) for as long as the
 * batch is run.  Fields are as in ap_alignment_plot. */
typedef struct ap_job {
    const uint8_t *x;
    int64_t m;
    const uint8_t *y;
    int64_t n;
    int32_t w;
    ap_scores scores;
    void *out;
    int32_t out_elem_bytes;
    int64_t ld;
} ap_job;

/* Batch options; zero-initialised means automatic. */
typedef struct ap_batch_options {
    int32_t autotune;         /* 1: time candidate schedules per window class at
                                 create time (runs the jobs, writing their outputs) */
    int32_t chunk;            /* > 0: plot columns per tile for every job */
    int32_t lanes_per_strip;  /* > 0: threads per strip group, when compiled */
} ap_batch_options;

/* What ap_batch_create chose (informational). */
typedef struct ap_batch_info {
    int32_t groups;           /* persistent kernels (one per comb variant) */
    int32_t jobs;             /* jobs with a non-empty plot */
    int64_t tiles;            /* tiles over all groups */
    int64_t logical_cells;    /* sum over jobs of (m-w)(n-w)w */
    int64_t physical_cells;   /* comb cell updates incl. warm-up and padding */
    double tune_ms;           /* time spent autotuning */
} ap_batch_info;

typedef struct ap_batch ap_batch;

/*
 * Plans a batch: validates every job (the rules of ap_alignment_plot), groups
 * the jobs by comb variant, orders each group's tiles most expensive first,
 * optionally autotunes the chunk length and threads per strip of each window
 * class, and captures one CUDA graph.  The graph resets a work-queue counter
 * per group and runs one persistent kernel per group, all groups side by
 * side.  Uses the current device.  The batch owns a little device memory (job
 * parameters, tile lists, counters), freed by ap_batch_destroy.  Errors: those
 * of ap_alignment_plot for the first bad job (the message names it),
 * AP_E_INVAL for njobs < 0 or null pointers, AP_E_CUDA.
 */
ap_status ap_batch_create(const ap_job *jobs, int32_t njobs,
                          const ap_batch_options *options, ap_batch **batch);

/* Runs the batch's graph on `stream` (stream-ordered, asynchronous). */
ap_status ap_batch_run(ap_batch *batch, void *stream);

/* Fills `info` (host) with the batch's plan. */
ap_status ap_batch_get_info(const ap_batch *batch, ap_batch_info *info);

/* Frees the batch (after its last run has finished).  Null is a no-op. */
ap_status ap_batch_destroy(ap_batch *batch);

/* ------------------------------------------------------------------------
 * Serving: dot-plot requests from host memory, admitted by device memory
 * and free slots, with their work overlapping on the GPU (continuous
 * batching).  Not in the paper: it serves the same computation
 * (ap_alignment_dots) to many clients.
 * ---------------------------------------------------------------------- */

/* One request.  x and y are HOST pointers; ap_server_submit copies them, so
 * the caller may free them as soon as it returns.  The result is every
 * window pair with P[i][j] >= threshold (row-major ap_dot records, as in
 * ap_alignment_dots), at most max_dots of them; a larger count ends the job
 * with AP_E_OVERFLOW, still reporting the full count and the first
 * max_dots dots. */
typedef struct ap_request {
    const uint8_t *x;
    int64_t m;
    const uint8_t *y;
    int64_t n;
    int32_t w;
    ap_scores scores;
    int32_t threshold;
    int64_t max_dots;
} ap_request;

/* Server counters (ap_server_get_stats).  Latency is from submit to the
 * moment the result is ready, over completed jobs. */
typedef struct ap_server_stats {
    int64_t submitted;
    int64_t completed;        /* finished with AP_OK or AP_E_OVERFLOW */
    int64_t failed;           /* finished with another error or cancelled */
    int64_t queued;           /* waiting for a slot or memory */
    int64_t running;          /* admitted, not finished */
    int64_t logical_cells;    /* sum of (m-w)(n-w)w over completed jobs */
    int64_t peak_device_bytes;/* largest device memory held by admitted jobs */
    double latency_p50_ms;
    double latency_p99_ms;
    double latency_max_ms;
} ap_server_stats;

typedef struct ap_server ap_server;

/*
 * Starts a server on the current device with `max_slots` concurrent jobs
 * (1..64) and `mem_budget` bytes of device memory for admitted jobs (their
 * sequences, plot band, row counts and dots).  A scheduler thread admits
 * queued requests in arrival order when a slot is free and the job's memory
 * fits the budget; each admitted job runs on its own stream, so the work of
 * different jobs overlaps on the device.  Errors: AP_E_INVAL, AP_E_CUDA.
 */
ap_status ap_server_create(int64_t mem_budget, int32_t max_slots, ap_server **server);

/* Queues a request and returns its ticket (> 0).  Validation errors of
 * ap_alignment_dots are returned here; a job that can never fit the memory
 * budget returns AP_E_NOMEM. */
ap_status ap_server_submit(ap_server *server, const ap_request *request, uint64_t *ticket);

/* State of a ticket: AP_E_BUSY while queued or running, else the job's final
 * status (AP_OK, AP_E_OVERFLOW, AP_E_CANCELLED, AP_E_CUDA ...).  AP_E_INVAL for
 * an unknown (or already fetched) ticket. */
ap_status ap_server_poll(ap_server *server, uint64_t ticket, ap_status *state);

/* Blocks until the job has finished or `timeout_ms` has passed (< 0: no
 * limit).  Returns the job's final status, or AP_E_TIMEOUT. */
ap_status ap_server_wait(ap_server *server, uint64_t ticket, int32_t timeout_ms);

/* Copies a finished job's result into `dots` (HOST, room for `cap` records)
 * and its full count into *count, then forgets the ticket.  Returns the job's
 * final status; AP_E_BUSY if it has not finished (nothing is consumed). */
ap_status ap_server_fetch(ap_server *server, uint64_t ticket, ap_dot *dots, int64_t cap,
                          int64_t *count);

/* Cancels a queued job (it never runs) or a running one (its result is
 * dropped when its GPU work ends).  Its state becomes AP_E_CANCELLED. */
ap_status ap_server_cancel(ap_server *server, uint64_t ticket);

ap_status ap_server_get_stats(ap_server *server, ap_server_stats *stats);

/* Stops the scheduler after the jobs already admitted have finished, drops
 * queued ones, and frees everything.  Null is a no-op. */
ap_status ap_server_destroy(ap_server *server);

#ifdef __cplusplus
}
#endif

#endif /* ALNPLOT_H */
