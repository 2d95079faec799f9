// api.cu -- the C ABI of libalnplot.so (declared in include/alnplot.h).
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "alnplot_internal.h"
#include "plan.h"

namespace ap {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_chunk_override{0};
static std::atomic<int32_t> g_groups_override{0};
static std::atomic<int64_t> g_band_override{0};
static std::atomic<int32_t> g_lane_override{0};

int64_t band_rows_override() { return g_band_override.load(); }

int64_t band_rows_for(int64_t automatic, int64_t spw, int64_t rows)
{
    int64_t br = automatic;
    const int64_t o = band_rows_override();
    if (o > 0) br = (o + spw - 1) / spw * spw;
    br = std::max<int64_t>(spw, br / spw * spw);
    return std::min(br, std::max<int64_t>(spw, (rows + spw - 1) / spw * spw));
}

ap_status fail(ap_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap_;
    va_start(ap_, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap_);
    va_end(ap_);
    g_last_error = buf;
    return s;
}

ap_status fail_cuda(cudaError_t e, const char *what)
{
    return fail(AP_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Scores -> blow-up {nu, mu, 0} and scale.  Normalised form: gap 0,
// 0 <= mismatch < match.  Every alignment score of {a, b, 0} is g times its
// score under {a/g, b/g, 0} with g = gcd(a, b), so the plot is g times the
// reduced scheme's plot: {m, 0, 0} is m x LCS, {4, 2, 0} is 2 x {2, 1, 0}.
// The reduced scheme is combed through the Section 2 blow-up (nu = 1: LCS).
ap_status score_mode(const ap_scores *sc, int *nu, int *mu, int *scale)
{
    *nu = 1;
    *mu = 0;
    *scale = 1;
    if (!sc) return AP_OK;
    if (sc->gap != 0 || sc->mismatch < 0 || sc->mismatch >= sc->match)
        return fail(AP_E_INVAL, "scores {%d,%d,%d} are not normalised (need gap 0, "
                    "0 <= mismatch < match)", sc->match, sc->mismatch, sc->gap);
    int a = sc->match, b = sc->mismatch;
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    const int g = a;                                     // gcd(match, mismatch)
    const int rn = sc->match / g, rm = sc->mismatch / g;
    if (rn > 8 || (int64_t)sc->match > 65535)
        return fail(AP_E_UNSUPPORTED, "scores {%d,%d,0}: built are schemes whose reduced form "
                    "{m/g, x/g, 0} (g = gcd(m, x)) has m/g <= 8", sc->match, sc->mismatch);
    *nu = rn;
    *mu = rm;
    *scale = g;
    return AP_OK;
}

int current_device()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return dev;
}

ap_status plan_plot(int64_t m, int64_t n, int32_t w, const ap_scores *scores, int groups,
                    int64_t chunk, Plan *pl, int64_t step, int lane_bits)
{
    if (step < 1) return fail(AP_E_INVAL, "step = %lld: must be >= 1", (long long)step);
    if (w < 1) return fail(AP_E_INVAL, "w = %d: the window length must be >= 1", w);
    if (m < 0 || n < 0) return fail(AP_E_INVAL, "negative sequence length");
    int nu = 1, mu = 0, scale = 1;
    ap_status s = score_mode(scores, &nu, &mu, &scale);
    if (s != AP_OK) return s;
    std::string why;
    if (!choose_variant(w, nu, mu, groups, step, pl, &why, lane_bits))
        return fail(AP_E_UNSUPPORTED, "%s", why.c_str());
    pl->scale = scale;
    pl->max_value = nu * scale * w;                      // = match * w
    // plot rows: x-windows 0, step, 2 step, ... below m - w
    const int64_t rows = m > w ? (m - w + step - 1) / step : 0;
    const int64_t cols = std::max<int64_t>(0, n - w);
    tile_plan(pl, rows, cols, chunk, current_device());
    return AP_OK;
}

ap_status check_output(const Plan &pl, const void *x, const void *y, const void *out,
                       int32_t out_elem_bytes, int64_t ld)
{
    if (out_elem_bytes != 1 && out_elem_bytes != 2)
        return fail(AP_E_INVAL, "out_elem_bytes = %d: must be 1 or 2", out_elem_bytes);
    if (out_elem_bytes == 1 && pl.max_value > 255)
        return fail(AP_E_INVAL, "uint8 output cannot hold values up to %d", pl.max_value);
    if (pl.max_value > 65535)
        return fail(AP_E_INVAL, "uint16 output cannot hold values up to %d", pl.max_value);
    if (pl.rows == 0 || pl.cols == 0) return AP_OK;   // empty plot
    if (!x || !y || !out) return fail(AP_E_INVAL, "null pointer");
    if (ld < pl.cols)
        return fail(AP_E_INVAL, "ld = %lld < cols = %lld", (long long)ld, (long long)pl.cols);
    return AP_OK;
}

namespace {

ap_status make_plan(int64_t m, int64_t n, int32_t w, const ap_scores *scores, Plan *pl,
                    int64_t step = 1)
{
    return plan_plot(m, n, w, scores, g_groups_override.load(), g_chunk_override.load(), pl, step,
                     g_lane_override.load());
}

constexpr int64_t kBandBudget = 1LL << 30;   // bytes of banded plot per dots pass

int64_t align256(int64_t v) { return (v + 255) & ~(int64_t)255; }

struct DotsLayout {
    int64_t band_rows = 0, band_ld = 0;
    int elem = 1;
    int64_t plot_off = 0, counts_off = 0, offsets_off = 0, running_off = 0, total = 0;
};

DotsLayout dots_layout(const Plan &pl)
{
    DotsLayout L;
    L.elem = pl.max_value > 255 ? 2 : 1;
    L.band_ld = (pl.cols + 31) / 32 * 32;   // whole 32-byte sectors per row block
    L.band_rows = band_rows_for(kBandBudget / std::max<int64_t>(1, L.band_ld * L.elem),
                                pl.strips_per_warp, pl.rows);
    L.plot_off = 0;
    L.counts_off = align256(L.band_rows * L.band_ld * L.elem);
    L.offsets_off = L.counts_off + align256(L.band_rows * 4);
    L.running_off = L.offsets_off + align256(L.band_rows * 8);
    L.total = L.running_off + 256;
    return L;
}

}  // namespace
}  // namespace ap

using namespace ap;

extern "C" {

const char *ap_version(void) { return "alnplot 0.1 (sm_103a seaweed strip comb)"; }

const char *ap_last_error(void) { return g_last_error.c_str(); }

const char *ap_status_string(ap_status s)
{
    switch (s) {
    case AP_OK: return "AP_OK";
    case AP_E_INVAL: return "AP_E_INVAL";
    case AP_E_UNSUPPORTED: return "AP_E_UNSUPPORTED";
    case AP_E_NOMEM: return "AP_E_NOMEM";
    case AP_E_OVERFLOW: return "AP_E_OVERFLOW";
    case AP_E_CUDA: return "AP_E_CUDA";
    case AP_E_TIMEOUT: return "AP_E_TIMEOUT";
    case AP_E_BUSY: return "AP_E_BUSY";
    case AP_E_CANCELLED: return "AP_E_CANCELLED";
    }
    return "AP_E_UNKNOWN";
}

ap_status ap_set_chunk(int64_t chunk)
{
    if (chunk < 0) return fail(AP_E_INVAL, "chunk = %lld: must be >= 0", (long long)chunk);
    g_chunk_override.store(chunk);
    return AP_OK;
}

ap_status ap_set_band_rows(int64_t rows)
{
    if (rows < 0) return fail(AP_E_INVAL, "band rows = %lld: must be >= 0", (long long)rows);
    g_band_override.store(rows);
    return AP_OK;
}

ap_status ap_set_lane_bits(int32_t bits)
{
    if (bits != 0 && bits != 8 && bits != 10 && bits != 16)
        return fail(AP_E_INVAL, "lane bits = %d: must be 0 (automatic), 8, 10 or 16", bits);
    g_lane_override.store(bits);
    return AP_OK;
}

ap_status ap_set_lanes_per_strip(int32_t groups)
{
    if (groups != 0 && groups != 1 && groups != 2 && groups != 4 && groups != 8)
        return fail(AP_E_INVAL, "lanes per strip = %d: must be 0 (automatic), 1, 2, 4 or 8", groups);
    g_groups_override.store(groups);
    return AP_OK;
}

ap_status ap_plot_shape(int64_t m, int64_t n, int32_t w, int64_t *rows, int64_t *cols)
{
    if (!rows || !cols) return fail(AP_E_INVAL, "ap_plot_shape: null output pointer");
    if (w < 1) return fail(AP_E_INVAL, "w = %d: the window length must be >= 1", w);
    if (m < 0 || n < 0) return fail(AP_E_INVAL, "negative sequence length");
    *rows = std::max<int64_t>(0, m - w);
    *cols = std::max<int64_t>(0, n - w);
    return AP_OK;
}

ap_status ap_plot_plan(int64_t m, int64_t n, int32_t w, const ap_scores *scores, ap_plan *out)
{
    if (!out) return fail(AP_E_INVAL, "ap_plot_plan: null plan pointer");
    Plan pl;
    ap_status s = make_plan(m, n, w, scores, &pl);
    if (s != AP_OK) return s;
    out->lane_bits = pl.v->lane_bits;
    out->strips_per_reg = pl.v->lane_bits == 8 ? 4 : (pl.v->lane_bits == 10 ? 3 : 2);
    out->rows_per_lane = pl.v->rows;
    out->lanes_per_strip = pl.v->groups;
    out->comb_rows = pl.comb_rows;
    out->chunk = (int32_t)pl.chunk;
    out->tiles = pl.ntiles;
    out->physical_cells = pl.ntiles ? physical_cells(pl) : 0;
    out->logical_cells = pl.rows * pl.cols * (int64_t)w;
    out->tables = plan_tables(pl);
    out->smem_per_block = (int32_t)pl.smem;
    return AP_OK;
}

ap_status ap_alignment_plot(const uint8_t *x, int64_t m, const uint8_t *y, int64_t n, int32_t w,
                            const ap_scores *scores, void *out, int32_t out_elem_bytes,
                            int64_t ld, void *stream)
{
    Plan pl;
    ap_status s = make_plan(m, n, w, scores, &pl);
    if (s != AP_OK) return s;
    s = check_output(pl, x, y, out, out_elem_bytes, ld);
    if (s != AP_OK || pl.rows == 0 || pl.cols == 0) return s;
    cudaError_t e = launch_comb(pl, x, m, y, n, out, out_elem_bytes, ld, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda(e, "strip comb launch");
    return AP_OK;
}

ap_status ap_alignment_plot_step(const uint8_t *x, int64_t m, const uint8_t *y, int64_t n,
                                 int32_t w, const ap_scores *scores, int64_t step, void *out,
                                 int32_t out_elem_bytes, int64_t ld, void *stream)
{
    Plan pl;
    ap_status s = make_plan(m, n, w, scores, &pl, step);
    if (s != AP_OK) return s;
    s = check_output(pl, x, y, out, out_elem_bytes, ld);
    if (s != AP_OK || pl.rows == 0 || pl.cols == 0) return s;
    cudaError_t e = launch_comb(pl, x, m, y, n, out, out_elem_bytes, ld, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda(e, "strip comb launch");
    return AP_OK;
}

ap_status ap_dots_workspace_size(int64_t m, int64_t n, int32_t w, const ap_scores *scores,
                                 int64_t *bytes)
{
    if (!bytes) return fail(AP_E_INVAL, "ap_dots_workspace_size: null output pointer");
    Plan pl;
    ap_status s = make_plan(m, n, w, scores, &pl);
    if (s != AP_OK) return s;
    *bytes = dots_layout(pl).total;
    return AP_OK;
}

ap_status ap_alignment_dots(const uint8_t *x, int64_t m, const uint8_t *y, int64_t n, int32_t w,
                            const ap_scores *scores, int32_t threshold, ap_dot *dots, int64_t cap,
                            int64_t *count, void *workspace, int64_t workspace_bytes, void *stream)
{
    if (!count) return fail(AP_E_INVAL, "ap_alignment_dots: null count pointer");
    if (cap < 0) return fail(AP_E_INVAL, "negative dot capacity");
    if (cap > 0 && !dots) return fail(AP_E_INVAL, "ap_alignment_dots: null dot buffer");
    Plan pl;
    ap_status s = make_plan(m, n, w, scores, &pl);
    if (s != AP_OK) return s;
    *count = 0;
    if (pl.rows == 0 || pl.cols == 0) return AP_OK;
    if (!x || !y) return fail(AP_E_INVAL, "ap_alignment_dots: null sequence pointer");
    const DotsLayout L = dots_layout(pl);
    if (!workspace || workspace_bytes < L.total)
        return fail(AP_E_NOMEM, "workspace of %lld bytes given, %lld needed",
                    (long long)workspace_bytes, (long long)L.total);
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    void *band = ws + L.plot_off;
    int32_t *counts = (int32_t *)(ws + L.counts_off);
    int64_t *offsets = (int64_t *)(ws + L.offsets_off);
    int64_t *running = (int64_t *)(ws + L.running_off);
    cudaError_t e = cudaMemsetAsync(running, 0, sizeof(int64_t), st);
    if (e != cudaSuccess) return fail_cuda(e, "workspace reset");
    for (int64_t r0 = 0; r0 < pl.rows; r0 += L.band_rows) {
        const int64_t br = std::min(L.band_rows, pl.rows - r0);
        Plan bp = pl;
        tile_plan(&bp, br, pl.cols, g_chunk_override.load(), current_device());
        e = launch_comb(bp, x + r0, m - r0, y, n, band, L.elem, L.band_ld, st);
        if (e != cudaSuccess) return fail_cuda(e, "strip comb launch");
        e = dots_pass(band, L.elem, br, pl.cols, L.band_ld, threshold, r0, dots, cap, counts,
                      offsets, running, st);
        if (e != cudaSuccess) return fail_cuda(e, "dot extraction");
    }
    int64_t total = 0;
    e = cudaMemcpyAsync(&total, running, sizeof total, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(e, "dot count read-back");
    *count = total;
    if (total > cap)
        return fail(AP_E_OVERFLOW, "%lld dots, buffer holds %lld", (long long)total,
                    (long long)cap);
    return AP_OK;
}

ap_status ap_plot_dots_workspace_size(int64_t rows, int64_t *bytes)
{
    if (!bytes || rows < 0) return fail(AP_E_INVAL, "ap_plot_dots_workspace_size: bad argument");
    *bytes = align256(rows * 4) + align256(rows * 8) + 256;
    return AP_OK;
}

ap_status ap_plot_dots(const void *plot, int32_t elem_bytes, int64_t rows, int64_t cols,
                       int64_t ld, int32_t threshold, ap_dot *dots, int64_t cap, int64_t *count,
                       void *workspace, int64_t workspace_bytes, void *stream)
{
    if (!count) return fail(AP_E_INVAL, "ap_plot_dots: null count pointer");
    if (elem_bytes != 1 && elem_bytes != 2) return fail(AP_E_INVAL, "elem_bytes must be 1 or 2");
    if (rows < 0 || cols < 0 || ld < cols) return fail(AP_E_INVAL, "bad plot shape");
    if (cap < 0 || (cap > 0 && !dots)) return fail(AP_E_INVAL, "bad dot buffer");
    *count = 0;
    if (rows == 0 || cols == 0) return AP_OK;
    if (!plot) return fail(AP_E_INVAL, "ap_plot_dots: null plot");
    int64_t need = 0;
    ap_plot_dots_workspace_size(rows, &need);
    if (!workspace || workspace_bytes < need)
        return fail(AP_E_NOMEM, "workspace of %lld bytes given, %lld needed",
                    (long long)workspace_bytes, (long long)need);
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    int32_t *counts = (int32_t *)ws;
    int64_t *offsets = (int64_t *)(ws + align256(rows * 4));
    int64_t *running = (int64_t *)(ws + align256(rows * 4) + align256(rows * 8));
    cudaError_t e = cudaMemsetAsync(running, 0, sizeof(int64_t), st);
    if (e == cudaSuccess)
        e = dots_pass(plot, elem_bytes, rows, cols, ld, threshold, 0, dots, cap, counts, offsets,
                      running, st);
    int64_t total = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, running, sizeof total, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(e, "plot dots");
    *count = total;
    if (total > cap)
        return fail(AP_E_OVERFLOW, "%lld dots, buffer holds %lld", (long long)total,
                    (long long)cap);
    return AP_OK;
}

ap_status ap_debug_bounds(uint32_t *flags)
{
    if (!flags) return fail(AP_E_INVAL, "ap_debug_bounds: null pointer");
    *flags = 0;
#ifdef AP_DEBUG_BOUNDS
    uint32_t *d = debug_flags();
    if (!d) return fail(AP_E_CUDA, "ap_debug_bounds: no violation word on this device");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(flags, d, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(uint32_t));
    if (e != cudaSuccess) return fail_cuda(e, "ap_debug_bounds");
    return AP_OK;
#else
    return fail(AP_E_UNSUPPORTED, "this build has no bounds checks (built without AP_DEBUG_BOUNDS)");
#endif
}

ap_status ap_plot_checksum(const void *plot, int32_t elem_bytes, int64_t rows, int64_t cols,
                           int64_t ld, int32_t nbins, uint64_t *result, void *stream)
{
    if (elem_bytes != 1 && elem_bytes != 2) return fail(AP_E_INVAL, "elem_bytes must be 1 or 2");
    if (rows < 0 || cols < 0 || ld < cols || nbins < 0 || nbins > 8192 || !result)
        return fail(AP_E_INVAL, "ap_plot_checksum: bad argument");
    if (rows > 0 && cols > 0 && !plot) return fail(AP_E_INVAL, "ap_plot_checksum: null plot");
    cudaError_t e = checksum_pass(plot, elem_bytes, rows, cols, ld, nbins, result,
                                  (cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda(e, "checksum");
    return AP_OK;
}

}  // extern "C"
