// host_plot.cu -- a plot (and its dots) computed into host memory, with the
// device-to-host copy of each plot band overlapping the comb of the next.
//
// The plot rows are combed band by band into two device band buffers taken
// from the caller's workspace.  Band b is combed on the caller's stream, its
// dots (if asked for) are appended on the same stream, and a second stream
// copies the band to the host plot while band b + 1 is combed into the other
// buffer.  This keeps the GPU combing while the plot streams out, and it lets
// the plot be larger than device memory.  On the 100k DNA plot (10 GB) a
// call takes 68.4 ms at best, the device-to-host link's pace (about 150 GB/s
// while the comb runs).  Measured slower or no better:
// * combing alternate bands on two streams (the concurrent band kernels
//   interfere);
// * the dots on the copy stream (they wait for SMs held by the next band's
//   comb, and the band copy waits behind them);
// * each band's copy split over two copy streams (68.8 ms), and a quarter
//   and a half band first so that the copies start sooner (68.3 ms);
// * the comb writing the plot straight into mapped pinned host memory, no
//   bands and no copies (72.9 ms).
#include <algorithm>
#include <mutex>
#include <vector>

#include "alnplot_internal.h"
#include "plan.h"

namespace ap {
namespace {

constexpr int64_t kHostBand = 1LL << 30;     // bytes per device band buffer (several waves of tiles)

int64_t align256(int64_t v) { return (v + 255) & ~(int64_t)255; }

// The copy stream and band events of ap_alignment_plot_host, created once per
// calling thread and device and reused by every later call (they live until
// the process exits).
struct HostPlotStreams {
    int device = -1;
    cudaStream_t copy = nullptr;
    cudaEvent_t combed[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
};

cudaError_t host_plot_streams(HostPlotStreams **out)
{
    static thread_local std::vector<HostPlotStreams> cache;
    const int dev = current_device();
    for (auto &r : cache)
        if (r.device == dev) {
            *out = &r;
            return cudaSuccess;
        }
    HostPlotStreams r;
    r.device = dev;
    cudaError_t e = cudaStreamCreateWithFlags(&r.copy, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&r.combed[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.copied[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        if (r.copy) cudaStreamDestroy(r.copy);
        for (int k = 0; k < 2; ++k) {
            if (r.combed[k]) cudaEventDestroy(r.combed[k]);
            if (r.copied[k]) cudaEventDestroy(r.copied[k]);
        }
        return e;
    }
    cache.reserve(8);
    cache.push_back(r);
    *out = &cache.back();
    return cudaSuccess;
}

struct HostLayout {
    int64_t band_rows = 0, band_ld = 0, x_off = 0, y_off = 0, buf_off[2] = {0, 0},
            counts_off[2] = {0, 0}, offsets_off[2] = {0, 0}, running_off = 0, dots_off = 0,
            total = 0;
};

HostLayout host_layout(const Plan &pl, int64_t m, int64_t n, int elem, int64_t dots_cap)
{
    HostLayout L;
    L.band_ld = (pl.cols + 31) / 32 * 32;
    L.band_rows = band_rows_for(kHostBand / std::max<int64_t>(1, L.band_ld * elem),
                                pl.strips_per_warp, pl.rows);
    int64_t o = 0;
    L.x_off = o;
    o += align256(m);
    L.y_off = o;
    o += align256(n);
    for (int k = 0; k < 2; ++k) {
        L.buf_off[k] = o;
        o += align256(L.band_rows * L.band_ld * elem);
    }
    for (int k = 0; k < 2; ++k) {
        L.counts_off[k] = o;
        o += align256(L.band_rows * 4);
        L.offsets_off[k] = o;
        o += align256(L.band_rows * 8);
    }
    L.running_off = o;
    o += 256;
    L.dots_off = o;
    o += align256(std::max<int64_t>(0, dots_cap) * (int64_t)sizeof(ap_dot));
    L.total = o;
    return L;
}

}  // namespace
}  // namespace ap

using namespace ap;

extern "C" {

ap_status ap_plot_host_workspace_size(int64_t m, int64_t n, int32_t w, const ap_scores *scores,
                                      int32_t out_elem_bytes, int64_t dots_cap, int64_t *bytes)
{
    if (!bytes || (out_elem_bytes != 1 && out_elem_bytes != 2) || dots_cap < 0)
        return fail(AP_E_INVAL, "ap_plot_host_workspace_size: bad argument");
    Plan pl;
    ap_status s = plan_plot(m, n, w, scores, 0, 0, &pl);
    if (s != AP_OK) return s;
    *bytes = host_layout(pl, m, n, out_elem_bytes, dots_cap).total;
    return AP_OK;
}

ap_status ap_alignment_plot_host(const uint8_t *x, int64_t m, const uint8_t *y, int64_t n,
                                 int32_t w, const ap_scores *scores, void *out,
                                 int32_t out_elem_bytes, int64_t ld, int32_t threshold,
                                 ap_dot *dots, int64_t dots_cap, int64_t *dots_count,
                                 void *workspace, int64_t workspace_bytes, void *stream)
{
    Plan pl;
    ap_status s = plan_plot(m, n, w, scores, 0, 0, &pl);
    if (s != AP_OK) return s;
    s = check_output(pl, x, y, out, out_elem_bytes, ld);
    if (s != AP_OK) return s;
    if (dots_cap < 0 || (dots_cap > 0 && !dots) || (dots_cap > 0 && !dots_count))
        return fail(AP_E_INVAL, "ap_alignment_plot_host: bad dot buffer");
    if (dots_count) *dots_count = 0;
    if (pl.rows == 0 || pl.cols == 0) return AP_OK;
    const HostLayout L = host_layout(pl, m, n, out_elem_bytes, dots_cap);
    if (!workspace || workspace_bytes < L.total)
        return fail(AP_E_NOMEM, "workspace of %lld bytes given, %lld needed",
                    (long long)workspace_bytes, (long long)L.total);
    const bool want_dots = dots_count != nullptr;
    NvtxRange range("alnplot: plot into host memory");
    char *ws = (char *)workspace;
    uint8_t *dx = (uint8_t *)(ws + L.x_off), *dy = (uint8_t *)(ws + L.y_off);
    int64_t *running = (int64_t *)(ws + L.running_off);
    ap_dot *ddots = (ap_dot *)(ws + L.dots_off);
    cudaStream_t st = (cudaStream_t)stream;

    // the caller's stream combs every band; the copy stream moves them out
    cudaStream_t cs[2] = {st, st};
    HostPlotStreams *hs = nullptr;
    cudaError_t e = host_plot_streams(&hs);
    if (e != cudaSuccess) return fail_cuda(e, "ap_alignment_plot_host: copy stream");
    cudaStream_t copy = hs->copy;
    cudaEvent_t *combed = hs->combed, *copied = hs->copied;
    // the previous call on this thread has finished with the copy stream
    // (every call synchronises it before returning)
    if (e == cudaSuccess) e = cudaMemcpyAsync(dx, x, (size_t)m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy, y, (size_t)n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && want_dots) e = cudaMemsetAsync(running, 0, sizeof(int64_t), st);
    // Band sizes: full bands, then halving ones (down to a quarter band) over
    // the last two bands' worth of rows, so that the copy of the final band,
    // which nothing overlaps, is short.  Whole strip groups per band.
    const int64_t spw = pl.strips_per_warp;
    const int64_t quarter = std::max<int64_t>(spw, L.band_rows / 4 / spw * spw);
    auto next_band = [&](int64_t left) -> int64_t {
        int64_t half = (left + 1) / 2;
        half = (half + spw - 1) / spw * spw;
        return std::min(left, std::min(L.band_rows, std::max(quarter, half)));
    };
    int band = 0;
    int64_t br = 0;
    for (int64_t r0 = 0; r0 < pl.rows && e == cudaSuccess; r0 += br, ++band) {
        const int k = band & 1;
        cudaStream_t sk = cs[k];
        br = next_band(pl.rows - r0);
        void *buf = ws + L.buf_off[k];
        if (band >= 2) e = cudaStreamWaitEvent(sk, copied[k], 0);   // buffer k is free again
        Plan bp = pl;
        tile_plan(&bp, br, pl.cols, 0, current_device());
        if (e == cudaSuccess)
            e = launch_comb(bp, dx + r0, m - r0, dy, n, buf, out_elem_bytes, L.band_ld, sk);
        // the copy may start as soon as the band is combed: the dot kernels
        // that follow on the compute stream only read the band
        if (e == cudaSuccess) e = cudaEventRecord(combed[k], sk);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(copy, combed[k], 0);
        if (e == cudaSuccess && want_dots)      // dots in band order on the compute stream
            e = dots_pass(buf, out_elem_bytes, br, pl.cols, L.band_ld, threshold, r0, ddots,
                          dots_cap, (int32_t *)(ws + L.counts_off[k]),
                          (int64_t *)(ws + L.offsets_off[k]), running, sk);
        char *dst = (char *)out + r0 * ld * out_elem_bytes;
        if (e == cudaSuccess && ld == L.band_ld)      // same row stride: one contiguous copy
            e = cudaMemcpyAsync(dst, buf, (size_t)(br * ld * out_elem_bytes), cudaMemcpyDeviceToHost,
                                copy);
        else if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(dst, (size_t)(ld * out_elem_bytes), buf,
                                  (size_t)(L.band_ld * out_elem_bytes),
                                  (size_t)(pl.cols * out_elem_bytes), (size_t)br,
                                  cudaMemcpyDeviceToHost, copy);
        if (e == cudaSuccess) e = cudaEventRecord(copied[k], copy);
    }
    int64_t total = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(copy);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && want_dots) {
        e = cudaMemcpyAsync(&total, running, sizeof total, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        const int64_t keep = std::min(total, dots_cap);
        if (e == cudaSuccess && keep > 0)
            e = cudaMemcpy(dots, ddots, (size_t)keep * sizeof(ap_dot), cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) {
        cudaStreamSynchronize(copy);      // leave the reused copy stream idle
        return fail_cuda(e, "ap_alignment_plot_host");
    }
    if (want_dots) {
        *dots_count = total;
        if (total > dots_cap)
            return fail(AP_E_OVERFLOW, "%lld dots, buffer holds %lld", (long long)total,
                        (long long)dots_cap);
    }
    return AP_OK;
}

}  // extern "C"
