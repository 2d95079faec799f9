// dots_noalloc.cu -- ap_plot_dots_noalloc: the dots of a plot with no device
// allocation at all.
//
// ap_plot_dots needs a caller-allocated workspace for its per-row counts,
// per-row offsets and running total.  Some callers cannot allocate device
// memory: a plug-in that runs inside a host program owning the GPU's memory
// budget, or a service that must not allocate once it has started.  For
// them, this entry point keeps that scratch in one fixed, file-scope device
// array inside the library.  Every GPU that loads the library holds the
// array until the process exits.
#include <cstdio>

#include "alnplot_internal.h"

namespace ap {
namespace {

constexpr int64_t kMaxRows = AP_PLOT_DOTS_NOALLOC_MAX_ROWS;
constexpr int64_t kCountsBytes = kMaxRows * 4;                 // int32 per row
constexpr int64_t kOffsetsOff = (kCountsBytes + 255) / 256 * 256;
constexpr int64_t kOffsetsBytes = kMaxRows * 8;                // int64 per row
constexpr int64_t kRunningOff = kOffsetsOff + (kOffsetsBytes + 255) / 256 * 256;
constexpr int64_t kScratchBytes = kRunningOff + 256;           // running total

// The scratch.  In host code this name is only a host-side stand-in for the
// device array, never a device address: the address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_dots_scratch[kScratchBytes];

// Device address of the scratch in the current context.  It is looked up
// on every call, with the calling thread's device current: the first lookup
// in a context loads this file's module (and with it the array), and a
// lookup per call never hands out an address from a context that
// cudaDeviceReset has since destroyed.  Next to the stream synchronisation
// every call makes, the lookup costs nothing.
ap_status scratch_address(void **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_dots_scratch);
    if (e != cudaSuccess || !p)
        return fail_cuda(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                         "cudaGetSymbolAddress of the static dots scratch");
    *out = p;
    return AP_OK;
}

}  // namespace
}  // namespace ap

using namespace ap;

extern "C" ap_status ap_plot_dots_noalloc(const void *plot, int32_t elem_bytes, int64_t rows,
                                          int64_t cols, int64_t ld, int32_t threshold,
                                          ap_dot *dots, int64_t cap, int64_t *count, void *stream)
{
    if (!count) return fail(AP_E_INVAL, "ap_plot_dots_noalloc: null count pointer");
    if (elem_bytes != 1 && elem_bytes != 2) return fail(AP_E_INVAL, "elem_bytes must be 1 or 2");
    if (rows < 0 || cols < 0 || ld < cols) return fail(AP_E_INVAL, "bad plot shape");
    if (cap < 0 || (cap > 0 && !dots)) return fail(AP_E_INVAL, "bad dot buffer");
    if (rows > kMaxRows)
        return fail(AP_E_NOMEM, "ap_plot_dots_noalloc: %lld plot rows exceed the static scratch "
                    "(at most %lld rows); use ap_plot_dots with a workspace",
                    (long long)rows, (long long)kMaxRows);
    // The address lookup comes before the empty-plot return, so that a call
    // with rows = 0 loads the array on this device without touching a plot:
    // callers warm a device up that way at start-up, before any capture.
    void *base = nullptr;
    ap_status s = scratch_address(&base);
    if (s != AP_OK) return s;
    *count = 0;
    if (rows == 0 || cols == 0) return AP_OK;
    if (!plot) return fail(AP_E_INVAL, "ap_plot_dots_noalloc: null plot");
    char *ws = (char *)base;
    int32_t *counts = (int32_t *)ws;
    int64_t *offsets = (int64_t *)(ws + kOffsetsOff);
    int64_t *running = (int64_t *)(ws + kRunningOff);
    cudaStream_t st = (cudaStream_t)stream;
    // The array keeps the previous call's contents: the running total must
    // start at zero; counts and offsets are overwritten for every row used.
    cudaError_t e = cudaMemsetAsync(running, 0, sizeof(int64_t), st);
    if (e == cudaSuccess)
        e = dots_pass(plot, elem_bytes, rows, cols, ld, threshold, 0, dots, cap, counts, offsets,
                      running, st);
    int64_t total = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, running, sizeof total, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(e, "ap_plot_dots_noalloc");
    *count = total;
    if (total > cap)
        return fail(AP_E_OVERFLOW, "%lld dots, buffer holds %lld", (long long)total,
                    (long long)cap);
    return AP_OK;
}
