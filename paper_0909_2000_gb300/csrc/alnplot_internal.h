// alnplot_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/alnplot.h"

namespace ap {

// Scoped NVTX range around a host-side phase of a call (comb launches, dot
// passes, band copies, batch and server work), for timeline profilers; a
// no-op unless a profiling tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Records a message for ap_last_error() on the calling thread and returns s.
ap_status fail(ap_status s, const char *fmt, ...);
ap_status fail_cuda(cudaError_t e, const char *what);

struct Plan;

// Scores -> blow-up {nu, mu, 0} of the gcd-reduced scheme (nu = 1: LCS) and
// the scale g = gcd(match, mismatch) of the plot; errors for other schemes.
ap_status score_mode(const ap_scores *sc, int *nu, int *mu, int *scale);

// Validated plan of one plot: variant (groups > 0 requests threads per strip
// group, lane_bits > 0 a lane format), tiling (chunk > 0 forces the chunk),
// vertical step (plot row r is the x-window at r * step).
ap_status plan_plot(int64_t m, int64_t n, int32_t w, const ap_scores *scores, int groups,
                    int64_t chunk, Plan *pl, int64_t step = 1, int lane_bits = 0);

// Output-argument checks shared by the plain and batched calls.
ap_status check_output(const Plan &pl, const void *x, const void *y, const void *out,
                       int32_t out_elem_bytes, int64_t ld);

int current_device();

// Band height (plot rows) of the banded calls: `automatic` unless
// ap_set_band_rows has forced one; whole strip groups of `spw` strips, at
// most the plot's rows rounded up to a strip group.
int64_t band_rows_for(int64_t automatic, int64_t spw, int64_t rows);

// Dots of a plot region [rows x cols] (ld elements per row) in row-major order,
// appended after *running dots; *running (device) grows by the region's count.
// counts: device, rows int32; offsets: device, rows int64.
cudaError_t dots_pass(const void *plot, int elem_bytes, int64_t rows, int64_t cols, int64_t ld,
                      int thr, int64_t row0, ap_dot *dots, int64_t cap, int32_t *counts,
                      int64_t *offsets, int64_t *running, cudaStream_t stream);

// result[0] = checksum, result[1 + v] = count of value v (v < nbins).
cudaError_t checksum_pass(const void *plot, int elem_bytes, int64_t rows, int64_t cols,
                          int64_t ld, int nbins, uint64_t *result, cudaStream_t stream);

}  // namespace ap
