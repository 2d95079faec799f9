// alnplot_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "../../include/alnplot.h"

namespace ap {

// Records a message for ap_last_error() on the calling thread and returns s.
ap_status fail(ap_status s, const char *fmt, ...);
ap_status fail_cuda(cudaError_t e, const char *what);

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
