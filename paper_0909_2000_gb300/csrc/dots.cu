// dots.cu -- thresholded dot lists and plot checksums on the GPU.
//
// A dot plot (Section 1 of the paper) shows one dot per window pair whose
// score passes a threshold.  The dots are produced in row-major order
// (i, then j), deterministically, in three stream-ordered passes over a plot
// region in device memory:
//   1. count the qualifying cells of every row,
//   2. exclusive prefix sum of the row counts (continuing a running device
//      total, so regions processed one after another concatenate in order),
//   3. write every row's dots at its offset; a warp scan over the lanes'
//      hit counts ranks the dots inside each 32 x 16-byte slice of the row.
// Rows are read with 16-byte vector loads when the plot is 16-byte aligned.
#include <cstdint>
#include <cuda_runtime.h>

#include "alnplot_internal.h"

namespace ap {

namespace {

template <typename T>
__device__ __forceinline__ int load_val(const void *plot, int64_t off)
{
    return (int)((const T *)plot)[off];
}

// Loads VEC = 16 / sizeof(T) plot values starting at element j of row `rowp`
// (vector load when `vec`, else element by element, with a bounds check).
template <typename T>
struct Vec16 {
    static constexpr int VEC = 16 / (int)sizeof(T);
    T v[VEC];
    __device__ __forceinline__ void load(const T *rowp, int64_t j, int64_t cols, bool vec)
    {
        if (vec && j + VEC <= cols) {
            const uint4 u = *(const uint4 *)(rowp + j);
            const T *t = (const T *)&u;
#pragma unroll
            for (int k = 0; k < VEC; ++k) v[k] = t[k];
        } else {
#pragma unroll
            for (int k = 0; k < VEC; ++k) v[k] = (j + k < cols) ? rowp[j + k] : (T)0;
        }
    }
};

// One warp per row: number of cells with value >= thr.
template <typename T>
__global__ void row_count_kernel(const void *plot, int64_t rows, int64_t cols, int64_t ld,
                                 int thr, int vec, int32_t *counts)
{
    constexpr int VEC = Vec16<T>::VEC;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < rows; i += nwarps) {
        const T *rowp = (const T *)plot + i * ld;
        int c = 0;
        for (int64_t j = (int64_t)lane * VEC; j < cols; j += 32 * VEC) {
            Vec16<T> q;
            q.load(rowp, j, cols, vec);
#pragma unroll
            for (int k = 0; k < VEC; ++k) c += (int)q.v[k] >= thr && j + k < cols;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) counts[i] = c;
    }
}

// Single-block exclusive scan of counts[0..rows) into offsets (int64),
// starting at *running; *running += total afterwards.
__global__ void scan_kernel(const int32_t *counts, int64_t rows, int64_t *offsets,
                            int64_t *running)
{
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t carry;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) carry = *running;
    __syncthreads();
    for (int64_t b = 0; b < rows; b += blockDim.x) {
        const int64_t i = b + tid;
        int64_t v = (i < rows) ? counts[i] : 0;
        int64_t x = v;   // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) warp_sums[wid] = x;
        __syncthreads();
        if (wid == 0) {
            const int nw = blockDim.x >> 5;
            int64_t s = (lane < nw) ? warp_sums[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int64_t t = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += t;
            }
            if (lane < nw) warp_sums[lane] = s;   // inclusive over warps
        }
        __syncthreads();
        const int64_t before = (wid > 0 ? warp_sums[wid - 1] : 0) + (x - v);
        if (i < rows) offsets[i] = carry + before;
        __syncthreads();
        if (tid == blockDim.x - 1) carry += warp_sums[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (tid == 0) *running = carry;
}

// One warp per row with dots: each lane takes VEC consecutive cells, a warp
// scan of the lanes' hit counts orders the writes, so dots come out in
// column order.  Rows without dots are skipped.
template <typename T>
__global__ void row_write_kernel(const void *plot, int64_t rows, int64_t cols, int64_t ld,
                                 int thr, int vec, const int32_t *counts,
                                 const int64_t *offsets, int64_t row0, ap_dot *dots, int64_t cap)
{
    constexpr int VEC = Vec16<T>::VEC;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < rows; i += nwarps) {
        if (counts[i] == 0) continue;
        int64_t off = offsets[i];
        if (off >= cap) continue;
        const T *rowp = (const T *)plot + i * ld;
        for (int64_t j0 = 0; j0 < cols && off < cap; j0 += 32 * VEC) {
            const int64_t j = j0 + (int64_t)lane * VEC;
            Vec16<T> q;
            q.load(rowp, j, cols, vec);
            int c = 0;
#pragma unroll
            for (int k = 0; k < VEC; ++k) c += (int)q.v[k] >= thr && j + k < cols;
            int x = c;   // inclusive scan over lanes
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += t;
            }
            const int total = __shfl_sync(0xffffffffu, x, 31);
            int64_t k0 = off + (x - c);
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                if ((int)q.v[k] >= thr && j + k < cols) {
                    if (k0 < cap) {
                        ap_dot dt;
                        dt.i = (uint32_t)(row0 + i);
                        dt.j = (uint32_t)(j + k);
                        dt.value = (uint16_t)q.v[k];
                        dt.pad = 0;
                        dots[k0] = dt;
                    }
                    ++k0;
                }
            }
            off += total;
        }
    }
}

template <typename T>
__global__ void checksum_kernel(const void *plot, int64_t rows, int64_t cols, int64_t ld,
                                int nbins, unsigned long long *result)
{
    extern __shared__ unsigned int hist[];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    unsigned long long sum = 0;
    for (int64_t i = blockIdx.x; i < rows; i += gridDim.x) {
        const unsigned long long wi = (unsigned long long)i * 2654435761ull + 1ull;
        const int64_t base = i * ld;
        for (int64_t j = threadIdx.x; j < cols; j += blockDim.x) {
            const int v = load_val<T>(plot, base + j);
            sum += (unsigned long long)v * (wi + (unsigned long long)j * 40503ull);
            if (v < nbins) atomicAdd(&hist[v], 1u);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd(&result[0], sum);
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (hist[b]) atomicAdd(&result[1 + b], (unsigned long long)hist[b]);
}

int grid_for(int64_t rows, int per_block)
{
    int64_t g = (rows + per_block - 1) / per_block;
    if (g > 65535) g = 65535;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

cudaError_t dots_pass(const void *plot, int elem_bytes, int64_t rows, int64_t cols, int64_t ld,
                      int thr, int64_t row0, ap_dot *dots, int64_t cap, int32_t *counts,
                      int64_t *offsets, int64_t *running, cudaStream_t stream)
{
    if (rows <= 0) return cudaSuccess;
    const int threads = 256, rows_per_block = threads / 32;
    const int grid = grid_for(rows, rows_per_block);
    const int vec = ((uintptr_t)plot % 16 == 0) && ((ld * elem_bytes) % 16 == 0);
    if (elem_bytes == 1)
        row_count_kernel<uint8_t><<<grid, threads, 0, stream>>>(plot, rows, cols, ld, thr, vec, counts);
    else
        row_count_kernel<uint16_t><<<grid, threads, 0, stream>>>(plot, rows, cols, ld, thr, vec, counts);
    // offsets are computed relative to the running total before this region
    scan_kernel<<<1, 1024, 0, stream>>>(counts, rows, offsets, running);
    if (cap > 0 && dots) {
        if (elem_bytes == 1)
            row_write_kernel<uint8_t><<<grid, threads, 0, stream>>>(plot, rows, cols, ld, thr, vec,
                                                                   counts, offsets, row0, dots, cap);
        else
            row_write_kernel<uint16_t><<<grid, threads, 0, stream>>>(plot, rows, cols, ld, thr, vec,
                                                                    counts, offsets, row0, dots, cap);
    }
    return cudaGetLastError();
}

cudaError_t checksum_pass(const void *plot, int elem_bytes, int64_t rows, int64_t cols,
                          int64_t ld, int nbins, uint64_t *result, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(result, 0, sizeof(uint64_t) * (size_t)(1 + nbins), stream);
    if (e != cudaSuccess || rows <= 0 || cols <= 0) return e;
    const int grid = grid_for(rows, 1) > 4096 ? 4096 : grid_for(rows, 1);
    const size_t sm = sizeof(unsigned int) * (size_t)(nbins > 0 ? nbins : 1);
    if (elem_bytes == 1)
        checksum_kernel<uint8_t><<<grid, 256, sm, stream>>>(plot, rows, cols, ld, nbins,
                                                           (unsigned long long *)result);
    else
        checksum_kernel<uint16_t><<<grid, 256, sm, stream>>>(plot, rows, cols, ld, nbins,
                                                            (unsigned long long *)result);
    return cudaGetLastError();
}

}  // namespace ap
