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
// Rows are read with 16-byte vector loads (four in flight per thread) when
// the plot is 16-byte aligned, and compared four bytes at a time.
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
// Cells >= thr among the 16 bytes of u, as a per-lane bit mask: bit k set
// iff element k passes (k < 16 for uint8, k < 8 for uint16).
template <typename T>
__device__ __forceinline__ uint32_t ge_mask(uint4 u, uint32_t thr)
{
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
    uint32_t m = 0;
    if (sizeof(T) == 1) {
        const uint32_t t4 = thr > 255u ? 0u : thr * 0x01010101u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t ge = (thr > 255u) ? 0u : __vcmpgeu4(w[q], t4);   // 0xFF per passing byte
            // gather the byte flags into 4 bits
            const uint32_t b = ge & 0x01010101u;
            m |= ((b | (b >> 7) | (b >> 14) | (b >> 21)) & 0xFu) << (4 * q);
        }
    } else {
        const uint32_t t2 = thr > 65535u ? 0u : thr * 0x00010001u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t ge = (thr > 65535u) ? 0u : __vcmpgeu2(w[q], t2);
            const uint32_t b = ge & 0x00010001u;
            m |= ((b | (b >> 15)) & 0x3u) << (2 * q);
        }
    }
    return m;
}

// Elements of the 16-byte slice starting at column j, as a mask of the valid
// ones (columns < cols); `vec` says whether whole 16-byte loads are aligned.
template <typename T>
__device__ __forceinline__ uint4 load16(const T *rowp, int64_t j, int64_t cols, bool vec,
                                        uint32_t *valid)
{
    constexpr int VEC = 16 / (int)sizeof(T);
    uint4 u = make_uint4(0, 0, 0, 0);
    if (j >= cols) {
        *valid = 0;
        return u;
    }
    if (vec && j + VEC <= cols) {
        *valid = (VEC == 16) ? 0xFFFFu : 0xFFu;
        return *(const uint4 *)(rowp + j);
    }
    union {
        uint4 u;
        T t[VEC];
    } w;
    uint32_t v = 0;
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        const bool in = j + k < cols;
        w.t[k] = in ? rowp[j + k] : (T)0;
        v |= (uint32_t)in << k;
    }
    *valid = v;
    return w.u;
}

constexpr int kUnroll = 4;   // 16-byte loads in flight per thread

// One warp per row: number of cells with value >= thr.
template <typename T>
__global__ void row_count_kernel(const void *plot, int64_t rows, int64_t cols, int64_t ld,
                                 int thr, int vec, int32_t *counts)
{
    constexpr int VEC = 16 / (int)sizeof(T);
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t uthr = thr < 0 ? 0u : (uint32_t)thr;
    for (int64_t i = warp; i < rows; i += nwarps) {
        const T *rowp = (const T *)plot + i * ld;
        int c = 0;
        for (int64_t j0 = 0; j0 < cols; j0 += 32 * VEC * kUnroll) {
            uint4 u[kUnroll];
            uint32_t valid[kUnroll];
#pragma unroll
            for (int r = 0; r < kUnroll; ++r)
                u[r] = load16<T>(rowp, j0 + (int64_t)(r * 32 + lane) * VEC, cols, vec, &valid[r]);
#pragma unroll
            for (int r = 0; r < kUnroll; ++r) c += __popc(ge_mask<T>(u[r], uthr) & valid[r]);
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

// One warp per row with dots: each lane takes 16-byte slices, a warp scan of
// the lanes' hit counts orders the writes, so dots come out in column order.
// Rows without dots are skipped.
template <typename T>
__global__ void row_write_kernel(const void *plot, int64_t rows, int64_t cols, int64_t ld,
                                 int thr, int vec, const int32_t *counts,
                                 const int64_t *offsets, int64_t row0, ap_dot *dots, int64_t cap)
{
    constexpr int VEC = 16 / (int)sizeof(T);
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t uthr = thr < 0 ? 0u : (uint32_t)thr;
    for (int64_t i = warp; i < rows; i += nwarps) {
        if (counts[i] == 0) continue;
        int64_t off = offsets[i];
        if (off >= cap) continue;
        const T *rowp = (const T *)plot + i * ld;
        for (int64_t j0 = 0; j0 < cols && off < cap; j0 += 32 * VEC * kUnroll) {
            uint4 u[kUnroll];
            uint32_t valid[kUnroll];
#pragma unroll
            for (int r = 0; r < kUnroll; ++r)
                u[r] = load16<T>(rowp, j0 + (int64_t)(r * 32 + lane) * VEC, cols, vec, &valid[r]);
#pragma unroll
            for (int r = 0; r < kUnroll; ++r) {
                const uint32_t hits = ge_mask<T>(u[r], uthr) & valid[r];
                const int c = __popc(hits);
                int x = c;   // inclusive scan over lanes
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += t;
                }
                const int total = __shfl_sync(0xffffffffu, x, 31);
                int64_t k0 = off + (x - c);
                union {
                    uint4 u;
                    T t[VEC];
                } vals;
                vals.u = u[r];
                const int64_t jb = j0 + (int64_t)(r * 32 + lane) * VEC;
                uint32_t hm = hits;
                while (hm) {
                    const int k = __ffs(hm) - 1;
                    hm &= hm - 1;
                    if (k0 < cap) {
                        ap_dot dt;
                        dt.i = (uint32_t)(row0 + i);
                        dt.j = (uint32_t)(jb + k);
                        dt.value = (uint16_t)vals.t[k];
                        dt.pad = 0;
                        dots[k0] = dt;
                    }
                    ++k0;
                }
                off += total;
            }
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
    NvtxRange range("alnplot: dots pass");
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
    NvtxRange range("alnplot: checksum");
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
