// int_probe.cu -- ap_int_issue_probe: the integer issue rate of this GPU, the
// denominator of the comb kernel's roofline, measured rather than assumed.
//
// Every thread keeps eight accumulators and updates each, per iteration,
// from two others with one three-input logic instruction (lop3), one
// multiply-add (mad.lo) or alternately one and the other.  The operands are
// all live accumulators, so nothing folds away; eight independent updates a
// thread and a full SM of warps hide the latencies, leaving the issue and
// pipe rates as the limit.
#include "alnplot_internal.h"

namespace ap {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;   // 64 warps an SM
constexpr int kProbeMaxBlocks = 4096;  // up to 512 SMs

// One word per block, written only when a thread's accumulators fold to the
// seed (so that the compiler keeps the work); 16 KB held by the library.
__device__ uint32_t g_probe_sink[kProbeMaxBlocks];

__device__ __forceinline__ uint32_t probe_lop3(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

__device__ __forceinline__ uint32_t probe_mad(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) int_probe_kernel(uint32_t *sink, int64_t iters, uint32_t seed)
{
    uint32_t a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed ^ (threadIdx.x * 2654435761u) ^ (uint32_t)(k * 40503);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t b = a[(k + 1) & 7], c = a[(k + 2) & 7];
            const bool mad = KIND == 1 || (KIND == 2 && (k & 1));
            a[k] = mad ? probe_mad(a[k], b, c) : probe_lop3(a[k], b, c);
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r ^= a[k];
    if (r == seed) sink[blockIdx.x] = r;   // keeps the results live; almost never taken
}

}  // namespace
}  // namespace ap

extern "C" ap_status ap_int_issue_probe(int32_t kind, int64_t iters, double *lane_ops_per_s)
{
    using namespace ap;
    if (!lane_ops_per_s) return fail(AP_E_INVAL, "ap_int_issue_probe: null result pointer");
    *lane_ops_per_s = 0.0;
    if (kind < 0 || kind > 2 || iters < 1)
        return fail(AP_E_INVAL, "ap_int_issue_probe: kind %d (0..2), iters %lld (>= 1)", kind, (long long)iters);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail_cuda(e, "ap_int_issue_probe: device query");
    const int blocks = sms * kProbeBlocksPerSm;
    void (*fn)(uint32_t *, int64_t, uint32_t) =
        kind == 0 ? int_probe_kernel<0> : (kind == 1 ? int_probe_kernel<1> : int_probe_kernel<2>);
    if (blocks > kProbeMaxBlocks)
        return fail(AP_E_UNSUPPORTED, "ap_int_issue_probe: %d SMs exceed the probe's sink", sms);
    uint32_t *sink = nullptr;
    e = cudaGetSymbolAddress((void **)&sink, g_probe_sink);
    if (e != cudaSuccess) return fail_cuda(e, "ap_int_issue_probe: sink address");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        fn<<<blocks, kProbeThreads>>>(sink, 1, 1u);   // warm-up (module load, clocks)
        e = cudaEventRecord(e0);
    }
    if (e == cudaSuccess) {
        fn<<<blocks, kProbeThreads>>>(sink, iters, 0x9E3779B9u);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail_cuda(e, "ap_int_issue_probe");
    *lane_ops_per_s = (double)blocks * kProbeThreads * (double)iters * 8.0 / (ms * 1e-3);
    return AP_OK;
}
