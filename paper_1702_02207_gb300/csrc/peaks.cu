// peaks.cu -- measured arithmetic peaks of the CUDA cores, the denominators of the
// "alu" roofline fractions of the batched RK4 kernels.
//
// Every thread of a full-occupancy grid (a whole number of CTAs per SM on every SM)
// runs NCH independent fused multiply-add chains for `iters` rounds: scalar FP32
// (fma.rn.f32), packed FP32 pairs (fma.rn.f32x2, two FMAs per instruction) or FP64
// (fma.rn.f64).  Independent chains hide the pipe latency, so the rate is the pipe's
// throughput; the loop body is unrolled so that loop control takes a few percent of
// the issue slots.  The chain values stay finite (a <- a * b + c with b < 1) and one
// thread's sum is stored only if it equals an impossible value, so nothing is
// eliminated and nothing is written.  Timed with CUDA events on a private stream
// after one warm-up launch; flop = 2 per FMA.
#include "../../include/cho.h"
#include "ctx.h"

namespace cho {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kUnroll = 16;

// Where a thread would store its sum if it ever reached the impossible value: static
// device memory of one CTA's size, so the measurement allocates nothing.
__device__ float g_sink32[kPeakThreads];
__device__ double g_sink64[kPeakThreads];

template <int NCH>
__global__ void __launch_bounds__(kPeakThreads) fma_f32_kernel(float* sink, float b, float c, int iters)
{
    float a[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) a[k] = 1e-3f * (float)threadIdx.x + (float)k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < NCH; ++k) a[k] = __fmaf_rn(a[k], b, c);
    }
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < NCH; ++k) sum += a[k];
    if (sum == -1.2345e30f) sink[threadIdx.x] = sum;
}

template <int NCH>
__global__ void __launch_bounds__(kPeakThreads) fma_f32x2_kernel(float* sink, float b, float c, int iters)
{
    float2 a[NCH];
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll
    for (int k = 0; k < NCH; ++k) a[k] = make_float2(1e-3f * (float)threadIdx.x + (float)k, (float)k - 0.5f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < NCH; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
    }
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < NCH; ++k) sum += a[k].x + a[k].y;
    if (sum == -1.2345e30f) sink[threadIdx.x] = sum;
}

template <int NCH>
__global__ void __launch_bounds__(kPeakThreads) fma_f64_kernel(double* sink, double b, double c, int iters)
{
    double a[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) a[k] = 1e-3 * (double)threadIdx.x + (double)k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < NCH; ++k) a[k] = __fma_rn(a[k], b, c);
    }
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < NCH; ++k) sum += a[k];
    if (sum == -1.2345e300) sink[threadIdx.x] = sum;
}

}  // namespace
}  // namespace cho

using namespace cho;

extern "C" cho_status cho_measure_fma_peak(cho_ctx* ctx, int32_t kind, int32_t iters, double* flops_per_s,
                                           double* seconds)
{
    clear_error();
    if (!ctx || !flops_per_s) return fail(CHO_EINVAL, "cho_measure_fma_peak: NULL argument");
    if (kind < 0 || kind > 2) return fail(CHO_EINVAL, "cho_measure_fma_peak: kind must be 0, 1 or 2");
    if (iters <= 0) return fail(CHO_EINVAL, "cho_measure_fma_peak: iters must be > 0");
    DeviceGuard g(ctx->device);
    if (!g.ok()) return fail(CHO_ECUDA, "cho_measure_fma_peak: cudaSetDevice failed");
    constexpr int NCH = 8;
    int per_sm = 0;
    cudaError_t e = cudaSuccess;
    if (kind == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_f32_kernel<NCH>, kPeakThreads, 0);
    if (kind == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_f32x2_kernel<NCH>, kPeakThreads, 0);
    if (kind == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_f64_kernel<NCH>, kPeakThreads, 0);
    if (e != cudaSuccess || per_sm <= 0) return fail(CHO_ECUDA, "cho_measure_fma_peak: occupancy query failed");
    const int grid = per_sm * ctx->sm_count;
    float* sink32 = nullptr;
    double* sink64 = nullptr;
    e = cudaGetSymbolAddress((void**)&sink32, g_sink32);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&sink64, g_sink64);
    if (e != cudaSuccess) return fail(CHO_ECUDA, "cho_measure_fma_peak: %s", cudaGetErrorString(e));
    cudaStream_t st = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {     // warm-up launch, then the timed one
        e = cudaEventRecord(ev[0], st);
        if (kind == 0) fma_f32_kernel<NCH><<<grid, kPeakThreads, 0, st>>>(sink32, 0.9999999f, 1e-7f, iters);
        if (kind == 1) fma_f32x2_kernel<NCH><<<grid, kPeakThreads, 0, st>>>(sink32, 0.9999999f, 1e-7f, iters);
        if (kind == 2) fma_f64_kernel<NCH><<<grid, kPeakThreads, 0, st>>>(sink64, 0.9999999, 1e-7, iters);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    }
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return fail(CHO_ECUDA, "cho_measure_fma_peak: %s", cudaGetErrorString(e));
    const double fma_per_thread = (double)iters * kUnroll * NCH * (kind == 1 ? 2.0 : 1.0);
    const double t = ms * 1e-3;
    *flops_per_s = 2.0 * fma_per_thread * (double)grid * kPeakThreads / t;
    if (seconds) *seconds = t;
    return CHO_OK;
}
