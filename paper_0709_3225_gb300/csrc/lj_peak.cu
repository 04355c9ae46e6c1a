// lj_measure_peak: the floating-point issue rate the roofline divides by,
// measured on the device at its current clocks.  The paper motivates the
// GPU by its peak floating-point rate against a CPU's (Section 1); here the
// rate is not taken from a datasheet but measured with chains of fused
// multiply-adds (FP32 scalar, FP32 packed pairs, FP64) that keep every
// FMA lane of every SM busy.
//
// Each thread runs kChains independent chains a <- a b + c (b slightly
// below 1, c small: the values stay near 1, no overflow or denormals), so
// consecutive FMAs of a chain are independent of the other chains and the
// pipeline latency is hidden.  The grid is 8 CTAs of 256 threads per SM
// (the SM's 2,048 resident threads).  The chains' sum is stored only if it
// equals an impossible value, which keeps the compiler from removing them
// without any store in practice.
#include <cuda_runtime.h>

#include "lj_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;

__device__ float g_peak_sink32;
__device__ double g_peak_sink64;

__global__ void __launch_bounds__(kThreads) k_peak_ffma(int iters, float b, float c)
{
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; i++) a[i] = 1.0f + 1e-3f * (float)(threadIdx.x + i);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
#pragma unroll
            for (int i = 0; i < kChains; i++) a[i] = fmaf(a[i], b, c);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += a[i];
    if (s == -1.0f) g_peak_sink32 = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_ffma2(int iters, float b, float c)
{
    float2 a[kChains];
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
    for (int i = 0; i < kChains; i++) a[i] = make_float2(1.0f + 1e-3f * (float)(threadIdx.x + i), 1.0f - 1e-3f * (float)i);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
#pragma unroll
            for (int i = 0; i < kChains; i++) a[i] = __ffma2_rn(a[i], b2, c2);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += a[i].x + a[i].y;
    if (s == -1.0f) g_peak_sink32 = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_dfma(int iters, double b, double c)
{
    double a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; i++) a[i] = 1.0 + 1e-3 * (double)(threadIdx.x + i);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
#pragma unroll
            for (int i = 0; i < kChains; i++) a[i] = fma(a[i], b, c);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += a[i];
    if (s == -1.0) g_peak_sink64 = s;
}

cudaError_t launch_peak(int kind, int grid, int iters, cudaStream_t st)
{
    if (kind == 0)
        k_peak_ffma<<<grid, kThreads, 0, st>>>(iters, 0.99999f, 1e-5f);
    else if (kind == 1)
        k_peak_ffma2<<<grid, kThreads, 0, st>>>(iters, 0.99999f, 1e-5f);
    else
        k_peak_dfma<<<grid, kThreads, 0, st>>>(iters, 0.99999, 1e-5);
    return cudaGetLastError();
}

}  // namespace

extern "C" int lj_measure_peak(int32_t kind, double *flops_per_s, double *ms, int32_t *sms)
{
    if (kind < 0 || kind > 2 || !flops_per_s) return LJ_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LJ_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LJ_ECUDA;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int status = LJ_OK;
    const int grid = nsm * kCtasPerSm;
    const double flops_per_iter = 2.0 * (kind == 1 ? 2 : 1) * kChains * kUnroll * (double)grid * kThreads;
    int iters = kind == 2 ? 16 : 256;
    float best = 0.0f, t = 0.0f;
    int best_iters = iters;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return LJ_ECUDA;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        status = LJ_ECUDA;
        goto done;
    }
    // Grow the chain length until one launch takes >= 20 ms, then time three
    // launches of that length and keep the fastest.
    for (int grow = 0; grow < 24; grow++) {
        if (launch_peak(kind, grid, iters, st) != cudaSuccess || cudaEventRecord(e0, st) != cudaSuccess ||
            launch_peak(kind, grid, iters, st) != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            status = LJ_ECUDA;
            goto done;
        }
        if (t >= 20.0f || iters >= (1 << 24)) break;
        iters *= 2;
    }
    best_iters = iters;
    best = t;
    for (int rep = 0; rep < 3; rep++) {
        if (cudaEventRecord(e0, st) != cudaSuccess || launch_peak(kind, grid, iters, st) != cudaSuccess ||
            cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            status = LJ_ECUDA;
            goto done;
        }
        if (t < best) best = t;
    }
    *flops_per_s = flops_per_iter * best_iters / (1e-3 * (double)best);
    if (ms) *ms = best;
    if (sms) *sms = nsm;
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return status;
}
