// Micro-benchmarks for the roofline denominators of the pair sums: FP32 FMA
// throughput issued as scalar FFMA and as packed f32x2 FMA, and the MUFU
// reciprocal-square-root rate. Independent dependency chains per thread keep
// the pipes full; results feed a value that is stored only under an
// impossible condition so that nothing is optimised away.
#include "kernels.h"

namespace nb {

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) ffma_peak_kernel(float *sink, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -12345.678f) sink[0] = s;
}

__global__ void __launch_bounds__(256) ffma2_peak_kernel(float *sink, int iters, float a, float b) {
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2(threadIdx.x * 1e-3f + c, c + 0.5f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == -12345.678f) sink[0] = s;
}

__global__ void __launch_bounds__(256) mufu_peak_kernel(float *sink, int iters) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.5f + threadIdx.x * 1e-3f + c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = rsqrtf(x[c]);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -12345.678f) sink[0] = s;
}

}  // namespace

// out[0] FP32 TFLOP/s with scalar FFMA, out[1] with packed f32x2 FMA,
// out[2] MUFU rsqrt Gop/s. One launch each, `blocks` CTAs of 256 threads.
cudaError_t measure_peaks(int blocks, float *sink, cudaStream_t st, double out[3]) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) return e;
    const int iters = 4096;
    const double thr = (double)blocks * 256;
    double per[3] = {thr * iters * kUnroll * kChains * 2.0, thr * iters * kUnroll * kChains * 4.0,
                     thr * iters * kUnroll * kChains};
    for (int k = 0; k < 3; ++k) {
        for (int rep = 0; rep < 2; ++rep) {  // first launch warms up
            cudaEventRecord(e0, st);
            if (k == 0) ffma_peak_kernel<<<blocks, 256, 0, st>>>(sink, iters, 0.999f, 1e-3f);
            if (k == 1) ffma2_peak_kernel<<<blocks, 256, 0, st>>>(sink, iters, 0.999f, 1e-3f);
            if (k == 2) mufu_peak_kernel<<<blocks, 256, 0, st>>>(sink, iters);
            cudaEventRecord(e1, st);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        out[k] = per[k] / (ms * 1e-3) / (k == 2 ? 1e9 : 1e12);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cudaGetLastError();
}

}  // namespace nb
